// Near part of the Stokes double layer (and of its evaluation at points):
// for one (target, source particle) pair,
//     D_stk_i = -X_i sum_j d_j D[q_j] + sum_j d_j D[y_i q_j] - d_i S[q . nu]
// (X the target relative to the source centre, global frame).  The thirteen
// expansions (order P1 = p + 1) are stored with the density index j turned
// into the source's local frame (q_l = sum_j R_jl q_j, y_i q_l likewise), so
// that the two divergences are local-frame divergences,
//     sum_j d_j D[q_j] = sum_l d'_l D[q_l],   sum_j d_j D[y_i q_j] = sum_l d'_l D[y_i q_l],
// and one pass of solid_terms serves them all: each term's local Cartesian
// gradient (cos and sin parts) is formed once and contracted with the
// coefficients of the four vector fields (3 components each) and of S[q . nu],
// whose local gradient is rotated to the global frame at the end.  The
// source's own nodes are evaluated separably (sdl_self_kernel).
#pragma once

#include "sbio_grad.cuh"

namespace sbio {

template <int NC>
struct SdlNearVisitor {
  const double* __restrict__ cf;   // 13 x NC: q_l (0..2), y_i q_l (3 + 3i + l), q . nu (12)
  double k_ru, k_rv, k_zu, k_zv, k_p, c1, s1;
  double cm, sm, tcc, tss, tsc, tcs;
  double div, t2[3], gS[3];

  __device__ __forceinline__ void begin(const GradFrame& f) {
    k_ru = f.k_ru; k_rv = f.k_rv; k_zu = f.k_zu; k_zv = f.k_zv; k_p = f.k_p; c1 = f.c1; s1 = f.s1;
    div = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l) t2[l] = gS[l] = 0.0;
  }
  __device__ __forceinline__ void order(int, double c, double s) {
    cm = c; sm = s;
    tcc = c1 * c; tss = s1 * s; tsc = s1 * c; tcs = c1 * s;
  }
  // acc += sum over the three components l of field (base + l) of its
  // coefficients times gradient component l (FMAs straight into acc)
  __device__ __forceinline__ void field(double& acc, int base, int kc, int ks, const double* Bc,
                                        const double* Bs) const {
#pragma unroll
    for (int l = 0; l < 3; ++l) acc = fma(cf[(base + l) * NC + kc], Bc[l], fma(cf[(base + l) * NC + ks], Bs[l], acc));
  }
  __device__ __forceinline__ void term(int n, int m, double, double Tu, double Tv, double Tp) {
    const double al = fma(k_ru, Tu, k_rv * Tv), z = fma(k_zu, Tu, k_zv * Tv), g = k_p * Tp;
    const double Bc[3] = {fma(al, tcc, g * tss), fma(al, tsc, -g * tcs), z * cm};
    const double Bs[3] = {fma(al, tcs, -g * tsc), fma(al, tss, g * tcc), z * sm};
    const int kc = n * n + n + m, ks = n * n + n - m;
    field(div, 0, kc, ks, Bc, Bs);
#pragma unroll
    for (int i = 0; i < 3; ++i) field(t2[i], 3 + 3 * i, kc, ks, Bc, Bs);
#pragma unroll
    for (int l = 0; l < 3; ++l) gS[l] = fma(cf[12 * NC + kc], Bc[l], fma(cf[12 * NC + ks], Bs[l], gS[l]));
  }
  __device__ __forceinline__ void term0(int n, double, double Tu, double Tv) {
    const double al = fma(k_ru, Tu, k_rv * Tv), z = fma(k_zu, Tu, k_zv * Tv);
    const double B[3] = {c1 * al, s1 * al, z};
    const int k = n * n + n;
#pragma unroll
    for (int l = 0; l < 3; ++l) div = fma(cf[l * NC + k], B[l], div);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int l = 0; l < 3; ++l) t2[i] = fma(cf[(3 + 3 * i + l) * NC + k], B[l], t2[i]);
#pragma unroll
    for (int l = 0; l < 3; ++l) gS[l] = fma(cf[12 * NC + k], B[l], gS[l]);
  }
};

template <int P1, int KIND>
__global__ void __launch_bounds__(kNearGradBlock) stokes_dl_near_kernel(const int32_t* __restrict__ pair_t,
                                                             const int32_t* __restrict__ pair_s, int64_t first,
                                                             int64_t count, const PartGeom* __restrict__ parts,
                                                             const double* __restrict__ xyz,
                                                             const double* __restrict__ coef,
                                                             const double* __restrict__ inv_tab,
                                                             double* __restrict__ u_out) {
  constexpr int NC = (P1 + 1) * (P1 + 1);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = first + r;
    const int t = pair_t[idx], i = pair_s[idx];
    const PartGeom& G = parts[i];
    const double X0 = xyz[(int64_t)t * 3 + 0] - G.c[0];
    const double X1 = xyz[(int64_t)t * 3 + 1] - G.c[1];
    const double X2 = xyz[(int64_t)t * 3 + 2] - G.c[2];
    const double xl = G.R[0] * X0 + G.R[3] * X1 + G.R[6] * X2;
    const double yl = G.R[1] * X0 + G.R[4] * X1 + G.R[7] * X2;
    const double zl = G.R[2] * X0 + G.R[5] * X1 + G.R[8] * X2;
    SdlNearVisitor<NC> vis;
    vis.cf = coef + (size_t)i * 13 * NC;
    solid_terms<P1, KIND>(xl, yl, zl, G.a, inv_tab, vis);
    const double* R = G.R;
    double t3[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t3[k] = R[k * 3 + 0] * vis.gS[0] + R[k * 3 + 1] * vis.gS[1] + R[k * 3 + 2] * vis.gS[2];
    atomicAdd(u_out + (int64_t)t * 3 + 0, -X0 * vis.div + vis.t2[0] - t3[0]);
    atomicAdd(u_out + (int64_t)t * 3 + 1, -X1 * vis.div + vis.t2[1] - t3[1]);
    atomicAdd(u_out + (int64_t)t * 3 + 2, -X2 * vis.div + vis.t2[2] - t3[2]);
  }
}

typedef void (*stokes_dl_near_launcher)(const DevGeom&, const int32_t*, const int32_t*, int64_t, int64_t, double*,
                                        cudaStream_t);

template <int P1, int KIND>
static void launch_stokes_dl_near_pk(const DevGeom& d, const int32_t* pt, const int32_t* ps, int64_t first,
                                     int64_t count, double* u, cudaStream_t st) {
  if (count <= 0) return;
  int64_t nb = (count + kNearGradBlock - 1) / kNearGradBlock;
  if (d.near_grid_cap > 0 && nb > d.near_grid_cap) nb = d.near_grid_cap;
  stokes_dl_near_kernel<P1, KIND><<<(unsigned)nb, kNearGradBlock, 0, st>>>(pt, ps, first, count, d.parts, d.xyz, d.sdl_coef,
                                                                d.inv, u);
  count_launch();
}

// pairs [0, n_pro) have prolate sources, [n_pro, n_all) oblate
template <int P1>
static void launch_stokes_dl_near_p(const DevGeom& d, const int32_t* pt, const int32_t* ps, int64_t n_pro,
                                    int64_t n_all, double* u, cudaStream_t st) {
  launch_stokes_dl_near_pk<P1, SBIO_PROLATE>(d, pt, ps, 0, n_pro, u, st);
  launch_stokes_dl_near_pk<P1, SBIO_OBLATE>(d, pt, ps, n_pro, n_all - n_pro, u, st);
}

template <int... Ps>
struct StokesDLNearTable {
  static stokes_dl_near_launcher get(int p) {
    stokes_dl_near_launcher tab[] = {launch_stokes_dl_near_p<Ps + 1>...};
    int ps[] = {Ps...};
    for (size_t k = 0; k < sizeof(ps) / sizeof(int); ++k)
      if (ps[k] == p) return tab[k];
    return nullptr;
  }
};

}  // namespace sbio
