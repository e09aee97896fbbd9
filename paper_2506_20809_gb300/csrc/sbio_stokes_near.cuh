// Near and self part of the Stokes single layer (Sec. 4.3, eq. (stokes)) for
// one (target, source particle) pair.  Four Laplace single-layer expansions of
// the source (densities f_1, f_2, f_3 and y . f, all carried to order P1 = p+1,
// exterior factor of Theorem 2, normalisation and sqrt 2 folded into `coef`)
// are evaluated with their gradients at the target:
//     F   = sum alpha q_n^|m|(u) Pbar_n^|m|(v) trig_m(phi)
//     grad F = e_u dF/du / h_u + e_v dF/dv / h_v + e_phi dF/dphi / h_phi
// (the directional derivatives of eq. (dSLevalformula) for the Cartesian unit
// vectors).  Near the source axis the v- and phi-derivatives use the
// regularised forms sqrt(1-v^2) dPbar/dv = (n+1) v D_n - (n-m+1) D_{n+1} and
// m Pbar/sqrt(1-v^2) = m D_n with D_n^m = Pbar_n^m / sqrt(1-v^2) (m >= 1), and
// sqrt(1-v^2) dP_n/dv = Pbar_n^1 for m = 0.  The velocity is then
//     u = 1/2 { (F_1, F_2, F_3) + R [ grad F_y - sum_j X_j grad F_j ] }
// with X the target relative to the source centre (global frame) and the
// gradients in the source's local frame.  Since X is fixed per pair, the
// bracket is the gradient of the single expansion F_y - sum_j X_j F_j, whose
// coefficients are formed term by term (one gradient instead of four).
#pragma once

#include "sbio_internal.cuh"
#include "sbio_near.cuh"
#include "sbio_grad.cuh"

namespace sbio {

// Values of S[f_1..3] and local-frame partial sums of the gradient of the one
// combined expansion H = S[y . f] - sum_j X_j S[f_j] (X fixed per pair), so
// that grad S[y . f] - sum_j X_j grad S[f_j] = grad H costs one gradient.
template <int NC>
struct StokesNearVisitor {
  const double* __restrict__ cf;   // 4 x NC: f_1, f_2, f_3, y . f
  double X0, X1, X2;
  double cm, sm;
  double F[3], Hu, Hv, Hp;
  GradFrame fr;

  __device__ __forceinline__ void begin(const GradFrame& f) {
    fr = f;
    F[0] = F[1] = F[2] = Hu = Hv = Hp = 0.0;
  }
  __device__ __forceinline__ void order(int, double c, double s) {
    cm = c;
    sm = s;
  }
  __device__ __forceinline__ double h(int k) const {
    return fma(-X2, cf[2 * NC + k], fma(-X1, cf[NC + k], fma(-X0, cf[k], cf[3 * NC + k])));
  }
  __device__ __forceinline__ void term(int n, int m, double T, double Tu, double Tv, double Tp) {
    const int kc = n * n + n + m, ks = n * n + n - m;
    const double hc = h(kc), hs = h(ks);
    const double a = fma(hc, cm, hs * sm), b = fma(hs, cm, -hc * sm);   // cos / d-phi parts
    Hu = fma(a, Tu, Hu);
    Hv = fma(a, Tv, Hv);
    Hp = fma(b, Tp, Hp);
    const double Tc = T * cm, Ts = T * sm;
#pragma unroll
    for (int j = 0; j < 3; ++j) F[j] = fma(cf[j * NC + kc], Tc, fma(cf[j * NC + ks], Ts, F[j]));
  }
  __device__ __forceinline__ void term0(int n, double T, double Tu, double Tv) {
    const int k = n * n + n;
    const double hk = h(k);
    Hu = fma(hk, Tu, Hu);
    Hv = fma(hk, Tv, Hv);
#pragma unroll
    for (int j = 0; j < 3; ++j) F[j] = fma(cf[j * NC + k], T, F[j]);
  }
};

template <int P1, int KIND>
__device__ __forceinline__ void stokes_pair(double xl, double yl, double zl, double a, const double* __restrict__ R,
                                            double X0, double X1, double X2, const double* __restrict__ coef,
                                            const double* __restrict__ inv_tab, double out[3]) {
  constexpr int NC = (P1 + 1) * (P1 + 1);
  StokesNearVisitor<NC> vis;
  vis.cf = coef;
  vis.X0 = X0;
  vis.X1 = X1;
  vis.X2 = X2;
  solid_terms<P1, KIND>(xl, yl, zl, a, inv_tab, vis);
  const GradFrame& f = vis.fr;
  const double rho = fma(f.k_ru, vis.Hu, f.k_rv * vis.Hv), ph = f.k_p * vis.Hp;
  const double w[3] = {f.c1 * rho - f.s1 * ph, f.s1 * rho + f.c1 * ph, fma(f.k_zu, vis.Hu, f.k_zv * vis.Hv)};
#pragma unroll
  for (int k = 0; k < 3; ++k)
    out[k] = 0.5 * (vis.F[k] + R[k * 3 + 0] * w[0] + R[k * 3 + 1] * w[1] + R[k * 3 + 2] * w[2]);
}

template <int P1, int KIND>
__global__ void __launch_bounds__(kNearGradBlock) stokes_near_kernel(const int32_t* __restrict__ pair_t,
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
    double o[3];
    stokes_pair<P1, KIND>(xl, yl, zl, G.a, G.R, X0, X1, X2, coef + (size_t)i * 4 * NC, inv_tab, o);
    atomicAdd(u_out + (int64_t)t * 3 + 0, o[0]);
    atomicAdd(u_out + (int64_t)t * 3 + 1, o[1]);
    atomicAdd(u_out + (int64_t)t * 3 + 2, o[2]);
  }
}

typedef void (*stokes_near_launcher)(const DevGeom&, int64_t, int64_t, const double*, double*, cudaStream_t);

template <int P1, int KIND>
static void launch_stokes_near_pk(const DevGeom& d, int64_t first, int64_t count, const double* inv, double* u,
                                  cudaStream_t st) {
  if (count <= 0) return;
  int64_t nb = (count + kNearGradBlock - 1) / kNearGradBlock;
  if (d.near_grid_cap > 0 && nb > d.near_grid_cap) nb = d.near_grid_cap;
  const unsigned blocks = (unsigned)nb;
  stokes_near_kernel<P1, KIND><<<blocks, kNearGradBlock, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts, d.xyz,
                                                        d.st_coef, inv, u);
  count_launch();
}

template <int P1>
static void launch_stokes_near_p(const DevGeom& d, int64_t n_pro, int64_t n_all, const double* inv, double* u,
                                 cudaStream_t st) {
  launch_stokes_near_pk<P1, SBIO_PROLATE>(d, 0, n_pro, inv, u, st);
  launch_stokes_near_pk<P1, SBIO_OBLATE>(d, n_pro, n_all - n_pro, inv, u, st);
}

template <int... Ps>
struct StokesNearTable {
  static stokes_near_launcher get(int p) {
    stokes_near_launcher tab[] = {launch_stokes_near_p<Ps + 1>...};
    int ps[] = {Ps...};
    for (size_t k = 0; k < sizeof(ps) / sizeof(int); ++k)
      if (ps[k] == p) return tab[k];
    return nullptr;
  }
};

}  // namespace sbio
