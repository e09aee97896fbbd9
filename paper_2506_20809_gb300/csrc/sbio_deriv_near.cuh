// Near part of the normal-derivative operators S' and D' (Sec. 3.3, eq.
// (dSLevalformula); Sec. 4.2 "Other layer potentials"): for a target node on
// another particle the normal at the target has u, v and phi components in
// the source's frame, so the gradient of the source's exterior expansions of
// S[sigma] and D[mu] (coefficients alpha, beta with the exterior factors of
// Theorems 1-2 folded in) is dotted with the target's outward normal.  One
// thread per (target, near source) pair, FP64, fully unrolled per order p.
#pragma once

#include "sbio_grad.cuh"

namespace sbio {

// Gradient dotted with the target's direction, term by term: with nl the
// direction in the source's frame, n_rho = c1 nl_x + s1 nl_y and
// n_phi = c1 nl_y - s1 nl_x, the directional derivative of a term is
// K_u Tu + K_v Tv (+ K_p Tp for the phi-derivative of its trig factor) with
// K_u = n_rho k_ru + nl_z k_zu, K_v = n_rho k_rv + nl_z k_zv, K_p = n_phi k_p.
template <bool DO_S, bool DO_D>
struct DerivNearVisitor {
  const double* __restrict__ alpha;
  const double* __restrict__ beta;
  double nl0, nl1, nl2;
  double Ku, Kv, Kp, cm, sm;
  double Sp, Dp;

  __device__ __forceinline__ void begin(const GradFrame& f) {
    const double nr = f.c1 * nl0 + f.s1 * nl1, np = f.c1 * nl1 - f.s1 * nl0;
    Ku = fma(nr, f.k_ru, nl2 * f.k_zu);
    Kv = fma(nr, f.k_rv, nl2 * f.k_zv);
    Kp = np * f.k_p;
    Sp = Dp = 0.0;
  }
  __device__ __forceinline__ void order(int, double c, double s) {
    cm = c;
    sm = s;
  }
  __device__ __forceinline__ void term(int n, int m, double, double Tu, double Tv, double Tp) {
    const double bn = fma(Ku, Tu, Kv * Tv), bp = Kp * Tp;
    const double Bc = fma(bn, cm, -bp * sm), Bs = fma(bn, sm, bp * cm);
    const int kc = n * n + n + m, ks = n * n + n - m;
    if (DO_S) Sp = fma(alpha[kc], Bc, fma(alpha[ks], Bs, Sp));
    if (DO_D) Dp = fma(beta[kc], Bc, fma(beta[ks], Bs, Dp));
  }
  __device__ __forceinline__ void term0(int n, double, double Tu, double Tv) {
    const double B = fma(Ku, Tu, Kv * Tv);
    const int k = n * n + n;
    if (DO_S) Sp = fma(alpha[k], B, Sp);
    if (DO_D) Dp = fma(beta[k], B, Dp);
  }
};

template <int P, int KIND, bool DO_S, bool DO_D>
__global__ void __launch_bounds__(128) deriv_near_kernel(const int32_t* __restrict__ pair_t,
                                                         const int32_t* __restrict__ pair_s, int64_t first,
                                                         int64_t count, const PartGeom* __restrict__ parts,
                                                         const double* __restrict__ xyz,
                                                         const double* __restrict__ nrm,
                                                         const double* __restrict__ alpha,
                                                         const double* __restrict__ beta,
                                                         const double* __restrict__ inv_tab,
                                                         double* __restrict__ Sp_out, double* __restrict__ Dp_out) {
  constexpr int NC = (P + 1) * (P + 1);
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
    const double n0 = nrm[(int64_t)t * 3 + 0], n1 = nrm[(int64_t)t * 3 + 1], n2 = nrm[(int64_t)t * 3 + 2];
    DerivNearVisitor<DO_S, DO_D> vis;
    vis.alpha = alpha + (size_t)i * NC;
    vis.beta = beta + (size_t)i * NC;
    // target direction in the source's local frame
    vis.nl0 = G.R[0] * n0 + G.R[3] * n1 + G.R[6] * n2;
    vis.nl1 = G.R[1] * n0 + G.R[4] * n1 + G.R[7] * n2;
    vis.nl2 = G.R[2] * n0 + G.R[5] * n1 + G.R[8] * n2;
    solid_terms<P, KIND>(xl, yl, zl, G.a, inv_tab, vis);
    if (DO_S) atomicAdd(Sp_out + t, vis.Sp);
    if (DO_D) atomicAdd(Dp_out + t, vis.Dp);
  }
}

typedef void (*deriv_near_launcher)(const DevGeom&, int64_t, int64_t, double*, double*, cudaStream_t);

template <int P, int KIND>
static void launch_deriv_near_pk(const DevGeom& d, int64_t first, int64_t count, double* Sp, double* Dp,
                                 cudaStream_t st) {
  if (count <= 0) return;
  int64_t nb = (count + 127) / 128;
  if (d.near_grid_cap > 0 && nb > d.near_grid_cap) nb = d.near_grid_cap;
  const unsigned blocks = (unsigned)nb;
  if (Sp && Dp)
    deriv_near_kernel<P, KIND, true, true><<<blocks, 128, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts, d.xyz,
                                                                   d.nrm, d.alpha, d.beta, d.inv, Sp, Dp);
  else if (Sp)
    deriv_near_kernel<P, KIND, true, false><<<blocks, 128, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts,
                                                                    d.xyz, d.nrm, d.alpha, d.beta, d.inv, Sp, Dp);
  else
    deriv_near_kernel<P, KIND, false, true><<<blocks, 128, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts,
                                                                    d.xyz, d.nrm, d.alpha, d.beta, d.inv, Sp, Dp);
  count_launch();
}

template <int P>
static void launch_deriv_near_p(const DevGeom& d, int64_t n_pro, int64_t n_all, double* Sp, double* Dp,
                                cudaStream_t st) {
  launch_deriv_near_pk<P, SBIO_PROLATE>(d, 0, n_pro, Sp, Dp, st);
  launch_deriv_near_pk<P, SBIO_OBLATE>(d, n_pro, n_all - n_pro, Sp, Dp, st);
}

template <int... Ps>
struct DerivNearTable {
  static deriv_near_launcher get(int p) {
    deriv_near_launcher tab[] = {launch_deriv_near_p<Ps>...};
    int ps[] = {Ps...};
    for (size_t k = 0; k < sizeof(ps) / sizeof(int); ++k)
      if (ps[k] == p) return tab[k];
    return nullptr;
  }
};

}  // namespace sbio
