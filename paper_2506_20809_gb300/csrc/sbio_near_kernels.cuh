// Near-field kernel templates and their launchers; instantiated for ranges of
// the expansion order p in the sbio_near_p*.cu translation units so that the
// fully unrolled variants compile in parallel.
#pragma once

#include <cmath>

#include "sbio_internal.cuh"
#include "sbio_near.cuh"

namespace sbio {

// ---------------------------------------------------------------------------
// near: one thread per (target, near source) pair
// ---------------------------------------------------------------------------
template <int P, int KIND, bool DO_S, bool DO_D>
__global__ void __launch_bounds__(128) near_kernel(const int32_t* __restrict__ pair_t,
                                                   const int32_t* __restrict__ pair_s, int64_t first, int64_t count,
                                                   const PartGeom* __restrict__ parts, const double* __restrict__ xyz,
                                                   const double* __restrict__ alpha,
                                                   const double* __restrict__ beta,
                                                   const double* __restrict__ inv_tab, double* __restrict__ S_out,
                                                   double* __restrict__ D_out) {
  // grid-stride over the pairs: a capped grid lets the near kernel share the
  // SMs with a concurrently running far-field kernel
  constexpr int NC = (P + 1) * (P + 1);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = first + r;
    const int t = pair_t[idx], i = pair_s[idx];
    const PartGeom& G = parts[i];
    const double dx = xyz[(int64_t)t * 3 + 0] - G.c[0];
    const double dy = xyz[(int64_t)t * 3 + 1] - G.c[1];
    const double dz = xyz[(int64_t)t * 3 + 2] - G.c[2];
    const double xl = G.R[0] * dx + G.R[3] * dy + G.R[6] * dz;
    const double yl = G.R[1] * dx + G.R[4] * dy + G.R[7] * dz;
    const double zl = G.R[2] * dx + G.R[5] * dy + G.R[8] * dz;
    double S, D;
    near_pair<P, KIND, DO_S, DO_D>(xl, yl, zl, G.a, alpha + (size_t)i * NC, beta + (size_t)i * NC, inv_tab, S, D);
    if (DO_S) atomicAdd(S_out + t, S);
    if (DO_D) atomicAdd(D_out + t, D);
  }
}

// The mixed-precision form (near_pair_mixed): FP32 coefficients, the exterior
// S multipliers (the first nm_count(P) entries of each particle's multiplier
// table) and the normalised Ferrers constants as a kernel parameter.
template <int P, int KIND, bool DO_S, bool DO_D>
__global__ void __launch_bounds__(128) near_kernel_mixed(const int32_t* __restrict__ pair_t,
                                                         const int32_t* __restrict__ pair_s, int64_t first,
                                                         int64_t count, const PartGeom* __restrict__ parts,
                                                         const double* __restrict__ xyz,
                                                         const float* __restrict__ alpha32,
                                                         const float* __restrict__ beta32,
                                                         const double* __restrict__ mult,
                                                         const double* __restrict__ inv_tab, const PbarTab<P> tab,
                                                         double* __restrict__ S_out, double* __restrict__ D_out) {
  constexpr int NC = (P + 1) * (P + 1);
  constexpr int NM = (P + 1) * (P + 2) / 2;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = first + r;
    const int t = pair_t[idx], i = pair_s[idx];
    const PartGeom& G = parts[i];
    const double dx = xyz[(int64_t)t * 3 + 0] - G.c[0];
    const double dy = xyz[(int64_t)t * 3 + 1] - G.c[1];
    const double dz = xyz[(int64_t)t * 3 + 2] - G.c[2];
    const double xl = G.R[0] * dx + G.R[3] * dy + G.R[6] * dz;
    const double yl = G.R[1] * dx + G.R[4] * dy + G.R[7] * dz;
    const double zl = G.R[2] * dx + G.R[5] * dy + G.R[8] * dz;
    double S, D;
    near_pair_mixed<P, KIND, DO_S, DO_D>(xl, yl, zl, G.a, alpha32 + (size_t)i * NC, beta32 + (size_t)i * NC,
                                         mult + (size_t)i * 4 * NM, inv_tab, tab, S, D);
    if (DO_S) atomicAdd(S_out + t, S);
    if (DO_D) atomicAdd(D_out + t, D);
  }
}

// Normalised Ferrers constants (FP64 closed forms rounded to FP32):
//   Pbar_0^0 = 1 / sqrt(4 pi);  Pbar_1^1 / Pbar_0^0 = sqrt(3) sv;
//   Pbar_m^m / Pbar_{m-1}^{m-1} = sqrt((2m+1) / (2m)) sv  (m >= 2);
//   a_nm = sqrt((2n+1)(2n-1) / ((n-m)(n+m))),
//   b_nm = sqrt((2n+1)(n+m-1)(n-m-1) / ((2n-3)(n-m)(n+m))),
// from (n-m) P_n^m = (2n-1) v P_{n-1}^m - (n+m-1) P_{n-2}^m and the ratios
// of the normalisations N_n^m.
template <int P>
static PbarTab<P> make_pbar_tab() {
  PbarTab<P> t{};
  t.mm[0] = (float)(1.0 / std::sqrt(4.0 * 3.141592653589793));
  if (P >= 1) t.mm[1] = (float)std::sqrt(3.0);
  for (int m = 2; m <= P; ++m) t.mm[m] = (float)std::sqrt((2.0 * m + 1.0) / (2.0 * m));
  for (int m = 0; m <= P; ++m)
    for (int n = m + 1; n <= P; ++n) {
      t.a[nm_index(n, m)] = (float)std::sqrt((2.0 * n + 1.0) * (2.0 * n - 1.0) / ((double)(n - m) * (n + m)));
      if (n >= m + 2)
        t.b[nm_index(n, m)] = (float)std::sqrt((2.0 * n + 1.0) * (n + m - 1.0) * (n - m - 1.0) /
                                               ((2.0 * n - 3.0) * (n - m) * (n + m)));
    }
  return t;
}

template <int P, int KIND>
static void launch_near_pk(const DevGeom& d, int64_t first, int64_t count, const double* inv_tab, double* S,
                           double* D, bool mixed, cudaStream_t st) {
  if (count <= 0) return;
  const int threads = d.near_block == 64 ? 64 : 128;
  int64_t nb = (count + threads - 1) / threads;
  if (d.near_grid_cap > 0 && nb > d.near_grid_cap) nb = d.near_grid_cap;
  const unsigned blocks = (unsigned)nb;
  if (mixed) {
    static const PbarTab<P> tab = make_pbar_tab<P>();
    if (S && D)
      near_kernel_mixed<P, KIND, true, true><<<blocks, threads, 0, st>>>(
          d.pair_t, d.pair_s, first, count, d.parts, d.xyz, d.alpha32, d.beta32, d.mult, inv_tab, tab, S, D);
    else if (S)
      near_kernel_mixed<P, KIND, true, false><<<blocks, threads, 0, st>>>(
          d.pair_t, d.pair_s, first, count, d.parts, d.xyz, d.alpha32, d.beta32, d.mult, inv_tab, tab, S, D);
    else
      near_kernel_mixed<P, KIND, false, true><<<blocks, threads, 0, st>>>(
          d.pair_t, d.pair_s, first, count, d.parts, d.xyz, d.alpha32, d.beta32, d.mult, inv_tab, tab, S, D);
    count_launch();
    return;
  }
  if (S && D)
    near_kernel<P, KIND, true, true><<<blocks, threads, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts, d.xyz,
                                                                 d.alpha, d.beta, inv_tab, S, D);
  else if (S)
    near_kernel<P, KIND, true, false><<<blocks, threads, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts, d.xyz,
                                                                  d.alpha, d.beta, inv_tab, S, D);
  else
    near_kernel<P, KIND, false, true><<<blocks, threads, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts, d.xyz,
                                                                  d.alpha, d.beta, inv_tab, S, D);
  count_launch();
}

template <int P>
static void launch_near_p(const DevGeom& d, int64_t n_pro, int64_t n_all, const double* inv_tab, double* S,
                          double* D, bool mixed, cudaStream_t st) {
  launch_near_pk<P, SBIO_PROLATE>(d, 0, n_pro, inv_tab, S, D, mixed, st);
  launch_near_pk<P, SBIO_OBLATE>(d, n_pro, n_all - n_pro, inv_tab, S, D, mixed, st);
}

template <int... Ps>
struct NearTable {
  static near_launcher get(int p) {
    near_launcher tab[] = {launch_near_p<Ps>...};
    int ps[] = {Ps...};
    for (size_t k = 0; k < sizeof(ps) / sizeof(int); ++k)
      if (ps[k] == p) return tab[k];
    return nullptr;
  }
};

}  // namespace sbio
