// Velocity and pressure of the Stokes single layer at arbitrary points for
// near (point, source particle) pairs (Sec. 4.3, eq. (stokes); Sec. 4.1
// particle-to-target algorithm).  One call of solid_grad gives the values
// and gradients of the four Laplace expansions (f_1, f_2, f_3, y . f at order
// p+1); the velocity is eq. (stokes) and the pressure is the divergence
//     p = -sum_j d_j S[f_j],
// the printed pressure kernel r / (4 pi |r|^3) (d_j (1/r) = -r_j / r^3).
#pragma once

#include "sbio_grad.cuh"

namespace sbio {

template <int P1, int KIND>
__global__ void __launch_bounds__(128) stokes_point_near_kernel(const int32_t* __restrict__ pair_t,
                                                                const int32_t* __restrict__ pair_s, int64_t first,
                                                                int64_t count, const PartGeom* __restrict__ parts,
                                                                const double* __restrict__ xyz,
                                                                const double* __restrict__ coef,
                                                                const double* __restrict__ inv_tab,
                                                                double* __restrict__ u_out,
                                                                double* __restrict__ p_out) {
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
    const double* cf = coef + (size_t)i * 4 * NC;
    const double* c[4] = {cf, cf + NC, cf + 2 * NC, cf + 3 * NC};
    double F[4], g[4][3];
    solid_grad<P1, KIND, 4>(xl, yl, zl, G.a, c, inv_tab, F, g);
    const double* R = G.R;
    double w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = g[3][k] - (X0 * g[0][k] + X1 * g[1][k] + X2 * g[2][k]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      atomicAdd(u_out + (int64_t)t * 3 + k,
                0.5 * (F[k] + R[k * 3 + 0] * w[0] + R[k * 3 + 1] * w[1] + R[k * 3 + 2] * w[2]));
    // divergence of (S[f_1], S[f_2], S[f_3]) in the global frame: the k-th
    // global component of grad S[f_k] is sum_l R[k][l] g_k[l]
    double dv = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) dv += R[k * 3 + 0] * g[k][0] + R[k * 3 + 1] * g[k][1] + R[k * 3 + 2] * g[k][2];
    atomicAdd(p_out + t, -dv);
  }
}

typedef void (*stokes_point_near_launcher)(const DevGeom&, int64_t, int64_t, double*, double*, cudaStream_t);

template <int P1, int KIND>
static void launch_stokes_point_near_pk(const DevGeom& d, int64_t first, int64_t count, double* u, double* pr,
                                        cudaStream_t st) {
  if (count <= 0) return;
  int64_t nb = (count + 127) / 128;
  if (d.near_grid_cap > 0 && nb > d.near_grid_cap) nb = d.near_grid_cap;
  stokes_point_near_kernel<P1, KIND><<<(unsigned)nb, 128, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts, d.xyz,
                                                                   d.st_coef, d.inv, u, pr);
  count_launch();
}

template <int P1>
static void launch_stokes_point_near_p(const DevGeom& d, int64_t n_pro, int64_t n_all, double* u, double* pr,
                                       cudaStream_t st) {
  launch_stokes_point_near_pk<P1, SBIO_PROLATE>(d, 0, n_pro, u, pr, st);
  launch_stokes_point_near_pk<P1, SBIO_OBLATE>(d, n_pro, n_all - n_pro, u, pr, st);
}

template <int... Ps>
struct StokesPointNearTable {
  static stokes_point_near_launcher get(int p) {
    stokes_point_near_launcher tab[] = {launch_stokes_point_near_p<Ps + 1>...};
    int ps[] = {Ps...};
    for (size_t k = 0; k < sizeof(ps) / sizeof(int); ++k)
      if (ps[k] == p) return tab[k];
    return nullptr;
  }
};

}  // namespace sbio
