// Near part of the Stokes double layer (and of its evaluation at points):
// for one (target, source particle) pair, the gradients of the source's
// thirteen folded expansions (order P1 = p + 1) at the target, in four passes
// of solid_grad over four expansions each, combined as
//     D_stk_i = -X_i sum_j d_j D[q_j] + sum_j d_j D[y_i q_j] - d_i S[q . nu]
// (X the target relative to the source centre, global frame).  The source's
// own nodes are evaluated separably (sdl_self_kernel).
#pragma once

#include "sbio_grad.cuh"

namespace sbio {

template <int P1, int KIND>
__global__ void __launch_bounds__(128) stokes_dl_near_kernel(const int32_t* __restrict__ pair_t,
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
    const double* cf = coef + (size_t)i * 13 * NC;
    const double* R = G.R;
    double div_q = 0.0, t2[3] = {0.0, 0.0, 0.0}, t3[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
    for (int pass = 0; pass < 4; ++pass) {
      // pass 0: q_1, q_2, q_3, q.nu; pass 1 + i: y_i q_1, y_i q_2, y_i q_3 (4th slot unused)
      const double* c[4];
      if (pass == 0) {
        c[0] = cf;
        c[1] = cf + NC;
        c[2] = cf + 2 * NC;
        c[3] = cf + 12 * NC;
      } else {
        const double* b = cf + (3 + 3 * (pass - 1)) * NC;
        c[0] = b;
        c[1] = b + NC;
        c[2] = b + 2 * NC;
        c[3] = b;
      }
      double F[4], g[4][3];
      solid_grad<P1, KIND, 4>(xl, yl, zl, G.a, c, inv_tab, F, g);
      // global gradient component k of expansion d: sum_l R[k][l] g_d[l]
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) s += R[k * 3 + 0] * g[k][0] + R[k * 3 + 1] * g[k][1] + R[k * 3 + 2] * g[k][2];
      if (pass == 0) {
        div_q = s;
#pragma unroll
        for (int k = 0; k < 3; ++k) t3[k] = R[k * 3 + 0] * g[3][0] + R[k * 3 + 1] * g[3][1] + R[k * 3 + 2] * g[3][2];
      } else {
        t2[pass - 1] = s;
      }
    }
    atomicAdd(u_out + (int64_t)t * 3 + 0, -X0 * div_q + t2[0] - t3[0]);
    atomicAdd(u_out + (int64_t)t * 3 + 1, -X1 * div_q + t2[1] - t3[1]);
    atomicAdd(u_out + (int64_t)t * 3 + 2, -X2 * div_q + t2[2] - t3[2]);
  }
}

typedef void (*stokes_dl_near_launcher)(const DevGeom&, const int32_t*, const int32_t*, int64_t, int64_t, double*,
                                        cudaStream_t);

template <int P1, int KIND>
static void launch_stokes_dl_near_pk(const DevGeom& d, const int32_t* pt, const int32_t* ps, int64_t first,
                                     int64_t count, double* u, cudaStream_t st) {
  if (count <= 0) return;
  int64_t nb = (count + 127) / 128;
  if (d.near_grid_cap > 0 && nb > d.near_grid_cap) nb = d.near_grid_cap;
  stokes_dl_near_kernel<P1, KIND><<<(unsigned)nb, 128, 0, st>>>(pt, ps, first, count, d.parts, d.xyz, d.sdl_coef,
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
