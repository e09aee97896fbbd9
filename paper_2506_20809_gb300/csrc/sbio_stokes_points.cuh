// Velocity and pressure of the Stokes single layer at arbitrary points for
// near (point, source particle) pairs (Sec. 4.3, eq. (stokes); Sec. 4.1
// particle-to-target algorithm).  One sweep of solid_terms over the four
// Laplace expansions (f_1, f_2, f_3, y . f at order p+1) gives the values
// S[f_k], the gradient of the combined expansion S[y . f] - sum_j X_j S[f_j]
// (the velocity's bracket in eq. (stokes), X fixed per pair) and the local
// (u, v, phi) derivative sums of each S[f_k], from which the pressure is the
// divergence
//     p = -sum_j d_j S[f_j],
// the printed pressure kernel r / (4 pi |r|^3) (d_j (1/r) = -r_j / r^3).
#pragma once

#include "sbio_grad.cuh"

namespace sbio {

template <int NC>
struct StokesPointVisitor {
  const double* __restrict__ cf;   // 4 x NC: f_1, f_2, f_3, y . f
  double X0, X1, X2;
  double cm, sm;
  double F[3], Fu[3], Fv[3], Fp[3], Hu, Hv, Hp;
  GradFrame fr;

  __device__ __forceinline__ void begin(const GradFrame& f) {
    fr = f;
#pragma unroll
    for (int j = 0; j < 3; ++j) F[j] = Fu[j] = Fv[j] = Fp[j] = 0.0;
    Hu = Hv = Hp = 0.0;
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
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double ac = cf[j * NC + kc], as = cf[j * NC + ks];
      const double aj = fma(ac, cm, as * sm), bj = fma(as, cm, -ac * sm);
      F[j] = fma(aj, T, F[j]);
      Fu[j] = fma(aj, Tu, Fu[j]);
      Fv[j] = fma(aj, Tv, Fv[j]);
      Fp[j] = fma(bj, Tp, Fp[j]);
    }
  }
  __device__ __forceinline__ void term0(int n, double T, double Tu, double Tv) {
    const int k = n * n + n;
    const double hk = h(k);
    Hu = fma(hk, Tu, Hu);
    Hv = fma(hk, Tv, Hv);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double aj = cf[j * NC + k];
      F[j] = fma(aj, T, F[j]);
      Fu[j] = fma(aj, Tu, Fu[j]);
      Fv[j] = fma(aj, Tv, Fv[j]);
    }
  }
  // local Cartesian gradient from (u, v, phi) derivative sums
  __device__ __forceinline__ void grad(double u_, double v_, double p_, double g[3]) const {
    const double rho = fma(fr.k_ru, u_, fr.k_rv * v_), ph = fr.k_p * p_;
    g[0] = fr.c1 * rho - fr.s1 * ph;
    g[1] = fr.s1 * rho + fr.c1 * ph;
    g[2] = fma(fr.k_zu, u_, fr.k_zv * v_);
  }
};

template <int P1, int KIND>
__global__ void __launch_bounds__(kNearGradBlock) stokes_point_near_kernel(const int32_t* __restrict__ pair_t,
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
    StokesPointVisitor<NC> vis;
    vis.cf = coef + (size_t)i * 4 * NC;
    vis.X0 = X0;
    vis.X1 = X1;
    vis.X2 = X2;
    solid_terms<P1, KIND>(xl, yl, zl, G.a, inv_tab, vis);
    const double* R = G.R;
    double w[3];
    vis.grad(vis.Hu, vis.Hv, vis.Hp, w);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      atomicAdd(u_out + (int64_t)t * 3 + k,
                0.5 * (vis.F[k] + R[k * 3 + 0] * w[0] + R[k * 3 + 1] * w[1] + R[k * 3 + 2] * w[2]));
    // divergence of (S[f_1], S[f_2], S[f_3]) in the global frame: the k-th
    // global component of grad S[f_k] is sum_l R[k][l] g_k[l]
    double dv = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double g[3];
      vis.grad(vis.Fu[k], vis.Fv[k], vis.Fp[k], g);
      dv += R[k * 3 + 0] * g[0] + R[k * 3 + 1] * g[1] + R[k * 3 + 2] * g[2];
    }
    atomicAdd(p_out + t, -dv);
  }
}

typedef void (*stokes_point_near_launcher)(const DevGeom&, int64_t, int64_t, double*, double*, cudaStream_t);

template <int P1, int KIND>
static void launch_stokes_point_near_pk(const DevGeom& d, int64_t first, int64_t count, double* u, double* pr,
                                        cudaStream_t st) {
  if (count <= 0) return;
  int64_t nb = (count + kNearGradBlock - 1) / kNearGradBlock;
  if (d.near_grid_cap > 0 && nb > d.near_grid_cap) nb = d.near_grid_cap;
  stokes_point_near_kernel<P1, KIND><<<(unsigned)nb, kNearGradBlock, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts, d.xyz,
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
