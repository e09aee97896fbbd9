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
// gradients in the source's local frame.  For the target's own particle the
// same formulas are evaluated at the own surface node (exterior limit).
#pragma once

#include "sbio_internal.cuh"
#include "sbio_near.cuh"

namespace sbio {

template <int P1, int KIND>
__device__ __forceinline__ void stokes_pair(double xl, double yl, double zl, double a, const double* __restrict__ R,
                                            double X0, double X1, double X2, const double* __restrict__ coef,
                                            const double* __restrict__ inv_tab, double out[3]) {
  constexpr double sgn = (KIND == SBIO_PROLATE) ? -1.0 : 1.0;
  constexpr int NC = (P1 + 1) * (P1 + 1);
  const SphCoord sc = to_spheroidal(xl, yl, zl, a, KIND);
  const double u = sc.u, v = sc.v, sv = sc.sv;
  const double u2s = u * u + sgn;
  const double rsu = rsqrt(u2s);
  const double su = u2s * rsu;
  const double inv_den = rsu * rsu;
  double qa[P1 + 3], qb[P1 + 3];
  miller_q01<P1 + 1, KIND>(u, rsu, inv_tab, qb, qa);   // qb = Q^0, qa = Q^1, n = 0..P1+2
  const double c = u * rsu;
  double F[4], Fu[4], Fv[4], Fp[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) F[d] = Fu[d] = Fv[d] = Fp[d] = 0.0;
  double cm = 1.0, sm = 0.0;
  const double c1 = sc.cph, s1 = sc.sph;
  double dmm = 1.0;   // D_m^m = (2m-1)!! sv^(m-1)
#pragma unroll
  for (int m = 0; m <= P1; ++m) {
    double* qm;
    if (m == 0) {
      qm = qb;
    } else if (m == 1) {
      qm = qa;
    } else {
      double* q1p = (m & 1) ? qb : qa;
      double* q2p = (m & 1) ? qa : qb;
      const double cc = -2.0 * (m - 1) * c;
#pragma unroll
      for (int n = m; n <= P1 + 1; ++n) q2p[n] = cc * q1p[n] + ((n - m + 2.0) * (n + m - 1.0)) * q2p[n];
      qm = q2p;
    }
    if (m == 0) {
      double pprev = 0.0, pcur = 1.0;
#pragma unroll
      for (int n = 0; n <= P1; ++n) {
        const double dq = (-sgn * (n + 1.0) * qm[n + 1] - (n + 1.0) * u * qm[n]) * inv_den;
        const double T = qm[n] * pcur, Tu = dq * pcur;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          const double al = coef[d * NC + n * n + n];
          F[d] = fma(al, T, F[d]);
          Fu[d] = fma(al, Tu, Fu[d]);
        }
        const double pnext = ((2.0 * n + 1.0) / (n + 1.0)) * (v * pcur) - ((double)n / (n + 1.0)) * pprev;
        pprev = pcur;
        pcur = pnext;
      }
    } else {
      if (m >= 2) dmm *= (2.0 * m - 1.0) * sv;
      double dprev = 0.0, dcur = dmm;
#pragma unroll
      for (int n = m; n <= P1; ++n) {
        const double dnext = ((2.0 * n + 1.0) / (n - m + 1.0)) * (v * dcur) - ((double)(n + m) / (n - m + 1.0)) * dprev;
        const double pb = sv * dcur;
        const double dq = (-sgn * (n - m + 1.0) * qm[n + 1] - (n + 1.0) * u * qm[n]) * inv_den;
        const double T = qm[n] * pb, Tu = dq * pb;
        const double Tv = qm[n] * ((n + 1.0) * v * dcur - (n - m + 1.0) * dnext);
        const double Tp = qm[n] * (m * dcur);
        const double Tc = T * cm, Ts = T * sm, Tuc = Tu * cm, Tus = Tu * sm, Tvc = Tv * cm, Tvs = Tv * sm;
        const double Tpc = -Tp * sm, Tps = Tp * cm;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          const double ac = coef[d * NC + n * n + n + m], as = coef[d * NC + n * n + n - m];
          F[d] = fma(ac, Tc, fma(as, Ts, F[d]));
          Fu[d] = fma(ac, Tuc, fma(as, Tus, Fu[d]));
          Fv[d] = fma(ac, Tvc, fma(as, Tvs, Fv[d]));
          Fp[d] = fma(ac, Tpc, fma(as, Tps, Fp[d]));
        }
        if (m == 1) {
          // delayed m = 0 v-derivative: sqrt(1-v^2) dP_n/dv = Pbar_n^1 = sv D_n^1
          const double T0 = qb[n] * pb;
#pragma unroll
          for (int d = 0; d < 4; ++d) Fv[d] = fma(coef[d * NC + n * n + n], T0, Fv[d]);
        }
        dprev = dcur;
        dcur = dnext;
      }
    }
    const double cn = cm * c1 - sm * s1;
    sm = sm * c1 + cm * s1;
    cm = cn;
  }
  // gradients in the local frame
  const double W2 = u * u + sgn * v * v;
  const double iW = rsqrt(W2);
  const double ia = 1.0 / a;
  const double eu0 = u * sv * c1 * iW, eu1 = u * sv * s1 * iW, eu2 = v * su * iW;
  const double ev0 = -su * v * c1 * iW, ev1 = -su * v * s1 * iW, ev2 = u * sv * iW;
  double g[4][3];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const double gu = Fu[d] * su * ia * iW, gv = Fv[d] * ia * iW, gp = Fp[d] * ia * rsu;
    g[d][0] = gu * eu0 + gv * ev0 - gp * s1;
    g[d][1] = gu * eu1 + gv * ev1 + gp * c1;
    g[d][2] = gu * eu2 + gv * ev2;
  }
  double w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] = g[3][k] - (X0 * g[0][k] + X1 * g[1][k] + X2 * g[2][k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) out[k] = 0.5 * (F[k] + R[k * 3 + 0] * w[0] + R[k * 3 + 1] * w[1] + R[k * 3 + 2] * w[2]);
}

template <int P1, int KIND>
__global__ void __launch_bounds__(128) stokes_near_kernel(const int32_t* __restrict__ pair_t,
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
  int64_t nb = (count + 127) / 128;
  if (d.near_grid_cap > 0 && nb > d.near_grid_cap) nb = d.near_grid_cap;
  const unsigned blocks = (unsigned)nb;
  stokes_near_kernel<P1, KIND><<<blocks, 128, 0, st>>>(d.pair_t, d.pair_s, first, count, d.parts, d.xyz,
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
