// Gradients of the exterior single-layer-type expansions of one source
// particle at a target (eq. (dSLevalformula) in Cartesian form):
//     F_d   = sum c_d[nm] q_n^|m|(u) Pbar_n^|m|(v) trig_m(phi)
//     grad F_d = e_u dF/du / h_u + e_v dF/dv / h_v + e_phi dF/dphi / h_phi
// with q the exterior radial functions (Miller sweeps for m = 0, 1, then the
// order recurrence) and the regularised v- and phi-derivatives near the
// source axis: sqrt(1-v^2) dPbar/dv = (n+1) v D_n - (n-m+1) D_{n+1} and
// m Pbar / sqrt(1-v^2) = m D_n with D_n^m = Pbar_n^m / sqrt(1-v^2) (m >= 1),
// and sqrt(1-v^2) dP_n/dv = Pbar_n^1 for m = 0.  (xl, yl, zl): target in the
// source's local frame; c_d: coefficients with the exterior factor and the
// normalisation folded in, index n^2 + n + m.
#pragma once

#include "sbio_internal.cuh"
#include "sbio_near.cuh"

namespace sbio {

// Threads per CTA of the Stokes near-gradient kernels.  They hold about 250
// registers per thread at the larger orders; a 64-thread CTA takes a quarter
// of an SM's register file (a 128-thread one half), so that capped near CTAs
// share an SM with the far kernel's CTAs instead of filling it.
constexpr int kNearGradBlock = 64;

// Term-by-term evaluation.  For every term of the exterior
// expansions at a target, solid_terms hands the visitor the radial-angular
// factors without the azimuthal trig:
//     T  = q_n^m(u) Pbar_n^m(v),       Tu = d/du [q_n^m] Pbar_n^m(v),
//     Tv = q_n^m(u) sqrt(1-v^2) dPbar_n^m/dv,
//     Tp = q_n^m(u) m Pbar_n^m(v) / sqrt(1-v^2)   (m >= 1),
// through vis.term(n, m, T, Tu, Tv, Tp) for m >= 1 (the cos and sin parts
// share them; vis.order(m, cos m phi, sin m phi) precedes the terms of order
// m) and vis.term0(n, T, Tu, Tv) for m = 0.  vis.begin(frame) first receives
// the factors that turn d/du, sqrt(1-v^2) d/dv and (1/sqrt(1-v^2)) d/dphi
// sums into local Cartesian gradients:
//     grad_x = c1 (k_ru Fu + k_rv Fv) - s1 k_p Fp,
//     grad_y = s1 (k_ru Fu + k_rv Fv) + c1 k_p Fp,
//     grad_z = k_zu Fu + k_zv Fv,
// (e_u / h_u, e_v / h_v, e_phi / h_phi of Table 1 in the source's frame),
// with Fp the phi-derivative sum (d/dphi of cos m phi -> -m sin m phi).
// The m = 0 terms n >= 1 are issued inside the order-1 sweep, which supplies
// their v-derivative sqrt(1-v^2) dP_n/dv = Pbar_n^1.
struct GradFrame {
  double k_ru, k_rv, k_zu, k_zv, k_p, c1, s1;
};

template <int P1, int KIND, class V>
__device__ __forceinline__ void solid_terms(double xl, double yl, double zl, double a,
                                            const double* __restrict__ inv_tab, V& vis) {
  constexpr double sgn = (KIND == SBIO_PROLATE) ? -1.0 : 1.0;
  const SphCoord sc = to_spheroidal(xl, yl, zl, a, KIND);
  const double u = sc.u, v = sc.v, sv = sc.sv;
  const double u2s = u * u + sgn;
  const double rsu = rsqrt(u2s);
  const double su = u2s * rsu;
  const double inv_den = rsu * rsu;
  double qa[P1 + 3], qb[P1 + 3];
  miller_q01<P1 + 1, KIND>(u, rsu, inv_tab, qb, qa);   // qb = Q^0, qa = Q^1, n = 0..P1+2
  const double c = u * rsu;
  {
    const double iW = rsqrt(u * u + sgn * v * v);
    const double ia = 1.0 / a;
    const double iW2a = iW * iW * ia;
    GradFrame fr;
    fr.k_ru = u * sv * su * iW2a;
    fr.k_rv = -su * v * iW2a;
    fr.k_zu = v * su * su * iW2a;
    fr.k_zv = u * sv * iW2a;
    fr.k_p = ia * rsu;
    fr.c1 = sc.cph;
    fr.s1 = sc.sph;
    vis.begin(fr);
  }
  const double c1 = sc.cph, s1 = sc.sph;
  // m = 0, n = 0 (P_0 = 1, no v-derivative)
  vis.term0(0, qb[0], (-sgn * qb[1] - u * qb[0]) * inv_den, 0.0);
  // order 1, with the m = 0 terms n >= 1
  vis.order(1, c1, s1);
  {
    double dprev = 0.0, dcur = 1.0;   // D_n^1 = Pbar_n^1 / sqrt(1-v^2), D_1^1 = 1
    double p0prev = 1.0, p0cur = v;   // P_0, P_1
#pragma unroll
    for (int n = 1; n <= P1; ++n) {
      const double dnext = ((2.0 * n + 1.0) / n) * (v * dcur) - ((n + 1.0) / n) * dprev;
      const double pb = sv * dcur;
      const double dq1 = (-sgn * n * qa[n + 1] - (n + 1.0) * u * qa[n]) * inv_den;
      vis.term(n, 1, qa[n] * pb, dq1 * pb, qa[n] * ((n + 1.0) * v * dcur - n * dnext), qa[n] * dcur);
      const double dq0 = (-sgn * (n + 1.0) * qb[n + 1] - (n + 1.0) * u * qb[n]) * inv_den;
      vis.term0(n, qb[n] * p0cur, dq0 * p0cur, qb[n] * pb);
      const double p0next = ((2.0 * n + 1.0) / (n + 1.0)) * (v * p0cur) - ((double)n / (n + 1.0)) * p0prev;
      p0prev = p0cur;
      p0cur = p0next;
      dprev = dcur;
      dcur = dnext;
    }
  }
  double cm = c1 * c1 - s1 * s1, sm = 2.0 * s1 * c1;   // order 2
  double dmm = 1.0;                                     // D_m^m = (2m-1)!! sv^(m-1)
#pragma unroll
  for (int m = 2; m <= P1; ++m) {
    double* q1p = (m & 1) ? qb : qa;   // order m-1
    double* q2p = (m & 1) ? qa : qb;   // order m-2, overwritten by order m
    const double cc = -2.0 * (m - 1) * c;
#pragma unroll
    for (int n = m; n <= P1 + 1; ++n) q2p[n] = cc * q1p[n] + ((n - m + 2.0) * (n + m - 1.0)) * q2p[n];
    const double* qm = q2p;
    dmm *= (2.0 * m - 1.0) * sv;
    vis.order(m, cm, sm);
    double dprev = 0.0, dcur = dmm;
#pragma unroll
    for (int n = m; n <= P1; ++n) {
      const double dnext = ((2.0 * n + 1.0) / (n - m + 1.0)) * (v * dcur) - ((double)(n + m) / (n - m + 1.0)) * dprev;
      const double pb = sv * dcur;
      const double dq = (-sgn * (n - m + 1.0) * qm[n + 1] - (n + 1.0) * u * qm[n]) * inv_den;
      vis.term(n, m, qm[n] * pb, dq * pb, qm[n] * ((n + 1.0) * v * dcur - (n - m + 1.0) * dnext), qm[n] * (m * dcur));
      dprev = dcur;
      dcur = dnext;
    }
    const double cn = cm * c1 - sm * s1;
    sm = sm * c1 + cm * s1;
    cm = cn;
  }
}

}  // namespace sbio
