// Near-field evaluation of one (target, source particle) pair: the exterior
// solid-harmonic expansions of Theorems 1-2,
//     S = sum_nm alpha_nm q_n^|m|(u) Pbar_n^|m|(v) trig_m(phi),
//     D = sum_nm beta_nm  q_n^|m|(u) Pbar_n^|m|(v) trig_m(phi),
// at the target's spheroidal coordinates (u, v, phi) relative to the source
// (Algorithm 1, near branch).  alpha / beta are the density coefficients with
// the exterior multiplier, the surface-harmonic normalisation and sqrt(2)
// (m != 0) already folded in, so the Legendre factors here are unnormalised:
// q the Q family of sbio_common.cuh, Pbar the Ferrers functions.
//
// FP64 throughout.  The order P is a template parameter so that every (n, m)
// loop is unrolled and all radial values live in registers.
#pragma once

#include "sbio_common.cuh"

namespace sbio {

// Inverse-integer table used by the rolled part of the Miller sweep: entry k
// holds 1/k for k >= 1, entry 0 the table's length.  The geometry sizes the
// table from its most elongated particle (at least kInvTable entries), so that
// the sweep can always start its full K steps above the top order.
constexpr int kInvTable = 512;

// Q family for m = 0 and m = 1, n = 0..P+1, normalised (see sbio_common.cuh).
template <int P, int KIND>
__device__ __forceinline__ void miller_q01(double u, double rsu, const double* __restrict__ inv_tab, double* q0,
                                           double* q1) {
  constexpr double sgn = (KIND == SBIO_PROLATE) ? -1.0 : 1.0;
  // start index above the top order; rolled part in FP64 with tabulated 1/n
  const float muf = logf((float)u + sqrtf((float)(u * u + sgn)));
  int K = (int)ceilf(19.0f / muf) + 2;
  const int kmax = (int)inv_tab[0] - P - 8;
  K = K < 4 ? 4 : (K > kmax ? kmax : K);
  int n = P + 1 + K;
  double a0 = 0.0, b0 = 1.0, a1 = 0.0, b1 = 1.0;   // q_{n+1}, q_n
  double nd = (double)n;
  double tu = (2.0 * nd + 1.0) * u;
  double inv_np1 = inv_tab[n + 1];
  const double twou = 2.0 * u;
  for (; n > P + 1; --n) {
    const double inv_n = inv_tab[n];
    // m = 0: n q_{n-1} = (2n+1) u q_n + sgn (n+1) q_{n+1}
    const double c0 = (tu * b0 + sgn * (nd + 1.0) * a0) * inv_n;
    // m = 1: (n+1) q_{n-1} = (2n+1) u q_n + sgn n q_{n+1}
    const double c1 = (tu * b1 + sgn * nd * a1) * inv_np1;
    a0 = b0; b0 = c0;
    a1 = b1; b1 = c1;
    inv_np1 = inv_n;
    nd -= 1.0;
    tu -= twou;
    if ((n & 15) == 0 && fabs(b0) + fabs(b1) > 1e200) {
      a0 *= 1e-200; b0 *= 1e-200; a1 *= 1e-200; b1 *= 1e-200;
    }
  }
  // n == P+1: b = q_{P+1}, a = q_{P+2}
  q0[P + 1] = b0;
  q1[P + 1] = b1;
  double x0 = a0, x1 = a1;   // q_{n+1}
#pragma unroll
  for (int k = P + 1; k >= 1; --k) {
    // q_{k-1} from q_k, q_{k+1}, exact constants
    const double y0 = ((2.0 * k + 1.0) / k) * u * q0[k] + (sgn * (k + 1.0) / k) * x0;
    const double y1 = ((2.0 * k + 1.0) / (k + 1.0)) * u * q1[k] + (sgn * k / (k + 1.0)) * x1;
    x0 = q0[k];
    x1 = q1[k];
    q0[k - 1] = y0;
    q1[k - 1] = y1;
  }
  // Casoratian at n = 1 (m = 0): u q_0 + sgn q_1 = 1;  q_0^1 = -1/s_u
  const double s0 = 1.0 / (u * q0[0] + sgn * q0[1]);
  const double s1 = -rsu / q1[0];
#pragma unroll
  for (int k = 0; k <= P + 1; ++k) {
    q0[k] *= s0;
    q1[k] *= s1;
  }
}

// S and D of one pair.  xl: target in the source's local frame.
template <int P, int KIND, bool DO_S, bool DO_D>
__device__ __forceinline__ void near_pair(double xl, double yl, double zl, double a, const double* __restrict__ alpha,
                                          const double* __restrict__ beta, const double* __restrict__ inv_tab,
                                          double& S, double& D) {
  constexpr double sgn = (KIND == SBIO_PROLATE) ? -1.0 : 1.0;
  const SphCoord sc = to_spheroidal(xl, yl, zl, a, KIND);
  const double u = sc.u, v = sc.v, sv = sc.sv;
  const double rsu = rsqrt(u * u + sgn);
  double qa[P + 2], qb[P + 2];   // Q^{m-1}, Q^{m-2} (rotating roles)
  miller_q01<P, KIND>(u, rsu, inv_tab, qb, qa);   // qb = Q^0, qa = Q^1
  const double c = u * rsu;                       // u / s_u
  double cm = 1.0, sm = 0.0;                      // cos(m phi), sin(m phi)
  const double c1 = sc.cph, s1 = sc.sph;
  double pmm = 1.0;                               // Pbar_m^m(v)
  double accS = 0.0, accD = 0.0;
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    // radial values of order m: m = 0 -> qb, m = 1 -> qa, m >= 2 by the order recurrence
    double* qm;
    if (m == 0) {
      qm = qb;
    } else if (m == 1) {
      qm = qa;
    } else {
      // Q^m_n = -2(m-1) c Q^{m-1}_n + (n-m+2)(n+m-1) Q^{m-2}_n, stored over Q^{m-2}
      double* q1p = (m & 1) ? qb : qa;   // order m-1
      double* q2p = (m & 1) ? qa : qb;   // order m-2 (overwritten)
      const double cc = -2.0 * (m - 1) * c;
#pragma unroll
      for (int n = m; n <= P; ++n) q2p[n] = cc * q1p[n] + ((n - m + 2.0) * (n + m - 1.0)) * q2p[n];
      qm = q2p;
    }
    if (m > 0) pmm *= (2.0 * m - 1.0) * sv;
    double Sc = 0.0, Ss = 0.0, Dc = 0.0, Ds = 0.0;
    double pprev = 0.0, pcur = pmm;
#pragma unroll
    for (int n = m; n <= P; ++n) {
      const double T = qm[n] * pcur;
      if (DO_S) {
        Sc = fma(alpha[n * n + n + m], T, Sc);
        if (m > 0) Ss = fma(alpha[n * n + n - m], T, Ss);
      }
      if (DO_D) {
        Dc = fma(beta[n * n + n + m], T, Dc);
        if (m > 0) Ds = fma(beta[n * n + n - m], T, Ds);
      }
      if (n < P) {
        // (n-m+1) P_{n+1} = (2n+1) v P_n - (n+m) P_{n-1}
        const double pnext = ((2.0 * n + 1.0) / (n - m + 1.0)) * (v * pcur) - ((double)(n + m) / (n - m + 1.0)) * pprev;
        pprev = pcur;
        pcur = pnext;
      }
    }
    if (m == 0) {
      accS += Sc;
      accD += Dc;
    } else {
      accS = fma(Sc, cm, fma(Ss, sm, accS));
      accD = fma(Dc, cm, fma(Ds, sm, accD));
    }
    const double cn = cm * c1 - sm * s1;
    sm = sm * c1 + cm * s1;
    cm = cn;
  }
  S = accS;
  D = accD;
}

// Mixed-precision form for SBIO_MIXED geometries.  The coordinates, the
// Miller sweep and the order recurrence of the Q family stay FP64 as in
// near_pair; each radial value enters as rho_nm = extS_nm q_n^m(u), the
// exterior S multiplier times Q (of order one for a target outside the
// source, since Q decreases away from the surface), rounded to FP32.  The
// Ferrers functions run normalised in FP32, Pbar_n^m = N_n^m P_n^m with N the
// surface-harmonic normalisation (sqrt 2 for m != 0), by the three-term
// recurrence in n; the n and m sums run in FP32 with TwoSum compensation,
// the angle recurrence in FP64 (cos and sin of m phi rounded once per m).
// Coefficients A = sigma and B = mu extD / extS in FP32, so that
// alpha q P = A rho Pbar and beta q P = B rho Pbar term by term.  On GB300
// the FP64 pipe runs at 1/64 of the FP32 rate (conversions between the two
// formats included); this form issues about 1,100 FP64-pipe instructions
// per pair at p = 16 against about 2,050.
template <int P>
struct PbarTab {
  float mm[P + 1];                  // Pbar_m^m = mm[m] sv Pbar_{m-1}^{m-1} (m >= 1); mm[0] = Pbar_0^0
  float a[(P + 1) * (P + 2) / 2];   // Pbar_n^m = a v Pbar_{n-1}^m - b Pbar_{n-2}^m, at nm_index(n, m)
  float b[(P + 1) * (P + 2) / 2];   // (a used for n >= m + 1, b for n >= m + 2, zero below)
};

template <int P, int KIND, bool DO_S, bool DO_D>
__device__ __forceinline__ void near_pair_mixed(double xl, double yl, double zl, double a,
                                                const float* __restrict__ A32, const float* __restrict__ B32,
                                                const double* __restrict__ extS, const double* __restrict__ inv_tab,
                                                const PbarTab<P>& tab, double& S, double& D) {
  constexpr double sgn = (KIND == SBIO_PROLATE) ? -1.0 : 1.0;
  const SphCoord sc = to_spheroidal(xl, yl, zl, a, KIND);
  const double u = sc.u;
  const float v32 = (float)sc.v, sv32 = (float)sc.sv;
  const double rsu = rsqrt(u * u + sgn);
  double qa[P + 2], qb[P + 2];   // Q^{m-1}, Q^{m-2} (rotating roles)
  miller_q01<P, KIND>(u, rsu, inv_tab, qb, qa);   // qb = Q^0, qa = Q^1
  const double c = u * rsu;
  double cm = 1.0, sm = 0.0;
  const double c1 = sc.cph, s1 = sc.sph;
  float pmm = tab.mm[0];                          // Pbar_m^m(v)
  float aSh = 0.f, aSl = 0.f, aDh = 0.f, aDl = 0.f;   // compensated m sums
#pragma unroll
  for (int m = 0; m <= P; ++m) {
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
      for (int n = m; n <= P; ++n) q2p[n] = cc * q1p[n] + ((n - m + 2.0) * (n + m - 1.0)) * q2p[n];
      qm = q2p;
    }
    if (m > 0) pmm *= tab.mm[m] * sv32;
    float Sc = 0.f, Scl = 0.f, Ss = 0.f, Ssl = 0.f, Dc = 0.f, Dcl = 0.f, Ds = 0.f, Dsl = 0.f;
    float pprev = 0.f, pcur = pmm;
#pragma unroll
    for (int n = m; n <= P; ++n) {
      const float T = (float)(extS[nm_index(n, m)] * qm[n]) * pcur;
      float s, e;
      if (DO_S) {
        two_sum_f32(Sc, A32[n * n + n + m] * T, s, e);
        Sc = s;
        Scl += e;
        if (m > 0) {
          two_sum_f32(Ss, A32[n * n + n - m] * T, s, e);
          Ss = s;
          Ssl += e;
        }
      }
      if (DO_D) {
        two_sum_f32(Dc, B32[n * n + n + m] * T, s, e);
        Dc = s;
        Dcl += e;
        if (m > 0) {
          two_sum_f32(Ds, B32[n * n + n - m] * T, s, e);
          Ds = s;
          Dsl += e;
        }
      }
      if (n < P) {
        const float pnext = fmaf(tab.a[nm_index(n + 1, m)] * v32, pcur, -tab.b[nm_index(n + 1, m)] * pprev);
        pprev = pcur;
        pcur = pnext;
      }
    }
    // the angle factors come from the FP64 recurrence, rounded once per order
    const float cmf = (float)cm, smf = (float)sm;
    float s2, e2;
    if (DO_S) {
      two_sum_f32(aSh, (Sc + Scl) * cmf, s2, e2);
      aSh = s2;
      aSl += e2;
      if (m > 0) {
        two_sum_f32(aSh, (Ss + Ssl) * smf, s2, e2);
        aSh = s2;
        aSl += e2;
      }
    }
    if (DO_D) {
      two_sum_f32(aDh, (Dc + Dcl) * cmf, s2, e2);
      aDh = s2;
      aDl += e2;
      if (m > 0) {
        two_sum_f32(aDh, (Ds + Dsl) * smf, s2, e2);
        aDh = s2;
        aDl += e2;
      }
    }
    const double cn = cm * c1 - sm * s1;
    sm = sm * c1 + cm * s1;
    cm = cn;
  }
  S = (double)aSh + (double)aSl;
  D = (double)aDh + (double)aDl;
}

}  // namespace sbio
