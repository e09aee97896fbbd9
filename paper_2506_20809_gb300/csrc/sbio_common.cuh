// Internal definitions shared by the host set-up and the CUDA kernels of the
// spheroidal boundary-integral library.  Nothing here is part of the C ABI.
//
// Radial functions in real arithmetic.  For a prolate spheroid the radial
// factors of the solid harmonics (Sec. 2.3) are the type-3 Legendre functions
// P_n^m(u), Q_n^m(u), u > 1.  For an oblate spheroid they are taken at x = i u;
// the library works with the real functions
//     p_n^m(u) = i^{-n} P_n^m(i u),      q_n^m(u) = i^{n+1} Q_n^m(i u),
// where (x^2-1)^{1/2} at x = i u is i sqrt(u^2+1).  With sgn = -1 (prolate) or
// +1 (oblate) and s_u = sqrt(u^2 + sgn) both families obey
//   P family:  (n-m+1) r_{n+1} = (2n+1) u r_n + sgn (n+m) r_{n-1},
//              r_m^m = (2m-1)!! s_u^m,  r_{m+1}^m = (2m+1) u r_m^m,
//   Q family:  (n+m) q_{n-1} = (2n+1) u q_n + sgn (n-m+1) q_{n+1}   (run downward),
//              normalised by the Casoratian at n = 1:  u q_0^0 + sgn q_1^0 = 1,
//              q_0^1 = -1/s_u,
//   order recurrence (both families, type 3):
//              r_n^{m+1} = -2m (u/s_u) r_n^m + (n-m+1)(n+m) r_n^{m-1},
//   derivatives d/du (from eq. (derivative)):
//              p' = ((n-m+1) p_{n+1} - (n+1) u p_n) / (u^2 + sgn),
//              q' = (-sgn (n-m+1) q_{n+1} - (n+1) u q_n) / (u^2 + sgn).
// The Q family is computed with Miller's backward recurrence for m = 0 and
// m = 1 (started K terms above the top order, K ~ 19/acosh(u) resp.
// 19/asinh(u), which makes the start error ~ e^{-2 mu K} < 1e-16), followed by
// the order recurrence, which is forward-stable for the Q family.  This
// replaces the paper's one continued fraction per order m (Sec. 2.3 steps 2-4)
// with two backward sweeps; both rest on the same three-term recurrence and
// Casoratian.
//
// Theorems 1-2 multipliers (m >= 0, K = (n-m)!/(n+m)!, s0 = sqrt(u0^2 + sgn)):
//   exterior S factor  aS = a K (-1)^m s0 p(u0)        (times q(u) Y)
//   exterior D factor  aD = K (-1)^m s0^2 p'(u0)        (times q(u) Y)
//   on-surface S       aS q(u0)
//   on-surface D       (D+ + D-)/2,  D+ = aD q(u0),  D- = K (-1)^m s0^2 q'(u0) p(u0)
// For the oblate case these are the paper's c, c~ forms rewritten for the
// real functions above (the powers of i cancel).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "sbio.h"

namespace sbio {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxP = SBIO_MAX_P;
constexpr int kMaxNM = (kMaxP + 3) * (kMaxP + 4) / 2;   // (n, m>=0) pairs up to p+2

__host__ __device__ inline int nm_count(int p) { return (p + 1) * (p + 2) / 2; }
__host__ __device__ inline int nm_index(int n, int m) { return n * (n + 1) / 2 + m; }
__host__ __device__ inline int coef_index(int n, int m) { return n * n + n + m; }

// FP32 far-field helpers shared by the mixed kernels.
// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum_f32(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// One MUFU reciprocal square root (approximate, flush-to-zero).
__device__ __forceinline__ float rsqrt_f32(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One particle as the kernels see it.
struct PartGeom {
  double a;       // half focal distance
  double u0;      // surface coordinate
  double A, C;    // semi-axes
  double c[3];    // centre
  double R[9];    // row-major rotation, x_global = c + R x_local
  double sgn;     // -1 prolate, +1 oblate
  int32_t kind;
  int32_t pad;
};

// Distance from (y0, y1) >= 0 to the ellipse (t0/e0)^2 + (t1/e1)^2 = 1 with
// e0 >= e1 > 0, for points outside it: bisection on the Lagrange parameter of
// the closest-point condition (D. Eberly, "Distance from a point to an
// ellipse, an ellipsoid, or a hyperellipsoid", Geometric Tools); shared by the
// host set-up and the device near-set kernels.
__host__ __device__ inline double ellipse_distance_hd(double e0, double e1, double y0, double y1) {
  if (y1 > 0.0) {
    if (y0 > 0.0) {
      const double z0 = y0 / e0, z1 = y1 / e1;
      const double g0 = z0 * z0 + z1 * z1 - 1.0;
      if (g0 == 0.0) return 0.0;
      const double r0 = (e0 / e1) * (e0 / e1);
      const double n0 = r0 * z0;
      double s0 = z1 - 1.0;
      double s1 = (g0 < 0.0) ? 0.0 : hypot(n0, z1) - 1.0;
      double s = 0.0;
      for (int it = 0; it < 2000; ++it) {
        s = 0.5 * (s0 + s1);
        if (s == s0 || s == s1) break;
        const double r0s = n0 / (s + r0), r1s = z1 / (s + 1.0);
        const double g = r0s * r0s + r1s * r1s - 1.0;
        if (g > 0.0) s0 = s;
        else if (g < 0.0) s1 = s;
        else break;
      }
      const double x0 = r0 * y0 / (s + r0), x1 = y1 / (s + 1.0);
      return hypot(x0 - y0, x1 - y1);
    }
    return fabs(y1 - e1);
  }
  const double num = e0 * y0, den = e0 * e0 - e1 * e1;
  if (num < den) {
    const double xd = num / den;
    const double x0 = e0 * xd, x1 = e1 * sqrt(fmax(0.0, 1.0 - xd * xd));
    return hypot(x0 - y0, x1);
  }
  return fabs(y0 - e0);
}

// Local Cartesian -> (u, v, sqrt(1-v^2), cos phi, sin phi) for a spheroid with
// half focal distance a.  Cancellation-free positive root of the quadratic
//   prolate: s = u^2-1,  s^2 + (1 - R^2) s - X^2 = 0
//   oblate:  s = u^2,    s^2 + (1 - R^2) s - Z^2 = 0
// with X = rho/a, Z = z/a, R^2 = X^2 + Z^2; sqrt(1-v^2) = X/sqrt(s) (prolate)
// or X/sqrt(1+s) (oblate) avoids cancellation at the poles.
struct SphCoord {
  double u, v, sv, cph, sph;
};

__host__ __device__ inline SphCoord to_spheroidal(double x, double y, double z, double a, int kind) {
  const double ia = 1.0 / a;
  const double X = sqrt(x * x + y * y) * ia;
  const double Z = z * ia;
  const double B = (1.0 - X) * (1.0 + X) - Z * Z;   // 1 - R^2
  const double cst = (kind == SBIO_PROLATE) ? X * X : Z * Z;
  const double disc = sqrt(B * B + 4.0 * cst);
  const double s = (B > 0.0) ? (2.0 * cst) / (B + disc) : 0.5 * (disc - B);
  SphCoord o;
  if (kind == SBIO_PROLATE) {
    o.u = sqrt(1.0 + s);
    o.sv = (s > 0.0) ? X / sqrt(s) : 1.0;
  } else {
    o.u = sqrt(s);
    o.sv = X / sqrt(1.0 + s);
  }
  o.v = (o.u > 0.0) ? Z / o.u : 0.0;
  if (o.sv > 1.0) o.sv = 1.0;
  if (o.v > 1.0) o.v = 1.0;
  if (o.v < -1.0) o.v = -1.0;
  const double rho = X * a;
  if (rho > 0.0) {
    o.cph = x / rho;
    o.sph = y / rho;
  } else {
    o.cph = 1.0;
    o.sph = 0.0;
  }
  return o;
}

// Largest aspect ratio accepted: the Miller sweeps start about 19/mu steps
// above the top order, mu = atanh(1/aspect ratio) on the surface, which is
// 38,000 steps at this bound.
constexpr double kMaxAspectRatio = 2000.0;
constexpr int kMaxMillerExtra = 1 << 16;

// Number of extra Miller steps for relative start error < ~1e-16
// (e^{-2 mu K} < 1e-16 with mu = acosh(u) or asinh(u)).
__host__ __device__ inline int miller_extra(double u, double sgn) {
  const double mu = log(u + sqrt(u * u + sgn));   // acosh(u) or asinh(u)
  const double k = ceil(19.0 / mu) + 2.0;
  int K = k > (double)kMaxMillerExtra ? kMaxMillerExtra : (int)k;
  if (K < 4) K = 4;
  return K;
}

// Host/device reference routines with runtime order (used for the per-
// particle multipliers on the host; kernels use their own unrolled forms).
// P family r[nm_index(n,m)] for n <= N.
__host__ __device__ inline void radial_P(double u, double sgn, int N, double* r) {
  const double su = sqrt(u * u + sgn);
  double pmm = 1.0;
  for (int m = 0; m <= N; ++m) {
    if (m > 0) pmm *= (2.0 * m - 1.0) * su;
    r[nm_index(m, m)] = pmm;
    if (m + 1 <= N) r[nm_index(m + 1, m)] = (2.0 * m + 1.0) * u * pmm;
    for (int n = m + 1; n < N; ++n)
      r[nm_index(n + 1, m)] =
          ((2.0 * n + 1.0) * u * r[nm_index(n, m)] + sgn * (n + m) * r[nm_index(n - 1, m)]) / (n - m + 1.0);
  }
}

// Q family q[nm_index(n,m)] for n <= N (N >= 1).
__host__ __device__ inline void radial_Q(double u, double sgn, int N, double* q) {
  const double su = sqrt(u * u + sgn);
  const int K = miller_extra(u, sgn);
  for (int m = 0; m <= 1; ++m) {
    double qp1 = 0.0, qn = 1.0;   // q_{n+1}, q_n (unnormalised) at n = N + K
    int n = N + K;
    for (; n >= 1; --n) {
      if (n <= N) q[nm_index(n, m)] = qn;   // index valid only for n >= m
      const double qm1 = ((2.0 * n + 1.0) * u * qn + sgn * (n - m + 1.0) * qp1) / (n + m);
      qp1 = qn;
      qn = qm1;
      // rescale to keep the sweep in range
      if (fabs(qn) > 1e250) {
        qp1 *= 1e-250;
        qn *= 1e-250;
        for (int k = n; k <= N; ++k)
          if (k >= m && k >= n) q[nm_index(k, m)] *= 1e-250;
      }
    }
    // n == 0 now: qn = q_0, qp1 = q_1
    double scale;
    if (m == 0) {
      scale = 1.0 / (u * qn + sgn * qp1);
      q[nm_index(0, 0)] = qn;
    } else {
      scale = -1.0 / (su * qn);
    }
    for (int k = (m == 0 ? 0 : 1); k <= N; ++k) q[nm_index(k, m)] *= scale;
  }
  const double c = u / su;
  for (int n = 2; n <= N; ++n)
    for (int m = 1; m < n; ++m)
      q[nm_index(n, m + 1)] = -2.0 * m * c * q[nm_index(n, m)] + (n - m + 1.0) * (n + m) * q[nm_index(n, m - 1)];
}

}  // namespace sbio
