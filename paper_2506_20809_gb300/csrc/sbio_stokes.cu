// Stokes single layer (viscosity 1) at all surface nodes through the
// Laplace-to-Stokes identity of Sec. 4.3, eq. (stokes):
//   stokes_prep : per particle, the modified-basis coefficients of y . f at
//                 order p+1 (exact product-quadrature transform), the folded
//                 expansion coefficients of f_1, f_2, f_3, y . f, the
//                 Stokeslet far-field sources w f at the nodes; zeroes u;
//   stokes_near : one thread per (target, near or own particle) pair
//                 (sbio_stokes_near.cuh), FP64, atomically added;
//   stokes_far  : tiled all-pairs Stokeslet quadrature over far particles,
//                 G = (I/r + r r^T/r^3)/(8 pi), FP64 or FP32 with two-sum
//                 compensated accumulation, atomically added.
#include "sbio_internal.cuh"
#include "sbio_stokes_near.cuh"

namespace sbio {

stokes_near_launcher stokes_near_lookup_a(int p);
stokes_near_launcher stokes_near_lookup_b(int p);
stokes_near_launcher stokes_near_lookup_c(int p);

constexpr double kInv8Pi = 0.039788735772973836;   // 1/(8 pi)

__global__ void __launch_bounds__(256) stokes_prep_kernel(
    int p, int n_v, int n_phi, int n_q, int n_f, const PartGeom* __restrict__ parts, const double* __restrict__ xyz,
    const double* __restrict__ w, const double* __restrict__ ptab, const double* __restrict__ trig,
    const double* __restrict__ sqrtw, const double* __restrict__ qv, const double* __restrict__ qw,
    const double* __restrict__ qptab, const double* __restrict__ qtrig, const double* __restrict__ ext,
    const double* __restrict__ normc1, const double* __restrict__ f, double* __restrict__ coef_out,
    double* __restrict__ src64, float4* __restrict__ src32, double* __restrict__ u_out) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  const int p1 = p + 1, nc = (p + 1) * (p + 1), nc1 = (p1 + 1) * (p1 + 1);
  const int nm = nm_count(p), nm1 = nm_count(p1), mw = 2 * p + 1, mw1 = 2 * p1 + 1;
  const int G = n_v * n_phi;
  double* fk = sm;                          // 3 x nc
  double* cy = fk + 3 * nc;                 // nc1
  double* L1 = cy + nc1;                    // 3 x max(n_q, n_v) x mw
  const int nrow = n_q > n_v ? n_q : n_v;
  double* hq = L1 + 3 * nrow * mw;          // n_q x n_f
  double* H = hq + n_q * n_f;               // n_q x mw1
  const PartGeom P = parts[i];
  for (int k = threadIdx.x; k < 3 * nc; k += blockDim.x) fk[k] = f[(size_t)i * 3 * nc + k];
  __syncthreads();
  // (1) Legendre stage of f_d on the transform grid
  for (int idx = threadIdx.x; idx < 3 * n_q * mw; idx += blockDim.x) {
    const int d = idx / (n_q * mw), r = idx - d * n_q * mw, j = r / mw, ms = r - j * mw, m = ms - p;
    const int am = m < 0 ? -m : m;
    const double s2 = m ? 1.4142135623730951 : 1.0;
    double acc = 0.0;
    for (int n = am; n <= p; ++n) acc = fma(fk[d * nc + n * n + n + m], s2 * qptab[(size_t)j * nm1 + nm_index(n, am)], acc);
    L1[(d * n_q + j) * mw + ms] = acc;
  }
  __syncthreads();
  // (2) values of (y - c) . f sqrt(u0^2 -+ v^2) at the grid points
  for (int idx = threadIdx.x; idx < n_q * n_f; idx += blockDim.x) {
    const int j = idx / n_f, l = idx - j * n_f;
    const double* tr = qtrig + (size_t)l * (p1 + 1) * 2;
    double Fd[3];
    for (int d = 0; d < 3; ++d) {
      const double* L = L1 + (d * n_q + j) * mw + p;
      double acc = L[0];
      for (int m = 1; m <= p; ++m) acc = fma(L[m], tr[2 * m], fma(L[-m], tr[2 * m + 1], acc));
      Fd[d] = acc;
    }
    const double v = qv[j], sv = sqrt((1.0 - v) * (1.0 + v));
    const double yl0 = P.A * sv * tr[2], yl1 = P.A * sv * tr[3], yl2 = P.C * v;   // cos phi, sin phi at m = 1
    double acc = 0.0;
    for (int d = 0; d < 3; ++d) acc = fma(P.R[d * 3 + 0] * yl0 + P.R[d * 3 + 1] * yl1 + P.R[d * 3 + 2] * yl2, Fd[d], acc);
    hq[idx] = acc;
  }
  __syncthreads();
  // (3) Fourier projection, |m| <= p+1
  for (int idx = threadIdx.x; idx < n_q * mw1; idx += blockDim.x) {
    const int j = idx / mw1, ms = idx - j * mw1, m = ms - p1, am = m < 0 ? -m : m;
    double acc = 0.0;
    for (int l = 0; l < n_f; ++l) acc = fma(hq[j * n_f + l], qtrig[((size_t)l * (p1 + 1) + am) * 2 + (m < 0 ? 1 : 0)], acc);
    H[idx] = acc * (2.0 * kPi / n_f);
  }
  __syncthreads();
  // (4) Legendre projection -> y.f coefficients of order p+1
  for (int k = threadIdx.x; k < nc1; k += blockDim.x) {
    const int n = (int)sqrt((double)k);
    const int m = k - n * n - n, am = m < 0 ? -m : m;
    const double s2 = m ? 1.4142135623730951 : 1.0;
    double acc = 0.0;
    for (int j = 0; j < n_q; ++j) acc = fma(qw[j] * H[j * mw1 + m + p1], s2 * qptab[(size_t)j * nm1 + nm_index(n, am)], acc);
    cy[k] = acc;
  }
  __syncthreads();
  // (5) folded coefficients of the four expansions (order p+1)
  for (int k = threadIdx.x; k < 4 * nc1; k += blockDim.x) {
    const int d = k / nc1, c = k - d * nc1;
    const int n = (int)sqrt((double)c);
    const int m = c - n * n - n, am = m < 0 ? -m : m;
    const double raw = (d < 3) ? (c < nc ? fk[d * nc + c] : 0.0) : cy[c];
    coef_out[(size_t)i * 4 * nc1 + k] = ext[(size_t)i * nm1 + nm_index(n, am)] * normc1[c] * raw;
  }
  // (6) far sources: w f at the own nodes (Legendre stage reuses L1)
  __syncthreads();
  for (int idx = threadIdx.x; idx < 3 * n_v * mw; idx += blockDim.x) {
    const int d = idx / (n_v * mw), r = idx - d * n_v * mw, j = r / mw, ms = r - j * mw, m = ms - p;
    const int am = m < 0 ? -m : m;
    const double s2 = m ? 1.4142135623730951 : 1.0;
    double acc = 0.0;
    for (int n = am; n <= p; ++n) acc = fma(fk[d * nc + n * n + n + m], s2 * ptab[(size_t)j * nm + nm_index(n, am)], acc);
    L1[(d * n_v + j) * mw + ms] = acc;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < G; l += blockDim.x) {
    const int j = l / n_phi, k = l - j * n_phi;
    const double* tr = trig + (size_t)k * (p + 1) * 2;
    const int64_t t = (int64_t)i * G + l;
    const double ws = w[t] / sqrtw[(size_t)i * n_v + j];
    double fw[3];
    for (int d = 0; d < 3; ++d) {
      const double* L = L1 + (d * n_v + j) * mw + p;
      double acc = L[0];
      for (int m = 1; m <= p; ++m) acc = fma(L[m], tr[2 * m], fma(L[-m], tr[2 * m + 1], acc));
      fw[d] = acc * ws;
    }
    const double y0 = xyz[t * 3 + 0] - P.c[0], y1 = xyz[t * 3 + 1] - P.c[1], y2 = xyz[t * 3 + 2] - P.c[2];
    double* s = src64 + t * 8;
    s[0] = y0; s[1] = y1; s[2] = y2; s[3] = fw[0];
    s[4] = fw[1]; s[5] = fw[2]; s[6] = 0.0; s[7] = 0.0;
    src32[t * 2 + 0] = make_float4((float)y0, (float)y1, (float)y2, (float)fw[0]);
    src32[t * 2 + 1] = make_float4((float)fw[1], (float)fw[2], 0.f, 0.f);
  }
}

// Self term (own particle) at u = u0, separable: for each of the four
// expansions the value and the three unit-vector derivatives are inverse
// transforms of the folded coefficients times q(u0) or q'(u0), with the
// Ferrers tables P, sqrt(1-v^2) dP/dv and m P / sqrt(1-v^2) at the GL nodes
// (the exterior limit of eq. (dSLevalformula) applied mode by mode).  The
// velocity is linear in the four expansions, so CTA (i, y) takes expansions
// 2y and 2y + 1 of particle i and adds its share to u (zeroed beforehand):
// 1/2 F_k to component k and -1/2 R X_k grad F_k for k < 3, 1/2 R grad F_y.
__global__ void __launch_bounds__(256) stokes_self_kernel(int p, int n_v, int n_phi, const PartGeom* __restrict__ parts,
                                                          const double* __restrict__ xyz,
                                                          const double* __restrict__ coef,
                                                          const double* __restrict__ qu0,
                                                          const double* __restrict__ dqu0,
                                                          const double* __restrict__ fP,
                                                          const double* __restrict__ fV,
                                                          const double* __restrict__ fF,
                                                          const double* __restrict__ trig1,
                                                          const double* __restrict__ gl_v,
                                                          double* __restrict__ u_out) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  const int p1 = p + 1, nc1 = (p1 + 1) * (p1 + 1), nm1 = nm_count(p1), mw1 = 2 * p1 + 1;
  const int G = n_v * n_phi;
  const PartGeom P = parts[i];
  const int d0 = 2 * blockIdx.y;                // expansions d0, d0 + 1
  const double* cf = coef + (size_t)i * 4 * nc1 + (size_t)d0 * nc1;
  const double* q0 = qu0 + (size_t)i * nm1;
  const double* dq0 = dqu0 + (size_t)i * nm1;
  // L[(dd * 4 + qty) * n_v + j][ms]: qty 0 value, 1 d/du, 2 sv d/dv, 3 d/dphi / sv
  for (int idx = threadIdx.x; idx < 8 * n_v * mw1; idx += blockDim.x) {
    const int row = idx / mw1, ms = idx - row * mw1, m = ms - p1, am = m < 0 ? -m : m;
    const int dq = row / n_v, j = row - dq * n_v, dd = dq >> 2, qty = dq & 3;
    const double* tab = (qty == 2) ? fV : (qty == 3 ? fF : fP);
    const double* rad = (qty == 1) ? dq0 : q0;
    double acc = 0.0;
    for (int n = am; n <= p1; ++n)
      acc = fma(cf[dd * nc1 + n * n + n + m] * rad[nm_index(n, am)], tab[(size_t)j * nm1 + nm_index(n, am)], acc);
    sm[idx] = acc;
  }
  __syncthreads();
  const double sgn = P.sgn, u = P.u0;
  const double su = P.A / P.a;                  // sqrt(u0^2 + sgn)
  const double ia = 1.0 / P.a;
  for (int l = threadIdx.x; l < G; l += blockDim.x) {
    const int j = l / n_phi, k = l - j * n_phi;
    const double* tr = trig1 + (size_t)k * (p1 + 1) * 2;
    double F[2][4];
    for (int dq = 0; dq < 8; ++dq) {
      const double* L = sm + ((size_t)dq * n_v + j) * mw1 + p1;
      double acc;
      if ((dq & 3) == 3) {   // d/dphi: cos -> -m sin, sin -> m cos (m inside the table)
        acc = 0.0;
        for (int m = 1; m <= p1; ++m) acc = fma(-L[m], tr[2 * m + 1], fma(L[-m], tr[2 * m], acc));
      } else {
        acc = L[0];
        for (int m = 1; m <= p1; ++m) acc = fma(L[m], tr[2 * m], fma(L[-m], tr[2 * m + 1], acc));
      }
      F[dq >> 2][dq & 3] = acc;
    }
    const double v = gl_v[j], sv = sqrt((1.0 - v) * (1.0 + v));
    const double c1 = tr[2], s1 = tr[3];
    const double iW = rsqrt(u * u + sgn * v * v);
    const double eu0 = u * sv * c1 * iW, eu1 = u * sv * s1 * iW, eu2 = v * su * iW;
    const double ev0 = -su * v * c1 * iW, ev1 = -su * v * s1 * iW, ev2 = u * sv * iW;
    const int64_t t = (int64_t)i * G + l;
    const double X[3] = {xyz[t * 3 + 0] - P.c[0], xyz[t * 3 + 1] - P.c[1], xyz[t * 3 + 2] - P.c[2]};
    double w[3] = {0.0, 0.0, 0.0}, val[3] = {0.0, 0.0, 0.0};
    for (int dd = 0; dd < 2; ++dd) {
      const int d = d0 + dd;
      const double gu = F[dd][1] * su * ia * iW, gv = F[dd][2] * ia * iW, gp = F[dd][3] * ia / su;
      const double g[3] = {gu * eu0 + gv * ev0 - gp * s1, gu * eu1 + gv * ev1 + gp * c1, gu * eu2 + gv * ev2};
      const double wt = (d == 3) ? 1.0 : -X[d];   // grad F_y - sum_j X_j grad F_j
      for (int c = 0; c < 3; ++c) w[c] = fma(wt, g[c], w[c]);
      if (d < 3) val[d] = F[dd][0];
    }
    for (int c = 0; c < 3; ++c)
      atomicAdd(u_out + t * 3 + c,
                0.5 * (val[c] + P.R[c * 3 + 0] * w[0] + P.R[c * 3 + 1] * w[1] + P.R[c * 3 + 2] * w[2]));
  }
}

struct alignas(32) dbl4s {
  double x, y, z, w;
};

__global__ void __launch_bounds__(kFarTile) stokes_far_fp64_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                                   const double* __restrict__ src64,
                                                                   const double* __restrict__ xyz,
                                                                   const PartGeom* __restrict__ parts,
                                                                   const int32_t* __restrict__ skip_ptr,
                                                                   const int32_t* __restrict__ skip_idx, int64_t N,
                                                                   double* __restrict__ u_out) {
  __shared__ dbl4s sh[kFarTile * 2];
  const int64_t t = (int64_t)blockIdx.x * kFarTile + threadIdx.x;
  const bool valid = t < N;
  double x = 0, y = 0, z = 0;
  int sp = 0, nxt = INT32_MAX;
  if (valid) {
    x = xyz[t * 3 + 0];
    y = xyz[t * 3 + 1];
    z = xyz[t * 3 + 2];
    sp = skip_ptr[t];
    nxt = skip_idx[sp];
  }
  double a0 = 0, a1 = 0, a2 = 0;
  int cur = -1;
  bool skip = true;
  double X = 0, Y = 0, Z = 0;
  const int per = (n_tiles + gridDim.y - 1) / gridDim.y;
  const int t_lo = blockIdx.y * per, t_hi = min(n_tiles, t_lo + per);
  for (int tl = t_lo; tl < t_hi; ++tl) {
    const int4 tile = tiles[tl];
    if (tile.x != cur) {
      cur = tile.x;
      if (valid) {
        while (nxt < cur) nxt = skip_idx[++sp];
        skip = (nxt == cur);
        X = x - parts[cur].c[0];
        Y = y - parts[cur].c[1];
        Z = z - parts[cur].c[2];
      }
    }
    if (__syncthreads_and(skip)) continue;
    if (threadIdx.x < tile.z) {
      const dbl4s* s = reinterpret_cast<const dbl4s*>(src64 + (int64_t)(tile.y + threadIdx.x) * 8);
      sh[threadIdx.x * 2 + 0] = s[0];
      sh[threadIdx.x * 2 + 1] = s[1];
    }
    __syncthreads();
    if (!skip) {
      for (int j = 0; j < tile.z; ++j) {
        const dbl4s A = sh[j * 2], B = sh[j * 2 + 1];
        const double dx = X - A.x, dy = Y - A.y, dz = Z - A.z;
        const double ri = rsqrt(dx * dx + dy * dy + dz * dz);
        const double rf = (dx * A.w + dy * B.x + dz * B.y) * ri * ri * ri;
        a0 += A.w * ri + rf * dx;
        a1 += B.x * ri + rf * dy;
        a2 += B.y * ri + rf * dz;
      }
    }
    __syncthreads();
  }
  if (valid) {
    atomicAdd(u_out + t * 3 + 0, a0 * kInv8Pi);
    atomicAdd(u_out + t * 3 + 1, a1 * kInv8Pi);
    atomicAdd(u_out + t * 3 + 2, a2 * kInv8Pi);
  }
}

// Stokeslet far field for one CTA: TT targets per thread against source tiles
// [t_lo, t_hi); two-sum accumulators and skip cursors in shared memory (as in
// the Laplace far kernel); PK computes two targets per f32x2 instruction.
// PR also sums the pressure quadrature with the printed kernel
// P = r / (4 pi |r|^3), which reuses the pair's f.r and 1/|r|: one more FMA.
// One CTA: targets [t_first, min(N, t_first + kFarTile * TT)) against source
// tiles [t_lo, t_hi) (the launch grid or a treecode group's tile list).
template <int TT, bool PK, bool PR>
__device__ __forceinline__ void stokes_far_block(int64_t t_first, int64_t N, int t_lo, int t_hi,
                                                 const int4* __restrict__ tiles, const float4* __restrict__ src32,
                                                 const float4* __restrict__ tgt32, const float4* __restrict__ cen32,
                                                 const int32_t* __restrict__ skip_ptr,
                                                 const int32_t* __restrict__ skip_idx, double* __restrict__ u_out,
                                                 double* __restrict__ p_out) {
  constexpr int NA = PR ? 4 : 3;               // accumulated quantities per target
  __shared__ float4 sh[(PK ? 3 : 2) * kFarTile];
  __shared__ float acc[2 * NA * TT * kFarTile];   // per target: (hi, lo) of u_x, u_y, u_z (and p)
  __shared__ int cursor[2 * TT * kFarTile];
  const int tid = threadIdx.x;
  const int64_t t0 = t_first + tid;
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    const int64_t t = t0 + (int64_t)q * kFarTile;
#pragma unroll
    for (int c = 0; c < 2 * NA; ++c) acc[(2 * NA * q + c) * kFarTile + tid] = 0.f;
    const int sp = (t < N) ? skip_ptr[t] : 0;
    cursor[(2 * q + 0) * kFarTile + tid] = sp;
    cursor[(2 * q + 1) * kFarTile + tid] = (t < N) ? skip_idx[sp] : INT32_MAX;
  }
  float X[TT], Y[TT], Z[TT];
  unsigned skipmask = (1u << TT) - 1u;
  int cur = -1;
  for (int tl = t_lo; tl < t_hi; ++tl) {
    const int4 tile = tiles[tl];
    if (tile.x != cur) {
      cur = tile.x;
      const float4 ch = cen32[cur * 2], cl = cen32[cur * 2 + 1];
      skipmask = 0u;
#pragma unroll
      for (int q = 0; q < TT; ++q) {
        const int64_t t = t0 + (int64_t)q * kFarTile;
        int sp = cursor[(2 * q + 0) * kFarTile + tid];
        int nxt = cursor[(2 * q + 1) * kFarTile + tid];
        while (nxt < cur) nxt = skip_idx[++sp];
        cursor[(2 * q + 0) * kFarTile + tid] = sp;
        cursor[(2 * q + 1) * kFarTile + tid] = nxt;
        if (t >= N || nxt == cur) skipmask |= 1u << q;
        float4 hi = make_float4(0.f, 0.f, 0.f, 0.f), lo = hi;
        if (t < N) {
          hi = tgt32[t * 2];
          lo = tgt32[t * 2 + 1];
        }
        X[q] = (hi.x - ch.x) + (lo.x - cl.x);
        Y[q] = (hi.y - ch.y) + (lo.y - cl.y);
        Z[q] = (hi.z - ch.z) + (lo.z - cl.z);
      }
    }
    const bool mine = skipmask != (1u << TT) - 1u;
    if (!__syncthreads_or(mine)) continue;
    if (tid < tile.z) {
      const float4 A = src32[(int64_t)(tile.y + tid) * 2 + 0];
      const float4 B = src32[(int64_t)(tile.y + tid) * 2 + 1];
      if (PK) {
        sh[tid * 3 + 0] = make_float4(-A.x, -A.x, -A.y, -A.y);
        sh[tid * 3 + 1] = make_float4(-A.z, -A.z, A.w, A.w);
        sh[tid * 3 + 2] = make_float4(B.x, B.x, B.y, B.y);
      } else {
        sh[tid * 2 + 0] = A;
        sh[tid * 2 + 1] = B;
      }
    }
    __syncthreads();
    if (mine) {
      float p0[TT], p1[TT], p2[TT], p3[TT];
      if constexpr (PK) {
        constexpr int TP = TT / 2 > 0 ? TT / 2 : 1;
        float2 Xp[TP], Yp[TP], Zp[TP], a0[TP], a1[TP], a2[TP], a3[TP];
#pragma unroll
        for (int k = 0; k < TP; ++k) {
          Xp[k] = make_float2(X[2 * k], X[2 * k + 1]);
          Yp[k] = make_float2(Y[2 * k], Y[2 * k + 1]);
          Zp[k] = make_float2(Z[2 * k], Z[2 * k + 1]);
          a0[k] = a1[k] = a2[k] = a3[k] = make_float2(0.f, 0.f);
        }
#pragma unroll 2
        for (int j = 0; j < tile.z; ++j) {
          const float4 A = sh[j * 3 + 0], B = sh[j * 3 + 1], Cc = sh[j * 3 + 2];
          const float2 myx = make_float2(A.x, A.y), myy = make_float2(A.z, A.w), myz = make_float2(B.x, B.y);
          const float2 fx = make_float2(B.z, B.w), fy = make_float2(Cc.x, Cc.y), fz = make_float2(Cc.z, Cc.w);
#pragma unroll
          for (int k = 0; k < TP; ++k) {
            const float2 dx = __fadd2_rn(Xp[k], myx), dy = __fadd2_rn(Yp[k], myy), dz = __fadd2_rn(Zp[k], myz);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 ri = make_float2(rsqrt_f32(r2.x), rsqrt_f32(r2.y));
            const float2 rf = __ffma2_rn(fz, dz, __ffma2_rn(fy, dy, __fmul2_rn(fx, dx)));
            // f / r + (f.r) r / r^3 = (1/r) (f + t r), t = (f.r) / r^2
            const float2 t = __fmul2_rn(rf, __fmul2_rn(ri, ri));
            a0[k] = __ffma2_rn(ri, __ffma2_rn(t, dx, fx), a0[k]);
            a1[k] = __ffma2_rn(ri, __ffma2_rn(t, dy, fy), a1[k]);
            a2[k] = __ffma2_rn(ri, __ffma2_rn(t, dz, fz), a2[k]);
            if (PR) a3[k] = __ffma2_rn(t, ri, a3[k]);   // (f.r) / r^3
          }
        }
#pragma unroll
        for (int k = 0; k < TP; ++k) {
          p0[2 * k] = a0[k].x; p0[2 * k + 1] = a0[k].y;
          p1[2 * k] = a1[k].x; p1[2 * k + 1] = a1[k].y;
          p2[2 * k] = a2[k].x; p2[2 * k + 1] = a2[k].y;
          p3[2 * k] = a3[k].x; p3[2 * k + 1] = a3[k].y;
        }
      } else {
#pragma unroll
        for (int q = 0; q < TT; ++q) p0[q] = p1[q] = p2[q] = p3[q] = 0.f;
#pragma unroll 2
        for (int j = 0; j < tile.z; ++j) {
          const float4 A = sh[j * 2], B = sh[j * 2 + 1];
#pragma unroll
          for (int q = 0; q < TT; ++q) {
            const float dx = X[q] - A.x, dy = Y[q] - A.y, dz = Z[q] - A.z;
            const float ri = rsqrt_f32(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            const float rf = fmaf(dz, B.y, fmaf(dy, B.x, dx * A.w));
            const float t = rf * (ri * ri);
            p0[q] = fmaf(ri, fmaf(t, dx, A.w), p0[q]);
            p1[q] = fmaf(ri, fmaf(t, dy, B.x), p1[q]);
            p2[q] = fmaf(ri, fmaf(t, dz, B.y), p2[q]);
            if (PR) p3[q] = fmaf(t, ri, p3[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < TT; ++q) {
        if (!((skipmask >> q) & 1u)) {
          const float pv[4] = {p0[q], p1[q], p2[q], p3[q]};
#pragma unroll
          for (int c = 0; c < NA; ++c) {
            float sum, err;
            two_sum_f32(acc[(2 * NA * q + 2 * c) * kFarTile + tid], pv[c], sum, err);
            acc[(2 * NA * q + 2 * c) * kFarTile + tid] = sum;
            acc[(2 * NA * q + 2 * c + 1) * kFarTile + tid] += err;
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    const int64_t t = t0 + (int64_t)q * kFarTile;
    if (t < N) {
      for (int c = 0; c < 3; ++c)
        atomicAdd(u_out + t * 3 + c,
                  ((double)acc[(2 * NA * q + 2 * c) * kFarTile + tid] +
                   (double)acc[(2 * NA * q + 2 * c + 1) * kFarTile + tid]) * kInv8Pi);
      if (PR)
        atomicAdd(p_out + t, ((double)acc[(2 * NA * q + 6) * kFarTile + tid] +
                              (double)acc[(2 * NA * q + 7) * kFarTile + tid]) * (2.0 * kInv8Pi));
    }
  }
  __syncthreads();   // the shared arrays may be reused by a following block of the same CTA
}

template <int TT, bool PK, bool PR>
__global__ void __launch_bounds__(kFarTile) stokes_far_mixed_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                                    const float4* __restrict__ src32,
                                                                    const float4* __restrict__ tgt32,
                                                                    const float4* __restrict__ cen32,
                                                                    const int32_t* __restrict__ skip_ptr,
                                                                    const int32_t* __restrict__ skip_idx, int64_t N,
                                                                    double* __restrict__ u_out,
                                                                    double* __restrict__ p_out) {
  const int per = (n_tiles + gridDim.y - 1) / gridDim.y;
  const int t_lo = blockIdx.y * per, t_hi = min(n_tiles, t_lo + per);
  stokes_far_block<TT, PK, PR>((int64_t)blockIdx.x * TT * kFarTile, N, t_lo, t_hi, tiles, src32, tgt32, cen32,
                               skip_ptr, skip_idx, u_out, p_out);
}

// Direct part of the Stokes treecode far field: one CTA per item (target
// group [groups[g].x, groups[g].y), tile range of the group's tile list).
__global__ void __launch_bounds__(kFarTile) stokes_far_tile_items_kernel(
    const int4* __restrict__ items, const int2* __restrict__ groups, const int4* __restrict__ tiles,
    const float4* __restrict__ src32, const float4* __restrict__ tgt32, const float4* __restrict__ cen32,
    const int32_t* __restrict__ skip_ptr, const int32_t* __restrict__ skip_idx, double* __restrict__ u_out) {
  const int4 w = items[blockIdx.x];
  const int2 grp = groups[w.x];
  stokes_far_block<2, true, false>(grp.x, grp.y, w.y, w.z, tiles, src32, tgt32, cen32, skip_ptr, skip_idx, u_out,
                                   nullptr);
}

void launch_stokes_far_tile_items(const DevGeom& d, const int2* groups, const int4* tiles, const int4* items,
                                  int n_items, double* u, cudaStream_t st) {
  if (n_items <= 0) return;
  stokes_far_tile_items_kernel<<<n_items, kFarTile, 0, st>>>(items, groups, tiles, d.st_src32, d.tgt32, d.cen32,
                                                             d.skip_ptr, d.skip_idx, u);
  count_launch();
}

template <int TT, bool PK>
static void launch_stokes_far_tt(const DevGeom& d, const GeomHost& h, int64_t NT, double* u, double* pr,
                                 cudaStream_t st) {
  const int nt = (int)h.tiles.size();
  const int64_t tb = (NT + (int64_t)kFarTile * TT - 1) / ((int64_t)kFarTile * TT);
  const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, h.st_far_splits));
  if (pr)
    stokes_far_mixed_kernel<TT, PK, true><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.st_src32, d.tgt32, d.cen32,
                                                                     d.skip_ptr, d.skip_idx, NT, u, pr);
  else
    stokes_far_mixed_kernel<TT, PK, false><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.st_src32, d.tgt32, d.cen32,
                                                                      d.skip_ptr, d.skip_idx, NT, u, nullptr);
}

// The Stokeslet far field alone (sources written by the prep kernel of the
// same or an earlier apply) at the NT targets of `d`, in the geometry's
// precision and Stokes launch shape.  pr (may be null): the pressure
// quadrature is summed into it in the same pass (mixed precision only; the
// FP64 form leaves it to a kernel of its own).
int launch_stokes_far_on(const DevGeom& d, const GeomHost& h, int64_t NT, double* u, double* pr, cudaStream_t st) {
  if (NT <= 0) return SBIO_OK;
  const int nt = (int)h.tiles.size();
  if (h.precision == SBIO_FP64) {
    if (pr) return set_error(SBIO_EINVAL, "the FP64 Stokeslet far kernel does not sum the pressure");
    const int64_t tb = (NT + kFarTile - 1) / kFarTile;
    const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, h.st_far_splits));
    stokes_far_fp64_kernel<<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.st_src64, d.xyz, d.parts, d.skip_ptr,
                                                      d.skip_idx, NT, u);
  } else {
    // targets per thread, packed f32x2 form if negative
    switch (h.st_far_tt) {
      case 1: launch_stokes_far_tt<1, false>(d, h, NT, u, pr, st); break;
      case 4: launch_stokes_far_tt<4, false>(d, h, NT, u, pr, st); break;
      case 8: launch_stokes_far_tt<8, false>(d, h, NT, u, pr, st); break;
      case -2: launch_stokes_far_tt<2, true>(d, h, NT, u, pr, st); break;
      case -4: launch_stokes_far_tt<4, true>(d, h, NT, u, pr, st); break;
      case -8: launch_stokes_far_tt<8, true>(d, h, NT, u, pr, st); break;
      default: launch_stokes_far_tt<2, false>(d, h, NT, u, pr, st); break;
    }
  }
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}

int launch_stokes_far(sbio_geom* g, double* u, cudaStream_t st) {
  // the treecode replaces the direct Stokeslet sum for mixed applies at the nodes
  if (g->tree && g->h.precision == SBIO_MIXED) return launch_tree_stokes_far(g, u, st);
  return launch_stokes_far_on(g->d, g->h, g->h.N, u, nullptr, st);
}

// Per-apply Stokes sources: the y.f coefficients at order p+1 and the folded
// near coefficients (st_coef), and the Stokeslet far sources (st_src64/32).
int launch_stokes_prep(sbio_geom* g, const double* f, cudaStream_t st) {
  const GeomHost& h = g->h;
  const DevGeom& d = g->d;
  const int p = h.p;
  const int p1 = p + 1, nc = (p + 1) * (p + 1), nc1 = (p1 + 1) * (p1 + 1), mw = 2 * p + 1, mw1 = 2 * p1 + 1;
  const int nrow = h.n_q > h.n_v ? h.n_q : h.n_v;
  const size_t smem = (size_t)(3 * nc + nc1 + 3 * nrow * mw + h.n_q * h.n_f + h.n_q * mw1) * sizeof(double);
  if (smem > 48 * 1024)
    SBIO_CUDA_TRY(cudaFuncSetAttribute(stokes_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  stokes_prep_kernel<<<h.M, 256, smem, st>>>(p, h.n_v, h.n_phi, h.n_q, h.n_f, d.parts, d.xyz, d.w, d.ptab, d.trig,
                                             d.sqrtw, d.st_qv, d.st_qw, d.st_qptab, d.st_qtrig, d.st_ext,
                                             d.st_normc, f, d.st_coef, d.st_src64, d.st_src32, nullptr);
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}

int launch_stokes(sbio_geom* g, const double* f, double* u, cudaStream_t st) {
  const GeomHost& h = g->h;
  const DevGeom& d = g->d;
  const int p = h.p;
  if (p > 20) return set_error(SBIO_ENOTSUP, "Stokes single layer is built for p <= 20 (p = %d)", p);
  stokes_near_launcher nl = stokes_near_lookup_a(p);
  if (!nl) nl = stokes_near_lookup_b(p);
  if (!nl) nl = stokes_near_lookup_c(p);
  if (!nl) return set_error(SBIO_ENOTSUP, "no Stokes near-field kernel for p = %d", p);
  const int p1 = p + 1, mw1 = 2 * p1 + 1;
  phase_mark(g, 0, st);
  int rc0 = launch_stokes_prep(g, f, st);
  if (rc0) return rc0;
  const size_t smem_self = (size_t)8 * h.n_v * mw1 * sizeof(double);
  if (smem_self > 48 * 1024)
    SBIO_CUDA_TRY(cudaFuncSetAttribute(stokes_self_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_self));
  SBIO_CUDA_TRY(cudaMemsetAsync(u, 0, (size_t)h.N * 3 * sizeof(double), st));
  stokes_self_kernel<<<dim3(h.M, 2), 256, smem_self, st>>>(p, h.n_v, h.n_phi, d.parts, d.xyz, d.st_coef, d.st_qu0, d.st_dqu0,
                                                  d.st_fP, d.st_fV, d.st_fF, d.st_trig1, d.st_glv, u);
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  phase_mark(g, 1, st);
  // the FP64 near kernels run beside the FP32 Stokeslet kernel unless phases
  // are being timed one by one
  const bool fork = g->overlap && !g->timing && g->near_stream && !h.pair_t.empty();
  SideFork sf;
  if (fork) {
    SBIO_CUDA_TRY(sf.fork(g, st));
    g->d.near_grid_cap = h.st_near_ctas_per_sm > 0 ? h.st_near_ctas_per_sm * sm_count() : 0;
    nl(g->d, h.n_pairs_prolate, (int64_t)h.pair_t.size(), d.inv, u, g->near_stream);
    g->d.near_grid_cap = 0;
    SBIO_CUDA_TRY(cudaGetLastError());
  } else if (!h.pair_t.empty()) {
    nl(d, h.n_pairs_prolate, (int64_t)h.pair_t.size(), d.inv, u, st);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  phase_mark(g, 2, st);
  int rc = launch_stokes_far(g, u, st);
  if (rc) return rc;
  SBIO_CUDA_TRY(sf.join());
  phase_mark(g, 3, st);
  return SBIO_OK;
}

}  // namespace sbio
