// Stokes double layer (viscosity 1) through Laplace potentials.
//
// The paper remarks (Sec. 4.3) that the Stokes double layer can be written in
// terms of Laplace double-layer potentials and their gradients.  With the
// stresslet D_stk[q](x)_i = 3/(4 pi) int (r.q)(r.nu) r_i / |r|^5 dS, r = x - y
// (the sign giving D_stk[const] = -q inside, like the Laplace double layer),
//     D_stk[q]_i = -x_i sum_j d_j D[q_j] + sum_j d_j D[y_i q_j] - d_i S[q . nu],
// x, y measured from the source particle's centre.  Per particle the prep
// kernel forms the thirteen exterior expansions, exact at order p + 1: the
// q_l (plain input coefficients), the y_i q_l (plain) and q . nu (modified
// basis, since nu sqrt(u0^2 -+ v^2) is of degree one), with the density
// index l of the first twelve in the particle's local frame
// (q_l = sum_j R_jl q_j, so that sum_j d_j acts as a local divergence), by the product
// quadrature of the Stokes grid ((p+2) GL x (2p+4) trapezoid), folded with
// the exterior factors of Theorems 1-2 and the normalisation; it also writes
// the far-field sources and, for the on-surface apply, initialises the output
// with -q/2 (principal value = exterior limit - q/2).  Near pairs evaluate
// the gradients pair by pair (sbio_stokes_dl_near.cuh), the own nodes take the
// exterior limit separably (sdl_self_kernel), far pairs use the stresslet
// quadrature here.
#include <algorithm>

#include "sbio_internal.cuh"
#include "sbio_stokes_dl_near.cuh"

struct sbio_targets;

namespace sbio {

// one lookup per translation unit of near kernels (orders 1-8, 9-12, then one each)
stokes_dl_near_launcher stokes_dl_near_lookup_a(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_b(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_c(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_d(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_e(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_f(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_g(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_h(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_i(int p);
stokes_dl_near_launcher stokes_dl_near_lookup_j(int p);

namespace {

constexpr double kTwoPiS = 6.283185307179586;
constexpr double k3Over4Pi = 0.238732414637843;   // 3/(4 pi)

__global__ void __launch_bounds__(256) sdl_prep_kernel(
    int p, int n_v, int n_phi, int n_q, int n_f, const PartGeom* __restrict__ parts, const double* __restrict__ xyz,
    const double* __restrict__ w, const double* __restrict__ ptab, const double* __restrict__ trig,
    const double* __restrict__ qv, const double* __restrict__ qw, const double* __restrict__ qptab,
    const double* __restrict__ qtrig, const double* __restrict__ extS1, const double* __restrict__ extD1,
    const double* __restrict__ normc1, const double* __restrict__ qhat, double* __restrict__ coef_out,
    double* __restrict__ src64, float4* __restrict__ src32, double* __restrict__ u_init, double init_factor) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  const int p1 = p + 1, nc = (p + 1) * (p + 1), nc1 = (p1 + 1) * (p1 + 1);
  const int nm = nm_count(p), nm1 = nm_count(p1), mw = 2 * p + 1, mw1 = 2 * p1 + 1;
  const int G = n_v * n_phi;
  const PartGeom P = parts[i];
  double* qh = sm;                              // 3 x nc
  double* Lq = qh + 3 * nc;                     // 3 x max(n_q, n_v) x mw
  const int nrow = n_q > n_v ? n_q : n_v;
  double* hv = Lq + 3 * nrow * mw;              // 10 x n_q x n_f
  double* Hm = hv + 10 * n_q * n_f;             // 10 x n_q x mw1
  for (int k = threadIdx.x; k < 3 * nc; k += blockDim.x) qh[k] = qhat[(size_t)i * 3 * nc + k];
  __syncthreads();
  // (1) far sources and the -q/2 start at the own nodes (surface rows)
  for (int idx = threadIdx.x; idx < 3 * n_v * mw; idx += blockDim.x) {
    const int d = idx / (n_v * mw), r = idx - d * n_v * mw, j = r / mw, ms = r - j * mw, m = ms - p;
    const int am = m < 0 ? -m : m;
    const double s2 = m ? 1.4142135623730951 : 1.0;
    double acc = 0.0;
    for (int n = am; n <= p; ++n) acc = fma(qh[d * nc + n * n + n + m], s2 * ptab[(size_t)j * nm + nm_index(n, am)], acc);
    Lq[(d * n_v + j) * mw + ms] = acc;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < G; l += blockDim.x) {
    const int j = l / n_phi, k = l - j * n_phi;
    const double* tr = trig + (size_t)k * (p + 1) * 2;
    const int64_t t = (int64_t)i * G + l;
    double qq[3];
    for (int d = 0; d < 3; ++d) {
      const double* L = Lq + (d * n_v + j) * mw + p;
      double acc = L[0];
      for (int m = 1; m <= p; ++m) acc = fma(L[m], tr[2 * m], fma(L[-m], tr[2 * m + 1], acc));
      qq[d] = acc;
    }
    const double wt = w[t];
    const double y0 = xyz[t * 3 + 0] - P.c[0], y1 = xyz[t * 3 + 1] - P.c[1], y2 = xyz[t * 3 + 2] - P.c[2];
    double* s = src64 + t * 8;
    s[0] = y0; s[1] = y1; s[2] = y2; s[3] = wt * qq[0];
    s[4] = wt * qq[1]; s[5] = wt * qq[2]; s[6] = 0.0; s[7] = 0.0;
    src32[t * 2 + 0] = make_float4((float)y0, (float)y1, (float)y2, (float)(wt * qq[0]));
    src32[t * 2 + 1] = make_float4((float)(wt * qq[1]), (float)(wt * qq[2]), 0.f, 0.f);
    if (u_init)
      for (int d = 0; d < 3; ++d) u_init[t * 3 + d] = init_factor * qq[d];
  }
  __syncthreads();
  // (2) q at the product-quadrature rows
  for (int idx = threadIdx.x; idx < 3 * n_q * mw; idx += blockDim.x) {
    const int d = idx / (n_q * mw), r = idx - d * n_q * mw, j = r / mw, ms = r - j * mw, m = ms - p;
    const int am = m < 0 ? -m : m;
    const double s2 = m ? 1.4142135623730951 : 1.0;
    double acc = 0.0;
    for (int n = am; n <= p; ++n) acc = fma(qh[d * nc + n * n + n + m], s2 * qptab[(size_t)j * nm1 + nm_index(n, am)], acc);
    Lq[(d * n_q + j) * mw + ms] = acc;
  }
  __syncthreads();
  // (3) the ten products at the grid points: y_i q_l (local l) and q . (nu sqrt(w))
  const double a = P.a, u0 = P.u0, su0 = sqrt(u0 * u0 + P.sgn);
  for (int l = threadIdx.x; l < n_q * n_f; l += blockDim.x) {
    const int j = l / n_f, k = l - j * n_f;
    const double* tr = qtrig + (size_t)k * (p1 + 1) * 2;
    double qq[3];
    for (int d = 0; d < 3; ++d) {
      const double* L = Lq + (d * n_q + j) * mw + p;
      double acc = L[0];
      for (int m = 1; m <= p; ++m) acc = fma(L[m], tr[2 * m], fma(L[-m], tr[2 * m + 1], acc));
      qq[d] = acc;
    }
    const double v = qv[j], sv = sqrt((1.0 - v) * (1.0 + v)), c1 = tr[2], s1 = tr[3];
    const double yl[3] = {a * su0 * sv * c1, a * su0 * sv * s1, a * u0 * v};
    const double nl[3] = {u0 * sv * c1, u0 * sv * s1, su0 * v};   // nu sqrt(u0^2 + sgn v^2), local frame
    double yg[3], ng[3], ql[3];
    for (int r = 0; r < 3; ++r) {
      yg[r] = P.R[r * 3 + 0] * yl[0] + P.R[r * 3 + 1] * yl[1] + P.R[r * 3 + 2] * yl[2];
      ng[r] = P.R[r * 3 + 0] * nl[0] + P.R[r * 3 + 1] * nl[1] + P.R[r * 3 + 2] * nl[2];
      ql[r] = P.R[0 * 3 + r] * qq[0] + P.R[1 * 3 + r] * qq[1] + P.R[2 * 3 + r] * qq[2];   // q in the local frame
    }
    for (int ii = 0; ii < 3; ++ii)
      for (int jj = 0; jj < 3; ++jj) hv[((3 * ii + jj) * n_q + j) * n_f + k] = yg[ii] * ql[jj];
    hv[(9 * n_q + j) * n_f + k] = qq[0] * ng[0] + qq[1] * ng[1] + qq[2] * ng[2];
  }
  __syncthreads();
  // (4) Fourier sums per row and order, with the quadrature weights
  const double dphi = kTwoPiS / n_f;
  for (int idx = threadIdx.x; idx < 10 * n_q * mw1; idx += blockDim.x) {
    const int d = idx / (n_q * mw1), r = idx - d * n_q * mw1, j = r / mw1, ms = r - j * mw1, m = ms - p1;
    const int am = m < 0 ? -m : m;
    const double* h = hv + (d * n_q + j) * n_f;
    double acc = 0.0;
    for (int k = 0; k < n_f; ++k) acc = fma(h[k], qtrig[((size_t)k * (p1 + 1) + am) * 2 + (m < 0 ? 1 : 0)], acc);
    Hm[idx] = acc * dphi * qw[j];
  }
  __syncthreads();
  // (5) Legendre sums and the fold with exterior factors and normalisation
  double* out = coef_out + (size_t)i * 13 * nc1;
  for (int idx = threadIdx.x; idx < 13 * nc1; idx += blockDim.x) {
    const int d = idx / nc1, k = idx - d * nc1;
    const int n = (int)sqrt((double)k);
    const int m = k - n * n - n, am = m < 0 ? -m : m;
    double c;
    if (d < 3) {
      // component d of q in the local frame
      c = (n <= p) ? P.R[0 * 3 + d] * qh[k] + P.R[1 * 3 + d] * qh[nc + k] + P.R[2 * 3 + d] * qh[2 * nc + k] : 0.0;
    } else {
      const int e = d - 3;   // 0..8: y_i q_l, 9: q . nu
      double acc = 0.0;
      for (int j = 0; j < n_q; ++j) acc = fma(Hm[(e * n_q + j) * mw1 + m + p1], qptab[(size_t)j * nm1 + nm_index(n, am)], acc);
      c = (m ? 1.4142135623730951 : 1.0) * acc;
    }
    const double ext = (d == 12) ? extS1[(size_t)i * nm1 + nm_index(n, am)] : extD1[(size_t)i * nm1 + nm_index(n, am)];
    out[idx] = ext * normc1[k] * c;
  }
}

struct alignas(32) sd4 {
  double x, y, z, w;
};

// FP64 stresslet quadrature: one target per thread.
__global__ void __launch_bounds__(kFarTile) stresslet_far_fp64_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                                      const double* __restrict__ src64,
                                                                      const double* __restrict__ nrm,
                                                                      const double* __restrict__ xyz,
                                                                      const PartGeom* __restrict__ parts,
                                                                      const int32_t* __restrict__ skip_ptr,
                                                                      const int32_t* __restrict__ skip_idx,
                                                                      int64_t N, double* __restrict__ u_out) {
  __shared__ sd4 sh[kFarTile * 3];
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
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
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
      const int64_t j = tile.y + threadIdx.x;
      const sd4* s = reinterpret_cast<const sd4*>(src64 + j * 8);
      const sd4 s1 = s[1];
      sh[threadIdx.x * 3 + 0] = s[0];
      sh[threadIdx.x * 3 + 1] = sd4{s1.x, s1.y, nrm[j * 3 + 0], nrm[j * 3 + 1]};
      sh[threadIdx.x * 3 + 2] = sd4{nrm[j * 3 + 2], 0.0, 0.0, 0.0};
    }
    __syncthreads();
    if (!skip) {
      for (int jj = 0; jj < tile.z; ++jj) {
        const sd4 a = sh[jj * 3], b = sh[jj * 3 + 1], c = sh[jj * 3 + 2];
        const double dx = X - a.x, dy = Y - a.y, dz = Z - a.z;
        const double ri = rsqrt(dx * dx + dy * dy + dz * dz);
        const double ri2 = ri * ri;
        const double rq = dx * a.w + dy * b.x + dz * b.y;
        const double rn = dx * b.z + dy * b.w + dz * c.x;
        const double s = rq * rn * (ri2 * ri2 * ri);
        a0 = fma(s, dx, a0);
        a1 = fma(s, dy, a1);
        a2 = fma(s, dz, a2);
      }
    }
    __syncthreads();
  }
  if (valid) {
    atomicAdd(u_out + t * 3 + 0, a0 * k3Over4Pi);
    atomicAdd(u_out + t * 3 + 1, a1 * k3Over4Pi);
    atomicAdd(u_out + t * 3 + 2, a2 * k3Over4Pi);
  }
}

// Mixed stresslet quadrature: FP32 pair sums, TT targets per thread, hi/lo
// target offsets per source particle, per-tile TwoSum folding.  PK computes
// two targets per f32x2 instruction, with every source value duplicated into
// a pair in shared memory: -y (3), q (3), nu (3).
template <int TT, bool PK>
__global__ void __launch_bounds__(kFarTile) stresslet_far_mixed_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                                       const float4* __restrict__ src32,
                                                                       const float4* __restrict__ nrm32,
                                                                       const float4* __restrict__ tgt32,
                                                                       const float4* __restrict__ cen32,
                                                                       const int32_t* __restrict__ skip_ptr,
                                                                       const int32_t* __restrict__ skip_idx,
                                                                       int64_t N, double* __restrict__ u_out) {
  __shared__ float4 sh[(PK ? 5 : 3) * kFarTile];
  __shared__ float acc[6 * TT * kFarTile];   // per target and component: hi, lo
  __shared__ int cursor[2 * TT * kFarTile];
  const int tid = threadIdx.x;
  const int per = (n_tiles + gridDim.y - 1) / gridDim.y;
  const int t_lo = blockIdx.y * per, t_hi = min(n_tiles, t_lo + per);
  const int64_t t0 = (int64_t)blockIdx.x * TT * kFarTile + tid;
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    const int64_t t = t0 + (int64_t)q * kFarTile;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[(6 * q + k) * kFarTile + tid] = 0.f;
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
      const int64_t j = tile.y + tid;
      const float4 a = src32[j * 2 + 0], b = src32[j * 2 + 1], c = nrm32[j];
      if (PK) {
        sh[tid * 5 + 0] = make_float4(-a.x, -a.x, -a.y, -a.y);
        sh[tid * 5 + 1] = make_float4(-a.z, -a.z, a.w, a.w);
        sh[tid * 5 + 2] = make_float4(b.x, b.x, b.y, b.y);
        sh[tid * 5 + 3] = make_float4(c.x, c.x, c.y, c.y);
        sh[tid * 5 + 4] = make_float4(c.z, c.z, 0.f, 0.f);
      } else {
        sh[tid * 3 + 0] = a;
        sh[tid * 3 + 1] = b;
        sh[tid * 3 + 2] = c;
      }
    }
    __syncthreads();
    if (mine) {
      float p0[TT], p1[TT], p2[TT];
#pragma unroll
      for (int q = 0; q < TT; ++q) p0[q] = p1[q] = p2[q] = 0.f;
      if constexpr (PK) {
        constexpr int TP = TT / 2 > 0 ? TT / 2 : 1;
        float2 Xp[TP], Yp[TP], Zp[TP], a0[TP], a1[TP], a2[TP];
#pragma unroll
        for (int k = 0; k < TP; ++k) {
          Xp[k] = make_float2(X[2 * k], X[2 * k + 1]);
          Yp[k] = make_float2(Y[2 * k], Y[2 * k + 1]);
          Zp[k] = make_float2(Z[2 * k], Z[2 * k + 1]);
          a0[k] = a1[k] = a2[k] = make_float2(0.f, 0.f);
        }
#pragma unroll 2
        for (int jj = 0; jj < tile.z; ++jj) {
          const float4 A = sh[jj * 5 + 0], B = sh[jj * 5 + 1], C = sh[jj * 5 + 2], D = sh[jj * 5 + 3],
                       E = sh[jj * 5 + 4];
          const float2 myx = make_float2(A.x, A.y), myy = make_float2(A.z, A.w), myz = make_float2(B.x, B.y);
          const float2 qx = make_float2(B.z, B.w), qy = make_float2(C.x, C.y), qz = make_float2(C.z, C.w);
          const float2 nx = make_float2(D.x, D.y), ny = make_float2(D.z, D.w), nz = make_float2(E.x, E.y);
#pragma unroll
          for (int k = 0; k < TP; ++k) {
            const float2 dx = __fadd2_rn(Xp[k], myx), dy = __fadd2_rn(Yp[k], myy), dz = __fadd2_rn(Zp[k], myz);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 ri = make_float2(rsqrt_f32(r2.x), rsqrt_f32(r2.y));
            const float2 ri2 = __fmul2_rn(ri, ri);
            const float2 rq = __ffma2_rn(dz, qz, __ffma2_rn(dy, qy, __fmul2_rn(dx, qx)));
            const float2 rn = __ffma2_rn(dz, nz, __ffma2_rn(dy, ny, __fmul2_rn(dx, nx)));
            const float2 sc = __fmul2_rn(__fmul2_rn(rq, rn), __fmul2_rn(__fmul2_rn(ri2, ri2), ri));
            a0[k] = __ffma2_rn(sc, dx, a0[k]);
            a1[k] = __ffma2_rn(sc, dy, a1[k]);
            a2[k] = __ffma2_rn(sc, dz, a2[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < TP; ++k) {
          p0[2 * k] = a0[k].x; p0[2 * k + 1] = a0[k].y;
          p1[2 * k] = a1[k].x; p1[2 * k + 1] = a1[k].y;
          p2[2 * k] = a2[k].x; p2[2 * k + 1] = a2[k].y;
        }
      } else {
#pragma unroll 2
      for (int jj = 0; jj < tile.z; ++jj) {
        const float4 a = sh[jj * 3], b = sh[jj * 3 + 1], c = sh[jj * 3 + 2];
#pragma unroll
        for (int q = 0; q < TT; ++q) {
          const float dx = X[q] - a.x, dy = Y[q] - a.y, dz = Z[q] - a.z;
          const float ri = rsqrt_f32(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
          const float ri2 = ri * ri;
          const float rq = fmaf(dz, b.y, fmaf(dy, b.x, dx * a.w));
          const float rn = fmaf(dz, c.z, fmaf(dy, c.y, dx * c.x));
          const float s = rq * rn * (ri2 * ri2 * ri);
          p0[q] = fmaf(s, dx, p0[q]);
          p1[q] = fmaf(s, dy, p1[q]);
          p2[q] = fmaf(s, dz, p2[q]);
        }
      }
      }
#pragma unroll
      for (int q = 0; q < TT; ++q) {
        if (!((skipmask >> q) & 1u)) {
          const float pv[3] = {p0[q], p1[q], p2[q]};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            float sum, err;
            two_sum_f32(acc[(6 * q + 2 * k) * kFarTile + tid], pv[k], sum, err);
            acc[(6 * q + 2 * k) * kFarTile + tid] = sum;
            acc[(6 * q + 2 * k + 1) * kFarTile + tid] += err;
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    const int64_t t = t0 + (int64_t)q * kFarTile;
    if (t < N)
      for (int k = 0; k < 3; ++k)
        atomicAdd(u_out + t * 3 + k,
                  ((double)acc[(6 * q + 2 * k) * kFarTile + tid] + (double)acc[(6 * q + 2 * k + 1) * kFarTile + tid]) *
                      k3Over4Pi);
  }
}

template <int TT, bool PK>
void launch_stresslet_far_tt(const DevGeom& tg, const DevGeom& src, const GeomHost& h, int64_t NT, double* u,
                             cudaStream_t st) {
  const int nt = (int)h.tiles.size();
  const int64_t tb = (NT + (int64_t)kFarTile * TT - 1) / ((int64_t)kFarTile * TT);
  const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, PK ? h.st_far_splits : 0));
  stresslet_far_mixed_kernel<TT, PK><<<grid, kFarTile, 0, st>>>(src.tiles, nt, src.st_src32, src.nrm32, tg.tgt32,
                                                                src.cen32, tg.skip_ptr, tg.skip_idx, NT, u);
}

// tg: the targets (positions, hi/lo parts, skip lists; a point set's view or
// the geometry itself); src: the geometry, whose source-side arrays (tiles,
// sources, source normals, centres) are always taken from it.
void launch_stresslet_far(const DevGeom& tg, const DevGeom& src, const GeomHost& h, int64_t NT, double* u,
                          cudaStream_t st) {
  if (NT <= 0) return;
  const int nt = (int)h.tiles.size();
  if (h.precision == SBIO_FP64) {
    const int64_t tb = (NT + kFarTile - 1) / kFarTile;
    const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, 0));
    stresslet_far_fp64_kernel<<<grid, kFarTile, 0, st>>>(src.tiles, nt, src.st_src64, src.nrm, tg.xyz, src.parts,
                                                         tg.skip_ptr, tg.skip_idx, NT, u);
  } else if (h.st_far_tt < 0) {
    // the geometry's tuned Stokes far shape, when packed (the Stokeslet and
    // stresslet pair costs are alike): |tt| targets per thread, tuned splits
    switch (h.st_far_tt) {
      case -2: launch_stresslet_far_tt<2, true>(tg, src, h, NT, u, st); break;
      case -4: launch_stresslet_far_tt<4, true>(tg, src, h, NT, u, st); break;
      default: launch_stresslet_far_tt<8, true>(tg, src, h, NT, u, st); break;
    }
  } else {
    launch_stresslet_far_tt<4, false>(tg, src, h, NT, u, st);
  }
  count_launch();
}

// Own-node (exterior-limit) part of the double layer, separable: for the
// thirteen expansions in groups [d0, d1), Legendre sums at the GL rows of
// q'(u0) P, q(u0) sqrt(1-v^2) dP/dv and q(u0) m P / sqrt(1-v^2) (the
// single-layer self tables), then Fourier sums at every node give the local
// gradient g_d in the source's frame.  The density index of expansions 0..11
// is in the local frame (q_l = sum_j R_jl q_j), so expansion d adds
//   d = l < 3 (q_l):          -X_k g_d[l] to every component k,
//   d = 3 + 3i + l (y_i q_l): g_d[l] to component i,
//   d = 12 (q . nu):          -(R g_d)_k to component k,
// with X the node relative to the centre.  Atomic adds: the near kernels may
// be adding to the same outputs on another stream.
__global__ void __launch_bounds__(256) sdl_self_kernel(int p, int n_v, int n_phi, int n_groups,
                                                       const PartGeom* __restrict__ parts,
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
  // expansions [d0, d1) of group blockIdx.y (the groups split the thirteen evenly)
  const int d0 = (int)(blockIdx.y * 13 / n_groups), d1 = (int)((blockIdx.y + 1) * 13 / n_groups);
  const int p1 = p + 1, nc1 = (p1 + 1) * (p1 + 1), nm1 = nm_count(p1), mw1 = 2 * p1 + 1;
  const int G = n_v * n_phi, nd = d1 - d0;
  const PartGeom P = parts[i];
  const double* cf = coef + (size_t)i * 13 * nc1;
  const double* q0 = qu0 + (size_t)i * nm1;
  const double* dq0 = dqu0 + (size_t)i * nm1;
  // sm[((dd * 3 + qty) * n_v + j) * mw1 + ms]: qty 0 d/du, 1 sv d/dv, 2 d/dphi / sv
  for (int idx = threadIdx.x; idx < nd * 3 * n_v * mw1; idx += blockDim.x) {
    const int row = idx / mw1, ms = idx - row * mw1, m = ms - p1, am = m < 0 ? -m : m;
    const int dq = row / n_v, j = row - dq * n_v, dd = dq / 3, qty = dq - 3 * dd;
    const double* tab = (qty == 1) ? fV : (qty == 2 ? fF : fP);
    const double* rad = (qty == 0) ? dq0 : q0;
    const double* c = cf + (size_t)(d0 + dd) * nc1;
    double acc = 0.0;
    for (int n = am; n <= p1; ++n)
      acc = fma(c[n * n + n + m] * rad[nm_index(n, am)], tab[(size_t)j * nm1 + nm_index(n, am)], acc);
    sm[idx] = acc;
  }
  __syncthreads();
  const double sgn = P.sgn, u = P.u0;
  const double su = P.A / P.a;   // sqrt(u0^2 + sgn)
  const double ia = 1.0 / P.a;
  const double* R = P.R;
  for (int l = threadIdx.x; l < G; l += blockDim.x) {
    const int j = l / n_phi, k = l - j * n_phi;
    const double* tr = trig1 + (size_t)k * (p1 + 1) * 2;
    const double v = gl_v[j], sv = sqrt((1.0 - v) * (1.0 + v));
    const double c1 = tr[2], s1 = tr[3];
    const double iW = rsqrt(u * u + sgn * v * v);
    const double eu0 = u * sv * c1 * iW, eu1 = u * sv * s1 * iW, eu2 = v * su * iW;
    const double ev0 = -su * v * c1 * iW, ev1 = -su * v * s1 * iW, ev2 = u * sv * iW;
    const int64_t t = (int64_t)i * G + l;
    const double X[3] = {xyz[t * 3 + 0] - P.c[0], xyz[t * 3 + 1] - P.c[1], xyz[t * 3 + 2] - P.c[2]};
    double out[3] = {0.0, 0.0, 0.0};
    for (int dd = 0; dd < nd; ++dd) {
      double F[3];
      for (int qty = 0; qty < 3; ++qty) {
        const double* L = sm + ((size_t)(dd * 3 + qty) * n_v + j) * mw1 + p1;
        double acc;
        if (qty == 2) {   // d/dphi: cos -> -m sin, sin -> m cos (m inside the table)
          acc = 0.0;
          for (int m = 1; m <= p1; ++m) acc = fma(-L[m], tr[2 * m + 1], fma(L[-m], tr[2 * m], acc));
        } else {
          acc = L[0];
          for (int m = 1; m <= p1; ++m) acc = fma(L[m], tr[2 * m], fma(L[-m], tr[2 * m + 1], acc));
        }
        F[qty] = acc;
      }
      const double gu = F[0] * su * ia * iW, gv = F[1] * ia * iW, gp = F[2] * ia / su;
      const double gl[3] = {gu * eu0 + gv * ev0 - gp * s1, gu * eu1 + gv * ev1 + gp * c1, gu * eu2 + gv * ev2};
      const int d = d0 + dd;
      if (d < 3) {
        // local divergence of (D[q_l]): component d of expansion d
        for (int r = 0; r < 3; ++r) out[r] -= X[r] * gl[d];
      } else if (d < 12) {
        const int ii = (d - 3) / 3, ll = (d - 3) - 3 * ii;
        out[ii] += gl[ll];
      } else {
        for (int r = 0; r < 3; ++r) out[r] -= R[r * 3 + 0] * gl[0] + R[r * 3 + 1] * gl[1] + R[r * 3 + 2] * gl[2];
      }
    }
    for (int r = 0; r < 3; ++r) atomicAdd(u_out + t * 3 + r, out[r]);
  }
}

int sdl_self(sbio_geom* g, double* u_out, cudaStream_t st) {
  const GeomHost& h = g->h;
  const DevGeom& d = g->d;
  const int p1 = h.p + 1, mw1 = 2 * p1 + 1;
  // one launch over (particle, group of expansions): four groups of 3-4
  // expansions give 4 M CTAs, each holding its group's Legendre sums
  constexpr int kGroups = 4;
  const int nd_max = (13 + kGroups - 1) / kGroups;
  const size_t smem = (size_t)nd_max * 3 * h.n_v * mw1 * sizeof(double);
  if (smem > 227 * 1024) return set_error(SBIO_ENOTSUP, "Stokes double layer self: p = %d too large", h.p);
  if (smem > 48 * 1024)
    SBIO_CUDA_TRY(cudaFuncSetAttribute(sdl_self_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sdl_self_kernel<<<dim3(h.M, kGroups), 256, smem, st>>>(h.p, h.n_v, h.n_phi, kGroups, d.parts, d.xyz, d.sdl_coef,
                                                         d.st_qu0, d.st_dqu0, d.st_fP, d.st_fV, d.st_fF, d.st_trig1,
                                                         d.st_glv, u_out);
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}

// u_init (may be null) is set to init_factor q at every node: -1/2 for the
// principal value, 0 for the exterior limit, -1 for the interior limit (the
// near, own-node and far parts add the exterior-limit field).
int sdl_prep(sbio_geom* g, const double* qhat, double* u_init, cudaStream_t st, double init_factor = -0.5) {
  const GeomHost& h = g->h;
  const DevGeom& d = g->d;
  const int p = h.p, p1 = p + 1, nc = (p + 1) * (p + 1), mw = 2 * p + 1, mw1 = 2 * p1 + 1;
  const int nrow = h.n_q > h.n_v ? h.n_q : h.n_v;
  const size_t smem =
      (size_t)(3 * nc + 3 * nrow * mw + 10 * h.n_q * h.n_f + 10 * h.n_q * mw1) * sizeof(double);
  if (smem > 227 * 1024) return set_error(SBIO_ENOTSUP, "Stokes double layer: p = %d exceeds shared memory", p);
  if (smem > 48 * 1024)
    SBIO_CUDA_TRY(cudaFuncSetAttribute(sdl_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sdl_prep_kernel<<<h.M, 256, smem, st>>>(p, h.n_v, h.n_phi, h.n_q, h.n_f, d.parts, d.xyz, d.w, d.ptab, d.trig,
                                          d.st_qv, d.st_qw, d.st_qptab, d.st_qtrig, d.st_ext, d.sdl_ext, d.st_normc,
                                          qhat, d.sdl_coef, d.st_src64, d.st_src32, u_init, init_factor);
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}

// Near CTAs per SM for the double layer's near pairs beside the far field
// (0 = uncapped): at least 4, since its near pairs carry a larger share of
// the work than the single layer's, on which the Stokes cap is tuned (with a
// cap of 2 the stokesdl100 apply ran 10 % slower than with 4 or more).
int sdl_near_cap(const GeomHost& h) {
  return h.st_near_ctas_per_sm > 0 ? std::max(4, h.st_near_ctas_per_sm) : 0;
}

stokes_dl_near_launcher sdl_near_for(int p) {
  stokes_dl_near_launcher (*const tab[])(int) = {stokes_dl_near_lookup_a, stokes_dl_near_lookup_b,
                                                  stokes_dl_near_lookup_c, stokes_dl_near_lookup_d,
                                                  stokes_dl_near_lookup_e, stokes_dl_near_lookup_f,
                                                  stokes_dl_near_lookup_g, stokes_dl_near_lookup_h,
                                                  stokes_dl_near_lookup_i, stokes_dl_near_lookup_j};
  for (auto f : tab)
    if (stokes_dl_near_launcher nl = f(p)) return nl;
  return nullptr;
}

}  // namespace
}  // namespace sbio

using namespace sbio;

extern "C" {

int sbio_apply_stokes_dl_limit(sbio_geom* g, const double* q_hat, double* u_out, int32_t side, void* stream) {
  clear_error();
  if (!g || !q_hat || !u_out) return set_error(SBIO_EINVAL, "null argument");
  if (side < -1 || side > 1) return set_error(SBIO_EINVAL, "side %d: -1 (interior), 0 or +1 (exterior)", side);
  const GeomHost& h = g->h;
  if (h.p > 20) return set_error(SBIO_ENOTSUP, "Stokes double layer is built for p <= 20 (p = %d)", h.p);
  stokes_dl_near_launcher nl = sdl_near_for(h.p);
  if (!nl) return set_error(SBIO_ENOTSUP, "no Stokes double-layer kernel for p = %d", h.p);
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  phase_mark(g, 0, st);
  // the rest of the apply adds the exterior limit: start from -q/2 (principal
  // value), 0 (exterior) or -q (interior) at every node
  int rc = sdl_prep(g, q_hat, u_out, st, -0.5 * (1 - side));
  if (rc) return rc;
  const DevGeom& d = g->d;
  const bool has_pairs = !h.pair_t.empty();
  const bool fork = g->overlap && !g->timing && g->near_stream && has_pairs;
  SideFork sf;
  if (fork) {
    // near pairs on the forked high-priority stream, beside the own nodes
    // (exterior limit at u = u0, separable self kernel) and the far field
    DevGeom v = d;
    v.near_grid_cap = sdl_near_cap(h) * sm_count();
    SBIO_CUDA_TRY(sf.fork(g, st));
    nl(v, d.pair_t, d.pair_s, h.n_pairs_prolate, (int64_t)h.pair_t.size(), u_out, g->near_stream);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  if ((rc = sdl_self(g, u_out, st))) return rc;
  // in order (no overlap, or phase timing): prep + self, near pairs, far field
  phase_mark(g, 1, st);
  if (!fork && has_pairs) {
    nl(d, d.pair_t, d.pair_s, h.n_pairs_prolate, (int64_t)h.pair_t.size(), u_out, st);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  phase_mark(g, 2, st);
  launch_stresslet_far(d, d, h, h.N, u_out, st);
  SBIO_CUDA_TRY(cudaGetLastError());
  SBIO_CUDA_TRY(sf.join());
  phase_mark(g, 3, st);
  return SBIO_OK;
}

int sbio_apply_stokes_dl(sbio_geom* g, const double* q_hat, double* u_out, void* stream) {
  return sbio_apply_stokes_dl_limit(g, q_hat, u_out, 0, stream);
}

int sbio_eval_targets_stokes_dl(sbio_targets* ts, const double* q_hat, double* u_out, void* stream) {
  clear_error();
  if (!ts || !q_hat || !u_out) return set_error(SBIO_EINVAL, "null argument");
  sbio_geom* g = nullptr;
  const DevGeom* view = nullptr;
  int64_t T = 0, n_pro = 0, n_pairs = 0;
  int rc = targets_view(ts, &g, &view, &T, &n_pro, &n_pairs);
  if (rc) return rc;
  const GeomHost& h = g->h;
  if (h.p > 20) return set_error(SBIO_ENOTSUP, "Stokes double layer is built for p <= 20 (p = %d)", h.p);
  stokes_dl_near_launcher nl = sdl_near_for(h.p);
  if (!nl) return set_error(SBIO_ENOTSUP, "no Stokes double-layer kernel for p = %d", h.p);
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (T == 0) return SBIO_OK;
  SBIO_CUDA_TRY(cudaMemsetAsync(u_out, 0, T * 3 * sizeof(double), st));
  if ((rc = sdl_prep(g, q_hat, nullptr, st))) return rc;
  // near pairs on the geometry's high-priority stream beside the far field
  // (as in the on-surface apply), unless phases are timed one by one
  const bool fork = g->overlap && !g->timing && g->near_stream && n_pairs > 0;
  SideFork sf;
  if (fork) {
    DevGeom v = *view;   // a copy: the near grid cap is per launch
    v.near_grid_cap = sdl_near_cap(h) * sm_count();
    SBIO_CUDA_TRY(sf.fork(g, st));
    nl(v, v.pair_t, v.pair_s, n_pro, n_pairs, u_out, g->near_stream);
    SBIO_CUDA_TRY(cudaGetLastError());
  } else if (n_pairs > 0) {
    nl(*view, view->pair_t, view->pair_s, n_pro, n_pairs, u_out, st);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  launch_stresslet_far(*view, g->d, h, T, u_out, st);
  SBIO_CUDA_TRY(cudaGetLastError());
  SBIO_CUDA_TRY(sf.join());
  return SBIO_OK;
}

}  // extern "C"
