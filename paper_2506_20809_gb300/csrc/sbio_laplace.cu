// Laplace single / double layer apply at all surface nodes (Algorithm 1 and
// its single-layer variant, Sec. 4.2), as three kernels on one stream:
//   synth  : per particle, node values of the densities (inverse surface
//            transform), the far-field source strengths q = w sigma and
//            d = w mu nu, the folded near-field coefficients, and the self
//            term (diagonal multipliers of Theorems 1-2 followed by the
//            inverse transform), which initialises the outputs;
//   near   : one thread per (target, near source particle) pair, exterior
//            expansion (sbio_near.cuh), FP64, atomically added;
//   far    : tiled all-pairs smooth quadrature over the nodes of far
//            particles (Sec. 4.1 "Far-field"), FP64 or FP32 with two-sum
//            compensated accumulation, atomically added.
#include <algorithm>
#include <vector>

#include "sbio_internal.cuh"
#include "sbio_near.cuh"

namespace sbio {

constexpr double kInv4Pi = 0.07957747154594767;   // 1/(4 pi)

struct alignas(32) dbl4 {
  double x, y, z, w;
};

// ---------------------------------------------------------------------------
// synth: densities at the nodes, far-field sources, near coefficients, self
// ---------------------------------------------------------------------------
// One CTA, one particle i.  `sm` holds 2 (p+1)^2 + 4 (p+1)(2p+1) doubles.
// write_self: 0 = no self output (zeros written where outputs are given),
// 1 = the on-surface S and D, 2 = normal derivatives S' and D' (with the
// derivative multiplier table passed as `mult`).  side: 0 = principal value;
// +1 / -1 = exterior / interior limit, i.e. D +- mu/2 (mode 1) and
// S' -+ sigma/2 (mode 2) from the density values at the node.
__device__ __forceinline__ void synth_particle(int i, double* sm, int p, int n_v, int n_phi,
                                               const PartGeom* __restrict__ parts, const double* __restrict__ xyz,
                                               const double* __restrict__ nrm, const double* __restrict__ w,
                                               const double* __restrict__ ptab, const double* __restrict__ trig,
                                               const double* __restrict__ sqrtw, const double* __restrict__ mult,
                                               const double* __restrict__ normc, const double* __restrict__ sigma,
                                               const double* __restrict__ mu, int write_self, int side,
                                               double* __restrict__ S_out, double* __restrict__ D_out,
                                               double* __restrict__ src64, float4* __restrict__ src32,
                                               double* __restrict__ alpha, double* __restrict__ beta,
                                               float* __restrict__ alpha32, float* __restrict__ beta32) {
  const int nc = (p + 1) * (p + 1), nm = nm_count(p), nmw = 2 * p + 1;
  const int G = n_v * n_phi;
  double* c_sig = sm;                 // nc
  double* c_mu = c_sig + nc;          // nc
  double* F = c_mu + nc;              // 4 x n_v x nmw: sigma, mu, S self, D self
  const bool hs = sigma != nullptr, hm = mu != nullptr;
  const double* mlt = mult + (size_t)i * 4 * nm;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const int n = (int)sqrt((double)k);
    const int m = k - n * n - n;
    const int am = m < 0 ? -m : m;
    const double cs = hs ? sigma[(size_t)i * nc + k] : 0.0;
    const double cmu = hm ? mu[(size_t)i * nc + k] : 0.0;
    c_sig[k] = cs;
    c_mu[k] = cmu;
    alpha[(size_t)i * nc + k] = mlt[0 * nm + nm_index(n, am)] * normc[k] * cs;
    beta[(size_t)i * nc + k] = mlt[1 * nm + nm_index(n, am)] * normc[k] * cmu;
    // the mixed near form's coefficients: alpha = extS N sigma, beta = extS N (mu extD / extS)
    if (alpha32) {
      alpha32[(size_t)i * nc + k] = (float)cs;
      beta32[(size_t)i * nc + k] = (float)(cmu * (mlt[1 * nm + nm_index(n, am)] / mlt[0 * nm + nm_index(n, am)]));
    }
  }
  __syncthreads();
  // stage 1: Legendre sums  F[j][m] = sum_n c_nm sqrt2^[m!=0] N P(v_j)
  for (int idx = threadIdx.x; idx < n_v * nmw; idx += blockDim.x) {
    const int j = idx / nmw, ms = idx - j * nmw, m = ms - p, am = m < 0 ? -m : m;
    const double s2 = m ? 1.4142135623730951 : 1.0;
    double fs = 0.0, fm = 0.0, fS = 0.0, fD = 0.0;
    for (int n = am; n <= p; ++n) {
      const int k = n * n + n + m;
      const double pt = s2 * ptab[(size_t)j * nm + nm_index(n, am)];
      const double a = c_sig[k] * pt, b = c_mu[k] * pt;
      fs += a;
      fm += b;
      fS = fma(mlt[2 * nm + nm_index(n, am)], a, fS);
      fD = fma(mlt[3 * nm + nm_index(n, am)], b, fD);
    }
    F[(0 * n_v + j) * nmw + ms] = fs;
    F[(1 * n_v + j) * nmw + ms] = fm;
    F[(2 * n_v + j) * nmw + ms] = fS;
    F[(3 * n_v + j) * nmw + ms] = fD;
  }
  __syncthreads();
  // stage 2: Fourier sums at every node of the particle
  const PartGeom P = parts[i];
  for (int l = threadIdx.x; l < G; l += blockDim.x) {
    const int j = l / n_phi, k = l - j * n_phi;
    const double* tr = trig + (size_t)k * (p + 1) * 2;
    const double* f0 = F + (0 * n_v + j) * nmw + p;
    const double* f1 = F + (1 * n_v + j) * nmw + p;
    const double* f2 = F + (2 * n_v + j) * nmw + p;
    const double* f3 = F + (3 * n_v + j) * nmw + p;
    double vs = f0[0], vm = f1[0], vS = f2[0], vD = f3[0];
    for (int m = 1; m <= p; ++m) {
      const double cth = tr[2 * m], sth = tr[2 * m + 1];
      vs = fma(f0[m], cth, fma(f0[-m], sth, vs));
      vm = fma(f1[m], cth, fma(f1[-m], sth, vm));
      vS = fma(f2[m], cth, fma(f2[-m], sth, vS));
      vD = fma(f3[m], cth, fma(f3[-m], sth, vD));
    }
    const int64_t t = (int64_t)i * G + l;
    const double sig_val = vs / sqrtw[(size_t)i * n_v + j];   // modified basis (Sec. 3.2)
    const double q = w[t] * sig_val;
    const double wm = w[t] * vm;
    const double d0 = wm * nrm[t * 3 + 0], d1 = wm * nrm[t * 3 + 1], d2 = wm * nrm[t * 3 + 2];
    const double y0 = xyz[t * 3 + 0] - P.c[0], y1 = xyz[t * 3 + 1] - P.c[1], y2 = xyz[t * 3 + 2] - P.c[2];
    double* s = src64 + t * 8;
    s[0] = y0; s[1] = y1; s[2] = y2; s[3] = q;
    s[4] = d0; s[5] = d1; s[6] = d2; s[7] = 0.0;
    src32[t * 2 + 0] = make_float4((float)y0, (float)y1, (float)y2, (float)q);
    src32[t * 2 + 1] = make_float4((float)d0, (float)d1, (float)d2, 0.f);
    // write_self == 2: the self sums are normal derivatives (multipliers of
    // Theorem 3 and its D' counterpart, in d/du), scaled by 1/h_u =
    // sqrt(u0^2 + sgn) / (a sqrt(u0^2 + sgn v^2)) on the surface (Table 2)
    const double sc = (write_self == 2) ? (P.A / P.a) / (P.a * sqrtw[(size_t)i * n_v + j]) : 1.0;
    // one-sided limits: the jump of D is mu, that of S' is -sigma
    const double jS = (write_self == 2) ? -0.5 * side * sig_val : 0.0;
    const double jD = (write_self == 1) ? 0.5 * side * vm : 0.0;
    if (S_out) S_out[t] = write_self ? fma(vS, sc, jS) : 0.0;
    if (D_out) D_out[t] = write_self ? fma(vD, sc, jD) : 0.0;
  }
}

__global__ void __launch_bounds__(256) synth_kernel(int p, int n_v, int n_phi, const PartGeom* __restrict__ parts,
                                                    const double* __restrict__ xyz, const double* __restrict__ nrm,
                                                    const double* __restrict__ w, const double* __restrict__ ptab,
                                                    const double* __restrict__ trig,
                                                    const double* __restrict__ sqrtw,
                                                    const double* __restrict__ mult,
                                                    const double* __restrict__ normc,
                                                    const double* __restrict__ sigma, const double* __restrict__ mu,
                                                    int write_self, int side, double* __restrict__ S_out,
                                                    double* __restrict__ D_out, double* __restrict__ src64,
                                                    float4* __restrict__ src32, double* __restrict__ alpha,
                                                    double* __restrict__ beta, float* __restrict__ alpha32,
                                                    float* __restrict__ beta32) {
  extern __shared__ double sm[];
  synth_particle(blockIdx.x, sm, p, n_v, n_phi, parts, xyz, nrm, w, ptab, trig, sqrtw, mult, normc, sigma, mu,
                 write_self, side, S_out, D_out, src64, src32, alpha, beta, alpha32, beta32);
}

// ---------------------------------------------------------------------------
// far: tiled all-pairs quadrature over far source nodes
// ---------------------------------------------------------------------------

// FP64 form: one target per thread, kFarTile sources per smem tile.
template <bool DO_S, bool DO_D>
__global__ void __launch_bounds__(kFarTile) far_fp64_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                            const double* __restrict__ src64,
                                                            const double* __restrict__ xyz,
                                                            const PartGeom* __restrict__ parts,
                                                            const int32_t* __restrict__ skip_ptr,
                                                            const int32_t* __restrict__ skip_idx, int64_t N,
                                                            double* __restrict__ S_out, double* __restrict__ D_out) {
  __shared__ dbl4 sh[kFarTile * 2];
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
  double accS = 0.0, accD = 0.0;
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
      const dbl4* s = reinterpret_cast<const dbl4*>(src64 + (int64_t)(tile.y + threadIdx.x) * 8);
      sh[threadIdx.x * 2 + 0] = s[0];
      sh[threadIdx.x * 2 + 1] = s[1];
    }
    __syncthreads();
    if (!skip) {
      for (int j = 0; j < tile.z; ++j) {
        const dbl4 a = sh[j * 2], b = sh[j * 2 + 1];
        const double dx = X - a.x, dy = Y - a.y, dz = Z - a.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double ri = rsqrt(r2);
        if (DO_S) accS = fma(a.w, ri, accS);
        if (DO_D) accD = fma((b.x * dx + b.y * dy + b.z * dz) * ri, ri * ri, accD);
      }
    }
    __syncthreads();
  }
  if (valid) {
    if (DO_S) atomicAdd(S_out + t, accS * kInv4Pi);
    if (DO_D) atomicAdd(D_out + t, accD * kInv4Pi);
  }
}

// Mixed form: FP32 pair sums, TT targets per thread.  The target position is
// taken relative to each source particle's centre through hi/lo FP32 parts
// (X = (x_hi - c_hi) + (x_lo - c_lo)), the sources are stored relative to
// their own centre, so the FP32 difference X - y_rel carries an error
// relative to |x - y| rather than to the box size.  Each tile's FP32 partial
// sum is folded into an (hi, lo) pair by TwoSum.
// One CTA of NT threads: targets [t_first, min(t_end, t_first + NT * TT)) (TT per
// thread, target t_first + tid + q NT) against source tiles [t_lo, t_hi) of up
// to kFarTile sources.  Only the target positions
// relative to the current source particle and the running tile partials live
// in registers; the two-sum accumulators and the skip-list cursors live in
// shared memory and are touched once per tile.
template <int TT, bool DO_S, bool DO_D, bool PK, int NT = kFarTile>
__device__ __forceinline__ void far_mixed_block(int64_t t_first, int64_t t_end, int t_lo, int t_hi,
                                                const int4* __restrict__ tiles, const float4* __restrict__ src32,
                                                const float4* __restrict__ tgt32, const float4* __restrict__ cen32,
                                                const int32_t* __restrict__ skip_ptr,
                                                const int32_t* __restrict__ skip_idx,
                                                double* __restrict__ S_out, double* __restrict__ D_out) {
  // tile of sources: scalar form (y - c, q), (d, 0).  The packed form uses
  // the expanded distance |x - y|^2 = (|x|^2 + |y|^2) - 2 x.y and
  // d.(x - y) = d.x - d.y, so that a pair costs 11 FP32 operations instead of
  // 13; per source it holds every value duplicated into an f32x2 pair:
  // (-2y.x, -2y.y), (-2y.z, |y|^2), (q, -d.y), (d.x, d.y), (d.z, 0)
  __shared__ float4 sh[(PK ? 5 : 2) * kFarTile];
  __shared__ float acc[4 * TT * NT];   // per target: S hi, S lo, D hi, D lo
  __shared__ int cursor[2 * TT * NT];  // per target: skip-list position, next skipped particle
  const int tid = threadIdx.x;
  const int64_t t0 = t_first + tid;
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    const int64_t t = t0 + (int64_t)q * NT;
    acc[(4 * q + 0) * NT + tid] = 0.f;
    acc[(4 * q + 1) * NT + tid] = 0.f;
    acc[(4 * q + 2) * NT + tid] = 0.f;
    acc[(4 * q + 3) * NT + tid] = 0.f;
    const int sp = (t < t_end) ? skip_ptr[t] : 0;
    cursor[(2 * q + 0) * NT + tid] = sp;
    cursor[(2 * q + 1) * NT + tid] = (t < t_end) ? skip_idx[sp] : INT32_MAX;
  }
  float X[TT], Y[TT], Z[TT], XX[TT];
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
        const int64_t t = t0 + (int64_t)q * NT;
        int sp = cursor[(2 * q + 0) * NT + tid];
        int nxt = cursor[(2 * q + 1) * NT + tid];
        while (nxt < cur) nxt = skip_idx[++sp];
        cursor[(2 * q + 0) * NT + tid] = sp;
        cursor[(2 * q + 1) * NT + tid] = nxt;
        if (t >= t_end || nxt == cur) skipmask |= 1u << q;
        float4 hi = make_float4(0.f, 0.f, 0.f, 0.f), lo = hi;
        if (t < t_end) {
          hi = tgt32[t * 2];
          lo = tgt32[t * 2 + 1];
        }
        X[q] = (hi.x - ch.x) + (lo.x - cl.x);
        Y[q] = (hi.y - ch.y) + (lo.y - cl.y);
        Z[q] = (hi.z - ch.z) + (lo.z - cl.z);
        if constexpr (PK) XX[q] = fmaf(Z[q], Z[q], fmaf(Y[q], Y[q], X[q] * X[q]));
      }
    }
    const bool mine = skipmask != (1u << TT) - 1u;
    if (!__syncthreads_or(mine)) continue;
    if constexpr (NT == kFarTile) {
      if (tid < tile.z) {
        const float4 a = src32[(int64_t)(tile.y + tid) * 2 + 0];
        const float4 b = src32[(int64_t)(tile.y + tid) * 2 + 1];
        if (PK) {
          const float yy = fmaf(a.z, a.z, fmaf(a.y, a.y, a.x * a.x));
          const float dy = fmaf(b.z, a.z, fmaf(b.y, a.y, b.x * a.x));
          sh[tid * 5 + 0] = make_float4(-2.f * a.x, -2.f * a.x, -2.f * a.y, -2.f * a.y);
          sh[tid * 5 + 1] = make_float4(-2.f * a.z, -2.f * a.z, yy, yy);
          sh[tid * 5 + 2] = make_float4(a.w, a.w, -dy, -dy);
          sh[tid * 5 + 3] = make_float4(b.x, b.x, b.y, b.y);
          sh[tid * 5 + 4] = make_float4(b.z, b.z, 0.f, 0.f);
        } else {
          sh[tid * 2 + 0] = a;
          sh[tid * 2 + 1] = b;
        }
      }
    } else {
      for (int sidx = tid; sidx < tile.z; sidx += NT) {
        const float4 a = src32[(int64_t)(tile.y + sidx) * 2 + 0];
        const float4 b = src32[(int64_t)(tile.y + sidx) * 2 + 1];
        if (PK) {
          const float yy = fmaf(a.z, a.z, fmaf(a.y, a.y, a.x * a.x));
          const float dy = fmaf(b.z, a.z, fmaf(b.y, a.y, b.x * a.x));
          sh[sidx * 5 + 0] = make_float4(-2.f * a.x, -2.f * a.x, -2.f * a.y, -2.f * a.y);
          sh[sidx * 5 + 1] = make_float4(-2.f * a.z, -2.f * a.z, yy, yy);
          sh[sidx * 5 + 2] = make_float4(a.w, a.w, -dy, -dy);
          sh[sidx * 5 + 3] = make_float4(b.x, b.x, b.y, b.y);
          sh[sidx * 5 + 4] = make_float4(b.z, b.z, 0.f, 0.f);
        } else {
          sh[sidx * 2 + 0] = a;
          sh[sidx * 2 + 1] = b;
        }
      }
    }
    __syncthreads();
    if (mine) {
      float pS[TT], pD[TT];
#pragma unroll
      for (int q = 0; q < TT; ++q) pS[q] = pD[q] = 0.f;
      if constexpr (PK) {
        // two targets per f32x2 operation (sm_100+ packed FP32), one MUFU rsqrt per pair
        constexpr int TP = TT / 2 > 0 ? TT / 2 : 1;
        float2 Xp[TP], Yp[TP], Zp[TP], XXp[TP], sS2[TP], sD2[TP];
#pragma unroll
        for (int k = 0; k < TT / 2; ++k) {
          Xp[k] = make_float2(X[2 * k], X[2 * k + 1]);
          Yp[k] = make_float2(Y[2 * k], Y[2 * k + 1]);
          Zp[k] = make_float2(Z[2 * k], Z[2 * k + 1]);
          XXp[k] = make_float2(XX[2 * k], XX[2 * k + 1]);
          sS2[k] = make_float2(0.f, 0.f);
          sD2[k] = make_float2(0.f, 0.f);
        }
#pragma unroll 2
        for (int j = 0; j < tile.z; ++j) {
          const float4 A = sh[j * 5 + 0], B = sh[j * 5 + 1], Cc = sh[j * 5 + 2], Dd = sh[j * 5 + 3],
                       Ee = sh[j * 5 + 4];
          const float2 mx = make_float2(A.x, A.y), my = make_float2(A.z, A.w), mz = make_float2(B.x, B.y);
          const float2 yy = make_float2(B.z, B.w), q2 = make_float2(Cc.x, Cc.y), ndy = make_float2(Cc.z, Cc.w);
          const float2 dwx = make_float2(Dd.x, Dd.y), dwy = make_float2(Dd.z, Dd.w), dwz = make_float2(Ee.x, Ee.y);
#pragma unroll
          for (int k = 0; k < TT / 2; ++k) {
            const float2 r2 =
                __ffma2_rn(Xp[k], mx, __ffma2_rn(Yp[k], my, __ffma2_rn(Zp[k], mz, __fadd2_rn(XXp[k], yy))));
            const float2 ri = make_float2(rsqrt_f32(r2.x), rsqrt_f32(r2.y));
            if (DO_S) sS2[k] = __ffma2_rn(q2, ri, sS2[k]);
            if (DO_D) {
              const float2 dn = __ffma2_rn(dwx, Xp[k], __ffma2_rn(dwy, Yp[k], __ffma2_rn(dwz, Zp[k], ndy)));
              sD2[k] = __ffma2_rn(__fmul2_rn(dn, ri), __fmul2_rn(ri, ri), sD2[k]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < TT / 2; ++k) {
          pS[2 * k] = sS2[k].x;
          pS[2 * k + 1] = sS2[k].y;
          pD[2 * k] = sD2[k].x;
          pD[2 * k + 1] = sD2[k].y;
        }
      } else {
#pragma unroll 2
        for (int j = 0; j < tile.z; ++j) {
          const float4 a = sh[j * 2], b = sh[j * 2 + 1];
#pragma unroll
          for (int q = 0; q < TT; ++q) {
            const float dx = X[q] - a.x, dy = Y[q] - a.y, dz = Z[q] - a.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float ri = rsqrt_f32(r2);
            if (DO_S) pS[q] = fmaf(a.w, ri, pS[q]);
            if (DO_D) {
              const float dn = fmaf(b.z, dz, fmaf(b.y, dy, b.x * dx));
              pD[q] = fmaf(dn * ri, ri * ri, pD[q]);
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < TT; ++q) {
        if (!((skipmask >> q) & 1u)) {
          float sum, err;
          if (DO_S) {
            two_sum_f32(acc[(4 * q + 0) * NT + tid], pS[q], sum, err);
            acc[(4 * q + 0) * NT + tid] = sum;
            acc[(4 * q + 1) * NT + tid] += err;
          }
          if (DO_D) {
            two_sum_f32(acc[(4 * q + 2) * NT + tid], pD[q], sum, err);
            acc[(4 * q + 2) * NT + tid] = sum;
            acc[(4 * q + 3) * NT + tid] += err;
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    const int64_t t = t0 + (int64_t)q * NT;
    if (t < t_end) {
      if (DO_S)
        atomicAdd(S_out + t, ((double)acc[(4 * q + 0) * NT + tid] + (double)acc[(4 * q + 1) * NT + tid]) * kInv4Pi);
      if (DO_D)
        atomicAdd(D_out + t, ((double)acc[(4 * q + 2) * NT + tid] + (double)acc[(4 * q + 3) * NT + tid]) * kInv4Pi);
    }
  }
  __syncthreads();   // the shared arrays are reused by the next block of a persistent CTA
}

template <int TT, bool DO_S, bool DO_D, bool PK>
__global__ void __launch_bounds__(kFarTile) far_mixed_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                             const float4* __restrict__ src32,
                                                             const float4* __restrict__ tgt32,
                                                             const float4* __restrict__ cen32,
                                                             const int32_t* __restrict__ skip_ptr,
                                                             const int32_t* __restrict__ skip_idx, int64_t N,
                                                             double* __restrict__ S_out, double* __restrict__ D_out) {
  const int per = (n_tiles + gridDim.y - 1) / gridDim.y;
  const int t_lo = blockIdx.y * per, t_hi = min(n_tiles, t_lo + per);
  far_mixed_block<TT, DO_S, DO_D, PK>((int64_t)blockIdx.x * TT * kFarTile, N, t_lo, t_hi, tiles, src32, tgt32, cen32,
                                      skip_ptr, skip_idx, S_out, D_out);
}

// Direct part of the treecode far field: one CTA per item (target group of
// at most 256 targets [groups[g].x, groups[g].y), tile range of the group's
// tile list).
// 4 targets per thread over 64 threads: a group's 256 targets in one CTA, each
// staged source serving 4 targets per thread (the group tiles are the same)
constexpr int kItemThreads = 64;
__global__ void __launch_bounds__(kItemThreads) far_tile_items_kernel(const int4* __restrict__ items,
                                                                  const int2* __restrict__ groups,
                                                                  const int4* __restrict__ tiles,
                                                                  const float4* __restrict__ src32,
                                                                  const float4* __restrict__ tgt32,
                                                                  const float4* __restrict__ cen32,
                                                                  const int32_t* __restrict__ skip_ptr,
                                                                  const int32_t* __restrict__ skip_idx,
                                                                  double* __restrict__ S_out,
                                                                  double* __restrict__ D_out) {
  const int4 w = items[blockIdx.x];
  const int2 grp = groups[w.x];
  far_mixed_block<4, true, true, true, kItemThreads>(grp.x, grp.y, w.y, w.z, tiles, src32, tgt32, cen32, skip_ptr,
                                                     skip_idx, S_out, D_out);
}

void launch_far_tile_items(const DevGeom& d, const int2* groups, const int4* tiles, const int4* items, int n_items,
                           double* S, double* D, cudaStream_t st) {
  if (n_items <= 0) return;
  far_tile_items_kernel<<<n_items, kItemThreads, 0, st>>>(items, groups, tiles, d.src32, d.tgt32, d.cen32,
                                                          d.skip_ptr, d.skip_idx, S, D);
  count_launch();
}

// Number of source splits so that the grid holds about `waves` resident
// rounds of CTAs on the device (never more splits than tiles).
int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = (dev >= 0 && dev < 64) ? cache[dev] : 0;
  if (sms == 0) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64) cache[dev] = sms;
  }
  return sms;
}

int far_split_count(int64_t target_blocks, int n_tiles, int requested) {
  if (requested > 0) return requested < n_tiles ? requested : n_tiles;
  const int sms = sm_count();
  const int64_t want = (int64_t)sms * 8 * 2;
  int64_t s = (want + target_blocks - 1) / target_blocks;
  if (s < 1) s = 1;
  if (s > n_tiles) s = n_tiles;
  return (int)s;
}

template <int TT, bool PK>
static void launch_far_mixed_tt(const DevGeom& d, int64_t NT, int nt, int splits, double* S, double* D,
                                cudaStream_t st) {
  static_assert(!PK || TT % 2 == 0, "packed form pairs targets");
  const int64_t tb = (NT + kFarTile * TT - 1) / (kFarTile * TT);
  const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, splits));
  if (S && D)
    far_mixed_kernel<TT, true, true, PK><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.src32, d.tgt32, d.cen32,
                                                                    d.skip_ptr, d.skip_idx, NT, S, D);
  else if (S)
    far_mixed_kernel<TT, true, false, PK><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.src32, d.tgt32, d.cen32,
                                                                     d.skip_ptr, d.skip_idx, NT, S, D);
  else
    far_mixed_kernel<TT, false, true, PK><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.src32, d.tgt32, d.cen32,
                                                                     d.skip_ptr, d.skip_idx, NT, S, D);
}

void launch_far_on(const DevGeom& d, const GeomHost& h, int64_t NT, double* S, double* D, cudaStream_t st) {
  if (NT <= 0) return;
  const int nt = (int)h.tiles.size();
  if (h.precision == SBIO_FP64) {
    const int64_t tb = (NT + kFarTile - 1) / kFarTile;
    const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, h.far_splits));
    if (S && D)
      far_fp64_kernel<true, true><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.src64, d.xyz, d.parts, d.skip_ptr,
                                                             d.skip_idx, NT, S, D);
    else if (S)
      far_fp64_kernel<true, false><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.src64, d.xyz, d.parts, d.skip_ptr,
                                                              d.skip_idx, NT, S, D);
    else
      far_fp64_kernel<false, true><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.src64, d.xyz, d.parts, d.skip_ptr,
                                                              d.skip_idx, NT, S, D);
  } else {
    // far_tt < 0 selects the packed f32x2 form with |far_tt| targets per thread
    switch (h.far_tt) {
      case 1: launch_far_mixed_tt<1, false>(d, NT, nt, h.far_splits, S, D, st); break;
      case 4: launch_far_mixed_tt<4, false>(d, NT, nt, h.far_splits, S, D, st); break;
      case 8: launch_far_mixed_tt<8, false>(d, NT, nt, h.far_splits, S, D, st); break;
      case -2: launch_far_mixed_tt<2, true>(d, NT, nt, h.far_splits, S, D, st); break;
      case -4: launch_far_mixed_tt<4, true>(d, NT, nt, h.far_splits, S, D, st); break;
      case -8: launch_far_mixed_tt<8, true>(d, NT, nt, h.far_splits, S, D, st); break;
      default: launch_far_mixed_tt<2, false>(d, NT, nt, h.far_splits, S, D, st); break;
    }
  }
  count_launch();
}

// the treecode replaces the direct sum for mixed S + D applies at the nodes
static bool far_by_tree(const sbio_geom* g, const double* S, const double* D) {
  return g->tree && g->h.precision == SBIO_MIXED && S && D;
}

static void launch_far(sbio_geom* g, double* S, double* D, cudaStream_t st) {
  if (far_by_tree(g, S, D)) {
    launch_tree_far(g, S, D, st);
    return;
  }
  launch_far_on(g->d, g->h, g->h.N, S, D, st);
}

// Persistent far field over many suspensions: CTAs pull work items
// (suspension, target block, first tile, end tile) from an atomic counter
// until the list is exhausted (items are ordered longest first).
template <int TT, bool PK>
__global__ void __launch_bounds__(kFarTile) far_persistent_kernel(const FarDesc* __restrict__ descs,
                                                                  const int4* __restrict__ items, int n_items,
                                                                  int* __restrict__ counter) {
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const int4 w = items[it];
    const FarDesc& D = descs[w.x];
    far_mixed_block<TT, true, true, PK>((int64_t)w.y * TT * kFarTile, D.N, w.z, w.w, D.tiles, D.src32, D.tgt32,
                                        D.cen32, D.skip_ptr, D.skip_idx, D.S, D.D);
  }
}

int launch_far_persistent(const FarDesc* descs, const int4* items, int n_items, int* counter, int tt, int grid,
                          cudaStream_t st) {
  switch (tt) {
    case 1: far_persistent_kernel<1, false><<<grid, kFarTile, 0, st>>>(descs, items, n_items, counter); break;
    case 4: far_persistent_kernel<4, false><<<grid, kFarTile, 0, st>>>(descs, items, n_items, counter); break;
    case 8: far_persistent_kernel<8, false><<<grid, kFarTile, 0, st>>>(descs, items, n_items, counter); break;
    case -2: far_persistent_kernel<2, true><<<grid, kFarTile, 0, st>>>(descs, items, n_items, counter); break;
    case -4: far_persistent_kernel<4, true><<<grid, kFarTile, 0, st>>>(descs, items, n_items, counter); break;
    case -8: far_persistent_kernel<8, true><<<grid, kFarTile, 0, st>>>(descs, items, n_items, counter); break;
    default: far_persistent_kernel<2, false><<<grid, kFarTile, 0, st>>>(descs, items, n_items, counter); break;
  }
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}

// Miller steps of every near pair of the S + D kernel (order P = p): the
// same start index as miller_q01 (K ~ 19/mu above the top order, clamped to
// the geometry's 1/k table), summed into one counter.  Diagnostic: it gives
// the near field's data-dependent FP64 work, which a per-pair constant
// cannot.
__global__ void __launch_bounds__(256) near_work_kernel(const int32_t* __restrict__ pair_t,
                                                        const int32_t* __restrict__ pair_s, int64_t count,
                                                        const PartGeom* __restrict__ parts,
                                                        const double* __restrict__ xyz,
                                                        const double* __restrict__ inv_tab, int P,
                                                        unsigned long long* __restrict__ steps) {
  unsigned long long k_sum = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += (int64_t)gridDim.x * blockDim.x) {
    const int t = pair_t[r], i = pair_s[r];
    const PartGeom& G = parts[i];
    const double dx = xyz[(int64_t)t * 3 + 0] - G.c[0];
    const double dy = xyz[(int64_t)t * 3 + 1] - G.c[1];
    const double dz = xyz[(int64_t)t * 3 + 2] - G.c[2];
    const double xl = G.R[0] * dx + G.R[3] * dy + G.R[6] * dz;
    const double yl = G.R[1] * dx + G.R[4] * dy + G.R[7] * dz;
    const double zl = G.R[2] * dx + G.R[5] * dy + G.R[8] * dz;
    const SphCoord sc = to_spheroidal(xl, yl, zl, G.a, G.kind);
    const double u = sc.u;
    const float muf = logf((float)u + sqrtf((float)(u * u + G.sgn)));
    int K = (int)ceilf(19.0f / muf) + 2;
    const int kmax = (int)inv_tab[0] - P - 8;
    K = K < 4 ? 4 : (K > kmax ? kmax : K);
    k_sum += (unsigned long long)K;
  }
  for (int o = 16; o > 0; o >>= 1) k_sum += __shfl_down_sync(0xffffffffu, k_sum, o);
  if ((threadIdx.x & 31) == 0 && k_sum) atomicAdd(steps, k_sum);
}

int launch_synth_mode(sbio_geom* g, const double* sigma, const double* mu, double* S, double* D, int self_mode,
                      cudaStream_t st, int side) {
  const GeomHost& h = g->h;
  const DevGeom& d = g->d;
  const double* mult = self_mode == 2 ? d.dmult : d.mult;
  const int nmw = 2 * h.p + 1, nc = (h.p + 1) * (h.p + 1);
  const size_t smem = (size_t)(2 * nc + 4 * h.n_v * nmw) * sizeof(double);
  if (smem > 48 * 1024) {
    SBIO_CUDA_TRY(cudaFuncSetAttribute(synth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  synth_kernel<<<h.M, 256, smem, st>>>(h.p, h.n_v, h.n_phi, d.parts, d.xyz, d.nrm, d.w, d.ptab, d.trig, d.sqrtw,
                                       mult, d.normc, sigma, mu, self_mode, side, S, D, d.src64, d.src32,
                                       d.alpha, d.beta, d.alpha32, d.beta32);
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}

int launch_synth(sbio_geom* g, const double* sigma, const double* mu, double* S, double* D, bool write_self,
                 cudaStream_t st) {
  return launch_synth_mode(g, sigma, mu, S, D, write_self ? 1 : 0, st);
}

int launch_near(sbio_geom* g, double* S, double* D, cudaStream_t st) {
  const GeomHost& h = g->h;
  if (h.pair_t.empty()) return SBIO_OK;
  near_launcher f = near_for_p(h.p);
  if (!f) return set_error(SBIO_ENOTSUP, "no near-field kernel for p = %d", h.p);
  f(g->d, h.n_pairs_prolate, (int64_t)h.pair_t.size(), g->d.inv, S, D, h.precision == SBIO_MIXED, st);
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}

int launch_laplace(sbio_geom* g, const double* sigma, const double* mu, double* S, double* D, uint32_t parts,
                   cudaStream_t st, int side) {
  phase_mark(g, 0, st);
  int rc = launch_synth_mode(g, sigma, mu, S, D, (parts & SBIO_PART_SELF) ? 1 : 0, st, side);
  if (rc) return rc;
  phase_mark(g, 1, st);
  // with phase timing on, run the phases in order so that each is timed alone
  const bool fork = g->overlap && !g->timing && g->near_stream && (parts & SBIO_PART_NEAR) &&
                    (parts & SBIO_PART_FAR) && !g->h.pair_t.empty();
  SideFork sf;
  if (fork) {
    SBIO_CUDA_TRY(sf.fork(g, st));
    // a few near CTAs per SM leave room for the far kernels' CTAs (the direct
    // sum and the treecode's phases want different shares)
    const int cap = far_by_tree(g, S, D) ? g->h.tree_near_ctas_per_sm : g->h.near_ctas_per_sm;
    g->d.near_grid_cap = cap > 0 ? cap * sm_count() : 0;
    rc = launch_near(g, S, D, g->near_stream);
    g->d.near_grid_cap = 0;
    if (rc) return rc;
  } else if (parts & SBIO_PART_NEAR) {
    rc = launch_near(g, S, D, st);
    if (rc) return rc;
  }
  phase_mark(g, 2, st);
  if (parts & SBIO_PART_FAR) {
    launch_far(g, S, D, st);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  SBIO_CUDA_TRY(sf.join());
  phase_mark(g, 3, st);
  return SBIO_OK;
}

int tune_launch_shape(sbio_geom* g, const TuneOps& ops, double* out, cudaStream_t st, double* best_far_ms) {
  GeomHost& h = g->h;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SBIO_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(SBIO_ECUDA, "event create failed");
  }
  // median of three event-timed launches after one warm-up
  auto time3 = [&](int (*fn)(sbio_geom*, double*, cudaStream_t), float* ms) -> int {
    int r = fn(g, out, st);
    float t[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < 3 && !r; ++k) {
      cudaEventRecord(e0, st);
      r = fn(g, out, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) r = set_error(SBIO_ECUDA, "autotune timing failed");
      cudaEventElapsedTime(&t[k], e0, e1);
    }
    *ms = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
    return r;
  };
  const int nt = (int)h.tiles.size();
  double best = 1e300;
  int best_tt = *ops.tt, best_sp = *ops.splits;
  const int tts[7] = {1, 2, 4, 8, -2, -4, -8};
  int rc = SBIO_OK;
  for (int a = 0; a < (h.precision == SBIO_FP64 ? 1 : 7) && !rc; ++a) {
    const int tt = (h.precision == SBIO_FP64) ? 1 : tts[a];
    const int att = tt < 0 ? -tt : tt;
    const int64_t tb = (h.N + (int64_t)kFarTile * att - 1) / ((int64_t)kFarTile * att);
    const int base = far_split_count(tb, nt, 0);
    const int cands[6] = {base > 1 ? base / 2 : 1, base, 2 * base, 4 * base, 8 * base, 16 * base};
    for (int b = 0; b < 6 && !rc; ++b) {
      if (b > 0 && cands[b - 1] >= nt) break;
      *ops.tt = tt;
      *ops.splits = cands[b] < nt ? cands[b] : nt;
      float med = 0.f;
      rc = time3(ops.far, &med);
      if (!rc && med < best) {
        best = med;
        best_tt = tt;
        best_sp = *ops.splits;
      }
    }
  }
  *ops.tt = best_tt;
  *ops.splits = best_sp;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  SBIO_CUDA_TRY(cudaGetLastError());
  *best_far_ms = best;
  // near CTAs per SM while the near field overlaps the far field
  return tune_near_cap(g, ops, out, st);
}

int tune_near_cap(sbio_geom* g, const TuneOps& ops, double* out, cudaStream_t st) {
  if (!ops.whole || !g->overlap || !g->near_stream || g->timing || g->h.pair_t.empty()) return SBIO_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SBIO_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(SBIO_ECUDA, "event create failed");
  }
  // whole applies, median of five after one warm-up, per cap
  const int caps[6] = {1, 2, 3, 4, 8, 0};
  float best_apply = 1e30f;
  int best_cap = *ops.cap;
  int rc = SBIO_OK;
  for (int c = 0; c < 6 && !rc; ++c) {
    if (caps[c] != 0 && caps[c] < ops.min_cap) continue;
    *ops.cap = caps[c];
    rc = ops.whole(g, out, st);
    float t[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < 5 && !rc; ++k) {
      cudaEventRecord(e0, st);
      rc = ops.whole(g, out, st);
      cudaEventRecord(e1, st);
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(SBIO_ECUDA, "autotune timing failed");
      if (!rc) cudaEventElapsedTime(&t[k], e0, e1);
    }
    std::sort(t, t + 5);
    const float m = t[2];
    if (!rc && m < best_apply) {
      best_apply = m;
      best_cap = caps[c];
    }
  }
  *ops.cap = best_cap;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}


}  // namespace sbio

using namespace sbio;

extern "C" {

int sbio_apply_laplace_parts(sbio_geom* g, const double* sigma_tilde, const double* mu_hat, double* S_out,
                             double* D_out, uint32_t parts, void* stream) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if ((sigma_tilde == nullptr) != (S_out == nullptr) || (mu_hat == nullptr) != (D_out == nullptr))
    return set_error(SBIO_EINVAL, "each output must be given exactly when its input is");
  if (!sigma_tilde && !mu_hat) return set_error(SBIO_EINVAL, "nothing to apply");
  if (parts & ~SBIO_PART_ALL) return set_error(SBIO_EINVAL, "unknown part bits 0x%x", parts);
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  return launch_laplace(g, sigma_tilde, mu_hat, S_out, D_out, parts, (cudaStream_t)stream);
}

int sbio_apply_laplace(sbio_geom* g, const double* sigma_tilde, const double* mu_hat, double* S_out, double* D_out,
                       void* stream) {
  return sbio_apply_laplace_parts(g, sigma_tilde, mu_hat, S_out, D_out, SBIO_PART_ALL, stream);
}

int sbio_apply_laplace_limit(sbio_geom* g, const double* sigma_tilde, const double* mu_hat, double* S_out,
                             double* D_out, int32_t side, void* stream) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (side < -1 || side > 1) return set_error(SBIO_EINVAL, "side %d: -1 (interior), 0 or +1 (exterior)", side);
  if ((sigma_tilde == nullptr) != (S_out == nullptr) || (mu_hat == nullptr) != (D_out == nullptr))
    return set_error(SBIO_EINVAL, "each output must be given exactly when its input is");
  if (!sigma_tilde && !mu_hat) return set_error(SBIO_EINVAL, "nothing to apply");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  return launch_laplace(g, sigma_tilde, mu_hat, S_out, D_out, SBIO_PART_ALL, (cudaStream_t)stream, side);
}

int sbio_apply_laplace_host(sbio_geom* g, const double* sigma_host, const double* mu_host, double* S_host,
                            double* D_host, void* stream) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if ((sigma_host == nullptr) != (S_host == nullptr) || (mu_host == nullptr) != (D_host == nullptr))
    return set_error(SBIO_EINVAL, "each output must be given exactly when its input is");
  if (!sigma_host && !mu_host) return set_error(SBIO_EINVAL, "nothing to apply");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nc = (size_t)(g->h.p + 1) * (g->h.p + 1) * g->h.M;
  const size_t N = (size_t)g->h.N;
  double* ds = sigma_host ? g->d.host_in : nullptr;
  double* dm = mu_host ? g->d.host_in + nc : nullptr;
  double* oS = S_host ? g->d.host_out : nullptr;
  double* oD = D_host ? g->d.host_out + N : nullptr;
  if (ds) SBIO_CUDA_TRY(cudaMemcpyAsync(ds, sigma_host, nc * sizeof(double), cudaMemcpyHostToDevice, st));
  if (dm) SBIO_CUDA_TRY(cudaMemcpyAsync(dm, mu_host, nc * sizeof(double), cudaMemcpyHostToDevice, st));
  int rc = launch_laplace(g, ds, dm, oS, oD, SBIO_PART_ALL, st);
  if (rc) return rc;
  if (oS) SBIO_CUDA_TRY(cudaMemcpyAsync(S_host, oS, N * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (oD) SBIO_CUDA_TRY(cudaMemcpyAsync(D_host, oD, N * sizeof(double), cudaMemcpyDeviceToHost, st));
  SBIO_CUDA_TRY(cudaStreamSynchronize(st));
  return SBIO_OK;
}

int sbio_geom_set_launch_shape(sbio_geom* g, int32_t far_tt, int32_t far_splits) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (far_tt != 1 && far_tt != 2 && far_tt != 4 && far_tt != 8 && far_tt != -2 && far_tt != -4 && far_tt != -8)
    return set_error(SBIO_EINVAL, "far_tt must be 1, 2, 4, 8 or -2, -4, -8 (packed)");
  if (far_splits < 0) return set_error(SBIO_EINVAL, "far_splits must be >= 0");
  g->h.far_tt = far_tt;
  g->h.far_splits = far_splits;
  return SBIO_OK;
}

int sbio_geom_set_near_cap(sbio_geom* g, int32_t ctas_per_sm) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (ctas_per_sm < 0) return set_error(SBIO_EINVAL, "ctas_per_sm must be >= 0");
  g->h.near_ctas_per_sm = ctas_per_sm;
  return SBIO_OK;
}

int sbio_geom_near_work(sbio_geom* g, int64_t* n_pairs, int64_t* miller_steps) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  const int64_t np = (int64_t)g->h.pair_t.size();
  unsigned long long steps = 0;
  if (np > 0) {
    unsigned long long* d_steps = nullptr;
    SBIO_CUDA_TRY(cudaMalloc(&d_steps, sizeof(unsigned long long)));
    cudaError_t e = cudaMemset(d_steps, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
      const int64_t nb = std::min<int64_t>((np + 255) / 256, (int64_t)sm_count() * 8);
      near_work_kernel<<<(unsigned)nb, 256>>>(g->d.pair_t, g->d.pair_s, np, g->d.parts, g->d.xyz, g->d.inv, g->h.p,
                                              d_steps);
      count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&steps, d_steps, sizeof(steps), cudaMemcpyDeviceToHost);
    cudaFree(d_steps);
    if (e != cudaSuccess) return set_error(SBIO_ECUDA, "near work count failed: %s", cudaGetErrorString(e));
  }
  if (n_pairs) *n_pairs = np;
  if (miller_steps) *miller_steps = (int64_t)steps;
  return SBIO_OK;
}

int sbio_geom_get_tuning(const sbio_geom* g, int32_t* far_tt, int32_t* far_splits, int32_t* near_ctas_per_sm) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (far_tt) *far_tt = g->h.far_tt;
  if (far_splits) *far_splits = g->h.far_splits;
  if (near_ctas_per_sm) *near_ctas_per_sm = g->h.near_ctas_per_sm;
  return SBIO_OK;
}

int sbio_geom_autotune(sbio_geom* g, void* stream, int32_t* far_tt, int32_t* far_splits, double* far_ms) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  GeomHost& h = g->h;
  DevGeom& d = g->d;
  const size_t nc = (size_t)(h.p + 1) * (h.p + 1) * h.M;
  // valid (zero-strength) sources so that the timed kernels read finite data
  SBIO_CUDA_TRY(cudaMemsetAsync(d.host_in, 0, 2 * nc * sizeof(double), st));
  int rc = launch_laplace(g, d.host_in, d.host_in + nc, d.host_out, d.host_out + h.N, SBIO_PART_SELF, st);
  if (rc) return rc;
  TuneOps ops;
  ops.far = [](sbio_geom* gg, double* out, cudaStream_t s) {
    launch_far(gg, out, out + gg->h.N, s);
    return SBIO_OK;
  };
  ops.whole = [](sbio_geom* gg, double* out, cudaStream_t s) {
    const size_t n = (size_t)(gg->h.p + 1) * (gg->h.p + 1) * gg->h.M;
    return launch_laplace(gg, gg->d.host_in, gg->d.host_in + n, out, out + gg->h.N, SBIO_PART_ALL, s);
  };
  ops.tt = &h.far_tt;
  ops.splits = &h.far_splits;
  ops.cap = &h.near_ctas_per_sm;
  double best = 0.0;
  // the direct kernel's shapes are tuned with the direct far field, also
  // when the geometry uses the treecode (whose direct part has a fixed shape)
  TreeFar* tree = g->tree;
  g->tree = nullptr;
  rc = tune_launch_shape(g, ops, d.host_out, st, &best);
  g->tree = tree;
  if (rc) return rc;
  if (tree) {
    // the near kernels' share beside the treecode's phases
    ops.cap = &h.tree_near_ctas_per_sm;
    rc = tune_near_cap(g, ops, d.host_out, st);
    if (rc) return rc;
  }
  if (far_tt) *far_tt = h.far_tt;
  if (far_splits) *far_splits = h.far_splits;
  if (far_ms) *far_ms = best;
  return SBIO_OK;
}

int sbio_apply_stokes_sl(sbio_geom* g, const double* f_tilde, double* u_out, void* stream) {
  clear_error();
  if (!g || !f_tilde || !u_out) return set_error(SBIO_EINVAL, "null argument");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  return launch_stokes(g, f_tilde, u_out, (cudaStream_t)stream);
}

int sbio_apply_stokes_sl_host(sbio_geom* g, const double* f_host, double* u_host, void* stream) {
  clear_error();
  if (!g || !f_host || !u_host) return set_error(SBIO_EINVAL, "null argument");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nc3 = (size_t)3 * (g->h.p + 1) * (g->h.p + 1) * g->h.M;
  const size_t n3 = (size_t)3 * g->h.N;
  SBIO_CUDA_TRY(cudaMemcpyAsync(g->d.host_in, f_host, nc3 * sizeof(double), cudaMemcpyHostToDevice, st));
  int rc = launch_stokes(g, g->d.host_in, g->d.host_out, st);
  if (rc) return rc;
  SBIO_CUDA_TRY(cudaMemcpyAsync(u_host, g->d.host_out, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SBIO_CUDA_TRY(cudaStreamSynchronize(st));
  return SBIO_OK;
}

int sbio_geom_set_stokes_tuning(sbio_geom* g, int32_t far_tt, int32_t far_splits, int32_t near_ctas_per_sm) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (far_tt != 1 && far_tt != 2 && far_tt != 4 && far_tt != 8 && far_tt != -2 && far_tt != -4 && far_tt != -8)
    return set_error(SBIO_EINVAL, "far_tt must be 1, 2, 4, 8 or -2, -4, -8 (packed)");
  if (far_splits < 0 || near_ctas_per_sm < 0) return set_error(SBIO_EINVAL, "far_splits and near cap must be >= 0");
  g->h.st_far_tt = far_tt;
  g->h.st_far_splits = far_splits;
  g->h.st_near_ctas_per_sm = near_ctas_per_sm;
  return SBIO_OK;
}

int sbio_geom_get_stokes_tuning(const sbio_geom* g, int32_t* far_tt, int32_t* far_splits, int32_t* near_ctas_per_sm) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (far_tt) *far_tt = g->h.st_far_tt;
  if (far_splits) *far_splits = g->h.st_far_splits;
  if (near_ctas_per_sm) *near_ctas_per_sm = g->h.st_near_ctas_per_sm;
  return SBIO_OK;
}

int sbio_geom_autotune_stokes(sbio_geom* g, void* stream, int32_t* far_tt, int32_t* far_splits, double* far_ms) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  GeomHost& h = g->h;
  DevGeom& d = g->d;
  const size_t nc3 = (size_t)3 * (h.p + 1) * (h.p + 1) * h.M;
  // zero forces: one whole apply writes finite Stokeslet sources for the far timings
  SBIO_CUDA_TRY(cudaMemsetAsync(d.host_in, 0, nc3 * sizeof(double), st));
  int rc = launch_stokes(g, d.host_in, d.host_out, st);
  if (rc) return rc;
  TuneOps ops;
  ops.far = [](sbio_geom* gg, double* out, cudaStream_t s) { return launch_stokes_far(gg, out, s); };
  ops.whole = [](sbio_geom* gg, double* out, cudaStream_t s) { return launch_stokes(gg, gg->d.host_in, out, s); };
  ops.tt = &h.st_far_tt;
  ops.splits = &h.st_far_splits;
  ops.cap = &h.st_near_ctas_per_sm;
  // the Stokes near kernels run 64-thread CTAs: caps of 1 or 2 CTAs per SM
  // starve them (stokes100 ran 911 applies/s at 2, 974 at 8 or uncapped,
  // while the whole-apply timings of the tuner differ by less than its noise)
  ops.min_cap = 4;
  double best = 0.0;
  TreeFar* tree = g->tree;   // tune the direct Stokeslet kernel's shapes
  g->tree = nullptr;
  rc = tune_launch_shape(g, ops, d.host_out, st, &best);
  g->tree = tree;
  if (rc) return rc;
  if (far_tt) *far_tt = h.st_far_tt;
  if (far_splits) *far_splits = h.st_far_splits;
  if (far_ms) *far_ms = best;
  return SBIO_OK;
}

}  // extern "C"
