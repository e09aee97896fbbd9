// Normal-derivative operators S'[sigma] and D'[mu] at every surface node
// (Sec. 3.3, Theorem 3 and eq. (dSLevalformula); Sec. 4.2 "Other layer
// potentials"), with the same three-way split as the layer potentials:
//   self: the synthesis kernel with the derivative multipliers (S' the
//         average of the exterior and interior limits, D' continuous) and
//         the 1/h_u surface factor;
//   near: gradient of the source's exterior expansions dotted with the
//         target's normal (sbio_deriv_near.cuh);
//   far:  smooth quadrature of the differentiated kernels
//         S': -q nu_x . r / (4 pi |r|^3)
//         D': (d . nu_x / |r|^3 - 3 (d . r)(nu_x . r) / |r|^5) / (4 pi),
//         r = x - y, q = w sigma, d = w mu nu_y (the far sources of the
//         synthesis kernel).
#include "sbio_deriv_near.cuh"
#include "sbio_internal.cuh"

namespace sbio {

deriv_near_launcher deriv_near_lookup_a(int p);
deriv_near_launcher deriv_near_lookup_b(int p);

namespace {

constexpr double kInv4PiD = 0.07957747154594767;   // 1/(4 pi)

struct alignas(32) dd4 {
  double x, y, z, w;
};

// FP64 form: one target per thread, kFarTile sources per shared-memory tile.
template <bool DO_S, bool DO_D>
__global__ void __launch_bounds__(kFarTile) far_deriv_fp64_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                                  const double* __restrict__ src64,
                                                                  const double* __restrict__ xyz,
                                                                  const double* __restrict__ nrm,
                                                                  const PartGeom* __restrict__ parts,
                                                                  const int32_t* __restrict__ skip_ptr,
                                                                  const int32_t* __restrict__ skip_idx, int64_t N,
                                                                  double* __restrict__ Sp_out,
                                                                  double* __restrict__ Dp_out) {
  __shared__ dd4 sh[kFarTile * 2];
  const int64_t t = (int64_t)blockIdx.x * kFarTile + threadIdx.x;
  const bool valid = t < N;
  double x = 0, y = 0, z = 0, nx = 0, ny = 0, nz = 0;
  int sp = 0, nxt = INT32_MAX;
  if (valid) {
    x = xyz[t * 3 + 0];
    y = xyz[t * 3 + 1];
    z = xyz[t * 3 + 2];
    nx = nrm[t * 3 + 0];
    ny = nrm[t * 3 + 1];
    nz = nrm[t * 3 + 2];
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
      const dd4* s = reinterpret_cast<const dd4*>(src64 + (int64_t)(tile.y + threadIdx.x) * 8);
      sh[threadIdx.x * 2 + 0] = s[0];
      sh[threadIdx.x * 2 + 1] = s[1];
    }
    __syncthreads();
    if (!skip) {
      for (int j = 0; j < tile.z; ++j) {
        const dd4 a = sh[j * 2], b = sh[j * 2 + 1];
        const double dx = X - a.x, dy = Y - a.y, dz = Z - a.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double ri = rsqrt(r2);
        const double ri2 = ri * ri, ri3 = ri2 * ri;
        const double rn = dx * nx + dy * ny + dz * nz;
        if (DO_S) accS = fma(-a.w * rn, ri3, accS);
        if (DO_D) {
          const double dr = b.x * dx + b.y * dy + b.z * dz;
          const double dn = b.x * nx + b.y * ny + b.z * nz;
          accD = fma(fma(-3.0 * dr * rn, ri2, dn), ri3, accD);
        }
      }
    }
    __syncthreads();
  }
  if (valid) {
    if (DO_S) atomicAdd(Sp_out + t, accS * kInv4PiD);
    if (DO_D) atomicAdd(Dp_out + t, accD * kInv4PiD);
  }
}

// Mixed form: FP32 pair sums, TT targets per thread, the targets taken
// relative to each source particle's centre through hi/lo FP32 parts, per-tile
// partials folded into (hi, lo) pairs by TwoSum in shared memory (the same
// scheme as the layer-potential far field).
template <int TT, bool DO_S, bool DO_D, bool PK>
__global__ void __launch_bounds__(kFarTile) far_deriv_mixed_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                                   const float4* __restrict__ src32,
                                                                   const float4* __restrict__ tgt32,
                                                                   const float4* __restrict__ cen32,
                                                                   const double* __restrict__ nrm,
                                                                   const int32_t* __restrict__ skip_ptr,
                                                                   const int32_t* __restrict__ skip_idx, int64_t N,
                                                                   double* __restrict__ Sp_out,
                                                                   double* __restrict__ Dp_out) {
  // scalar form: (y - c, -q), (d, 0) per source.  The packed form (two
  // targets per f32x2 operation) uses the expanded distance
  // |x - y|^2 = (|x|^2 + |y|^2) - 2 x.y, nu.(x - y) = nu.x + (nu/2).(-2y) and
  // -3 d.(x - y) = (-3d).x + 3 d.y, d.nu = (2d).(nu/2), with per source, every
  // value duplicated into a pair: -2y (3), |y|^2, -q, -3d (3), 3 d.y, 2d (3).
  __shared__ float4 sh[(PK ? 6 : 2) * kFarTile];
  __shared__ float acc[4 * TT * kFarTile];   // per target: S' hi, lo, D' hi, lo
  __shared__ int cursor[2 * TT * kFarTile];  // per target: skip-list position, next skipped particle
  const int tid = threadIdx.x;
  const int per = (n_tiles + gridDim.y - 1) / gridDim.y;
  const int t_lo = blockIdx.y * per, t_hi = min(n_tiles, t_lo + per);
  const int64_t t0 = (int64_t)blockIdx.x * TT * kFarTile + tid;
  float NX[TT], NY[TT], NZ[TT];
#pragma unroll
  for (int q = 0; q < TT; ++q) {
    const int64_t t = t0 + (int64_t)q * kFarTile;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[(4 * q + k) * kFarTile + tid] = 0.f;
    const int sp = (t < N) ? skip_ptr[t] : 0;
    cursor[(2 * q + 0) * kFarTile + tid] = sp;
    cursor[(2 * q + 1) * kFarTile + tid] = (t < N) ? skip_idx[sp] : INT32_MAX;
    NX[q] = (t < N) ? (float)nrm[t * 3 + 0] : 0.f;
    NY[q] = (t < N) ? (float)nrm[t * 3 + 1] : 0.f;
    NZ[q] = (t < N) ? (float)nrm[t * 3 + 2] : 0.f;
  }
  float X[TT], Y[TT], Z[TT], XX[TT], NXX[TT];
  if (PK) {
#pragma unroll
    for (int q = 0; q < TT; ++q) {   // the packed form takes nu / 2
      NX[q] *= 0.5f;
      NY[q] *= 0.5f;
      NZ[q] *= 0.5f;
    }
  }
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
        if (PK) {
          XX[q] = fmaf(Z[q], Z[q], fmaf(Y[q], Y[q], X[q] * X[q]));
          NXX[q] = 2.f * fmaf(NZ[q], Z[q], fmaf(NY[q], Y[q], NX[q] * X[q]));   // nu.x
        }
      }
    }
    const bool mine = skipmask != (1u << TT) - 1u;
    if (!__syncthreads_or(mine)) continue;
    if (tid < tile.z) {
      const float4 a = src32[(int64_t)(tile.y + tid) * 2 + 0];
      const float4 b = src32[(int64_t)(tile.y + tid) * 2 + 1];
      if (PK) {
        const float yy = fmaf(a.z, a.z, fmaf(a.y, a.y, a.x * a.x));
        const float dy3 = 3.f * fmaf(b.z, a.z, fmaf(b.y, a.y, b.x * a.x));
        sh[tid * 6 + 0] = make_float4(-2.f * a.x, -2.f * a.x, -2.f * a.y, -2.f * a.y);
        sh[tid * 6 + 1] = make_float4(-2.f * a.z, -2.f * a.z, yy, yy);
        sh[tid * 6 + 2] = make_float4(-a.w, -a.w, -3.f * b.x, -3.f * b.x);
        sh[tid * 6 + 3] = make_float4(-3.f * b.y, -3.f * b.y, -3.f * b.z, -3.f * b.z);
        sh[tid * 6 + 4] = make_float4(dy3, dy3, 2.f * b.x, 2.f * b.x);
        sh[tid * 6 + 5] = make_float4(2.f * b.y, 2.f * b.y, 2.f * b.z, 2.f * b.z);
      } else {
        sh[tid * 2 + 0] = make_float4(a.x, a.y, a.z, -a.w);
        sh[tid * 2 + 1] = b;
      }
    }
    __syncthreads();
    if (mine) {
      float pS[TT], pD[TT];
#pragma unroll
      for (int q = 0; q < TT; ++q) pS[q] = pD[q] = 0.f;
      if constexpr (PK) {
        constexpr int TP = TT / 2 > 0 ? TT / 2 : 1;
        float2 Xp[TP], Yp[TP], Zp[TP], XXp[TP], NXXp[TP], NXp[TP], NYp[TP], NZp[TP], sS2[TP], sD2[TP];
#pragma unroll
        for (int k = 0; k < TT / 2; ++k) {
          Xp[k] = make_float2(X[2 * k], X[2 * k + 1]);
          Yp[k] = make_float2(Y[2 * k], Y[2 * k + 1]);
          Zp[k] = make_float2(Z[2 * k], Z[2 * k + 1]);
          XXp[k] = make_float2(XX[2 * k], XX[2 * k + 1]);
          NXXp[k] = make_float2(NXX[2 * k], NXX[2 * k + 1]);
          NXp[k] = make_float2(NX[2 * k], NX[2 * k + 1]);
          NYp[k] = make_float2(NY[2 * k], NY[2 * k + 1]);
          NZp[k] = make_float2(NZ[2 * k], NZ[2 * k + 1]);
          sS2[k] = make_float2(0.f, 0.f);
          sD2[k] = make_float2(0.f, 0.f);
        }
#pragma unroll 2
        for (int j = 0; j < tile.z; ++j) {
          const float4 A = sh[j * 6 + 0], B = sh[j * 6 + 1], Cc = sh[j * 6 + 2], Dd = sh[j * 6 + 3],
                       Ee = sh[j * 6 + 4], Ff = sh[j * 6 + 5];
          const float2 m2x = make_float2(A.x, A.y), m2y = make_float2(A.z, A.w), m2z = make_float2(B.x, B.y);
          const float2 yy = make_float2(B.z, B.w), nq = make_float2(Cc.x, Cc.y), e0 = make_float2(Cc.z, Cc.w);
          const float2 e1 = make_float2(Dd.x, Dd.y), e2 = make_float2(Dd.z, Dd.w), dy3 = make_float2(Ee.x, Ee.y);
          const float2 d0 = make_float2(Ee.z, Ee.w), d1 = make_float2(Ff.x, Ff.y), d2 = make_float2(Ff.z, Ff.w);
#pragma unroll
          for (int k = 0; k < TT / 2; ++k) {
            const float2 r2 =
                __ffma2_rn(Xp[k], m2x, __ffma2_rn(Yp[k], m2y, __ffma2_rn(Zp[k], m2z, __fadd2_rn(XXp[k], yy))));
            const float2 ri = make_float2(rsqrt_f32(r2.x), rsqrt_f32(r2.y));
            const float2 ri2 = __fmul2_rn(ri, ri), ri3 = __fmul2_rn(ri2, ri);
            // nu.(x - y) = nu.x + (nu/2).(-2y)
            const float2 rn = __ffma2_rn(NZp[k], m2z, __ffma2_rn(NYp[k], m2y, __ffma2_rn(NXp[k], m2x, NXXp[k])));
            if (DO_S) sS2[k] = __ffma2_rn(__fmul2_rn(nq, rn), ri3, sS2[k]);
            if (DO_D) {
              const float2 dr3 = __ffma2_rn(e2, Zp[k], __ffma2_rn(e1, Yp[k], __ffma2_rn(e0, Xp[k], dy3)));   // -3 d.r
              const float2 dn = __ffma2_rn(d2, NZp[k], __ffma2_rn(d1, NYp[k], __fmul2_rn(d0, NXp[k])));     // d.nu
              sD2[k] = __ffma2_rn(__ffma2_rn(__fmul2_rn(dr3, rn), ri2, dn), ri3, sD2[k]);
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
          const float ri2 = ri * ri, ri3 = ri2 * ri;
          const float rn = fmaf(dz, NZ[q], fmaf(dy, NY[q], dx * NX[q]));
          if (DO_S) pS[q] = fmaf(a.w * rn, ri3, pS[q]);
          if (DO_D) {
            const float dr = fmaf(b.z, dz, fmaf(b.y, dy, b.x * dx));
            const float dn = fmaf(b.z, NZ[q], fmaf(b.y, NY[q], b.x * NX[q]));
            pD[q] = fmaf(fmaf(-3.f * dr * rn, ri2, dn), ri3, pD[q]);
          }
        }
      }
      }
#pragma unroll
      for (int q = 0; q < TT; ++q) {
        if (!((skipmask >> q) & 1u)) {
          float sum, err;
          if (DO_S) {
            two_sum_f32(acc[(4 * q + 0) * kFarTile + tid], pS[q], sum, err);
            acc[(4 * q + 0) * kFarTile + tid] = sum;
            acc[(4 * q + 1) * kFarTile + tid] += err;
          }
          if (DO_D) {
            two_sum_f32(acc[(4 * q + 2) * kFarTile + tid], pD[q], sum, err);
            acc[(4 * q + 2) * kFarTile + tid] = sum;
            acc[(4 * q + 3) * kFarTile + tid] += err;
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
      if (DO_S)
        atomicAdd(Sp_out + t,
                  ((double)acc[(4 * q + 0) * kFarTile + tid] + (double)acc[(4 * q + 1) * kFarTile + tid]) * kInv4PiD);
      if (DO_D)
        atomicAdd(Dp_out + t,
                  ((double)acc[(4 * q + 2) * kFarTile + tid] + (double)acc[(4 * q + 3) * kFarTile + tid]) * kInv4PiD);
    }
  }
}

// Mixed derivative far kernel: 4 targets per thread in the scalar form, or 8
// in the packed f32x2 form when the geometry's tuned Laplace far shape is a
// packed one (far_tt < 0).
template <int TT, bool PK, bool DO_S, bool DO_D>
void launch_far_deriv_mixed_tt(const DevGeom& d, const GeomHost& h, int64_t N, double* Sp, double* Dp,
                               cudaStream_t st) {
  const int nt = (int)h.tiles.size();
  const int64_t tb = (N + (int64_t)kFarTile * TT - 1) / ((int64_t)kFarTile * TT);
  // the packed form takes the geometry's tuned source splits (tuned for the
  // same packed target blocking of the Laplace kernel)
  const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, PK ? h.far_splits : 0));
  far_deriv_mixed_kernel<TT, DO_S, DO_D, PK><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.src32, d.tgt32, d.cen32,
                                                                        d.nrm, d.skip_ptr, d.skip_idx, N, Sp, Dp);
}

// N targets: the geometry's nodes, or the points of a target-set view (whose
// xyz, tgt32, nrm and skip lists are the points').
template <bool DO_S, bool DO_D>
void launch_far_deriv_sd(const DevGeom& d, const GeomHost& h, int64_t N, double* Sp, double* Dp, cudaStream_t st) {
  const int nt = (int)h.tiles.size();
  if (h.precision == SBIO_FP64) {
    const int64_t tb = (N + kFarTile - 1) / kFarTile;
    const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, 0));
    far_deriv_fp64_kernel<DO_S, DO_D><<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.src64, d.xyz, d.nrm, d.parts,
                                                                 d.skip_ptr, d.skip_idx, N, Sp, Dp);
  } else if (h.far_tt < 0) {
    launch_far_deriv_mixed_tt<8, true, DO_S, DO_D>(d, h, N, Sp, Dp, st);
  } else {
    launch_far_deriv_mixed_tt<4, false, DO_S, DO_D>(d, h, N, Sp, Dp, st);
  }
  count_launch();
}

void launch_far_deriv(const DevGeom& d, const GeomHost& h, int64_t N, double* Sp, double* Dp, cudaStream_t st) {
  if (N <= 0) return;
  if (Sp && Dp)
    launch_far_deriv_sd<true, true>(d, h, N, Sp, Dp, st);
  else if (Sp)
    launch_far_deriv_sd<true, false>(d, h, N, Sp, Dp, st);
  else
    launch_far_deriv_sd<false, true>(d, h, N, Sp, Dp, st);
}

deriv_near_launcher deriv_near_for_p(int p) {
  deriv_near_launcher nl = deriv_near_lookup_a(p);
  return nl ? nl : deriv_near_lookup_b(p);
}

}  // namespace

int launch_laplace_deriv(sbio_geom* g, const double* sigma, const double* mu, double* Sp, double* Dp,
                         cudaStream_t st, int side) {
  const GeomHost& h = g->h;
  if (h.p > 20) return set_error(SBIO_ENOTSUP, "S' / D' are built for p <= 20 (p = %d)", h.p);
  deriv_near_launcher nl = deriv_near_for_p(h.p);
  if (!nl) return set_error(SBIO_ENOTSUP, "no S' / D' near-field kernel for p = %d", h.p);
  phase_mark(g, 0, st);
  // self: writes (initialises) the outputs, and the far sources and near
  // coefficients of this apply
  int rc = launch_synth_mode(g, sigma, mu, Sp, Dp, 2, st, side);
  if (rc) return rc;
  phase_mark(g, 1, st);
  const bool fork = g->overlap && !g->timing && g->near_stream && !h.pair_t.empty();
  SideFork sf;
  if (fork) {
    SBIO_CUDA_TRY(sf.fork(g, st));
    g->d.near_grid_cap = h.near_ctas_per_sm > 0 ? h.near_ctas_per_sm * sm_count() : 0;
    nl(g->d, h.n_pairs_prolate, (int64_t)h.pair_t.size(), Sp, Dp, g->near_stream);
    g->d.near_grid_cap = 0;
    SBIO_CUDA_TRY(cudaGetLastError());
  } else if (!h.pair_t.empty()) {
    nl(g->d, h.n_pairs_prolate, (int64_t)h.pair_t.size(), Sp, Dp, st);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  phase_mark(g, 2, st);
  launch_far_deriv(g->d, h, h.N, Sp, Dp, st);
  SBIO_CUDA_TRY(cudaGetLastError());
  SBIO_CUDA_TRY(sf.join());
  phase_mark(g, 3, st);
  return SBIO_OK;
}

}  // namespace sbio

using namespace sbio;

extern "C" {

int sbio_apply_laplace_deriv(sbio_geom* g, const double* sigma_tilde, const double* mu_hat, double* Sp_out,
                             double* Dp_out, void* stream) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if ((sigma_tilde == nullptr) != (Sp_out == nullptr) || (mu_hat == nullptr) != (Dp_out == nullptr))
    return set_error(SBIO_EINVAL, "each output must be given exactly when its input is");
  if (!sigma_tilde && !mu_hat) return set_error(SBIO_EINVAL, "nothing to apply");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  return launch_laplace_deriv(g, sigma_tilde, mu_hat, Sp_out, Dp_out, (cudaStream_t)stream);
}

int sbio_apply_laplace_deriv_limit(sbio_geom* g, const double* sigma_tilde, const double* mu_hat, double* Sp_out,
                                   double* Dp_out, int32_t side, void* stream) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (side < -1 || side > 1) return set_error(SBIO_EINVAL, "side %d: -1 (interior), 0 or +1 (exterior)", side);
  if ((sigma_tilde == nullptr) != (Sp_out == nullptr) || (mu_hat == nullptr) != (Dp_out == nullptr))
    return set_error(SBIO_EINVAL, "each output must be given exactly when its input is");
  if (!sigma_tilde && !mu_hat) return set_error(SBIO_EINVAL, "nothing to apply");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  return launch_laplace_deriv(g, sigma_tilde, mu_hat, Sp_out, Dp_out, (cudaStream_t)stream, side);
}

int sbio_eval_targets_deriv(sbio_targets* ts, const double* dirs, const double* sigma_tilde, const double* mu_hat,
                            double* Sp_out, double* Dp_out, void* stream) {
  clear_error();
  sbio_geom* g = nullptr;
  const DevGeom* view = nullptr;
  int64_t T = 0, n_pro = 0, n_pairs = 0;
  int rc = targets_view(ts, &g, &view, &T, &n_pro, &n_pairs);
  if (rc) return rc;
  if ((sigma_tilde == nullptr) != (Sp_out == nullptr) || (mu_hat == nullptr) != (Dp_out == nullptr))
    return set_error(SBIO_EINVAL, "each output must be given exactly when its input is");
  if (!sigma_tilde && !mu_hat) return set_error(SBIO_EINVAL, "nothing to evaluate");
  if (T > 0 && !dirs) return set_error(SBIO_EINVAL, "null directions");
  const GeomHost& h = g->h;
  if (h.p > 20) return set_error(SBIO_ENOTSUP, "S' / D' are built for p <= 20 (p = %d)", h.p);
  deriv_near_launcher nl = deriv_near_for_p(h.p);
  if (!nl) return set_error(SBIO_ENOTSUP, "no S' / D' near-field kernel for p = %d", h.p);
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  if (T == 0) return SBIO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (Sp_out) SBIO_CUDA_TRY(cudaMemsetAsync(Sp_out, 0, T * sizeof(double), st));
  if (Dp_out) SBIO_CUDA_TRY(cudaMemsetAsync(Dp_out, 0, T * sizeof(double), st));
  // far sources and near coefficients of these densities (no self output)
  rc = launch_synth_mode(g, sigma_tilde, mu_hat, nullptr, nullptr, 0, st);
  if (rc) return rc;
  // the set's view with the directions as the target "normals": the near
  // kernel dots the expansion gradient with them, the far kernels the
  // differentiated quadrature; source normals are not read by either
  DevGeom v = *view;
  v.nrm = const_cast<double*>(dirs);   // read only
  const bool fork = g->overlap && !g->timing && g->near_stream && n_pairs > 0;
  SideFork sf;
  if (fork) {
    SBIO_CUDA_TRY(sf.fork(g, st));
    v.near_grid_cap = h.near_ctas_per_sm > 0 ? h.near_ctas_per_sm * sm_count() : 0;
    nl(v, n_pro, n_pairs, Sp_out, Dp_out, g->near_stream);
    v.near_grid_cap = 0;
    SBIO_CUDA_TRY(cudaGetLastError());
  } else if (n_pairs > 0) {
    nl(v, n_pro, n_pairs, Sp_out, Dp_out, st);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  launch_far_deriv(v, h, T, Sp_out, Dp_out, st);
  SBIO_CUDA_TRY(cudaGetLastError());
  SBIO_CUDA_TRY(sf.join());
  return SBIO_OK;
}

}  // extern "C"
