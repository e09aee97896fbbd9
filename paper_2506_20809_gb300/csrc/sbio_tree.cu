// Far field by a particle treecode (mixed precision), for suspensions past
// the size where the O(N^2) direct sum stops being the kernel of choice.  The
// paper evaluates its far field with an FMM (Sec. 4.1 "Far-field", Sec. 4.2);
// this is a Barnes-Hut style treecode over the particles with solid-harmonic
// multipoles, built to reproduce the same discrete far sum as the direct
// kernel: the smooth quadrature over the nodes of every particle that is
// neither the target's own nor one of its near particles.
//
// Expansions.  With the solid harmonics (m >= 0; P_n^m with the
// Condon-Shortley phase)
//     R_n^m(r) = r^n P_n^m(cos t) e^{i m p} / (n+m)!,
//     I_n^m(r) = (n-m)! P_n^m(cos t) e^{i m p} / r^{n+1},
// R_n^{-m} = (-1)^m conj(R_n^m), likewise I, the addition theorem reads
//     1 / |x - y| = sum_{n, |m| <= n} conj(R_n^m(y - c)) I_n^m(x - c),  |y-c| < |x-c|,
// so a cluster of charges q_j and dipoles d_j about c has the multipoles
//     M_n^m = sum_j q_j conj(R_n^m(y_j - c))                       (S)
//     M_n^m = sum_j d_j . grad conj(R_n^m)(y_j - c)                 (D)
// and its potential is sum_n [M_n^0 I_n^0 + 2 Re sum_{m>0} M_n^m I_n^m].
// The dipole moments use the ladder relations d/dz R_n^m = R_{n-1}^m,
// (d/dx + i d/dy) R_n^m = R_{n-1}^{m+1}, (d/dx - i d/dy) R_n^m = -R_{n-1}^{m-1}:
//     d . grad conj(R_n^m) = d_z conj R_{n-1}^m + delta conj R_{n-1}^{m+1}
//                            - conj(delta) conj R_{n-1}^{m-1},  delta = (d_x + i d_y)/2.
// A parent's multipoles are its children's translated by
//     M'_n^m = sum_{k <= n, |l| <= k} conj(R_k^l(c - c')) M_{n-k}^{m-l}.
// Both harmonics follow three-term recurrences in Cartesian coordinates
// (x, y, z, r^2), so no trigonometric function is evaluated.
//
// Tree and lists (host, once per geometry and accuracy setting).  A binary
// tree over the particles, split at the median centre along the longest
// extent; a leaf is one particle (its centre and major semi-axis bound all of
// its nodes).  Targets are taken in groups of at most 256 consecutive nodes
// of one particle (the direct kernel's target block).  For each group a walk from the root accepts
// a node when, for every target of the group, |x - c_n| >= r_n / theta and
// the node holds none of the group's own or near particles; a leaf that is
// not accepted goes to the group's direct list, evaluated by the direct
// mixed kernel with the per-target skip lists, so each (target, particle)
// pair outside the target's own and near set is counted exactly once.
// An accepted node is evaluated at the lowest order E of {8, 12, 16} (at
// most the tree's order P) whose truncation factor rho^(E+1), with
// rho = r_n / (|c_g - c_n| - R_g) over the group's bounding sphere, is no
// larger than s theta^(P+1), theta^(P+1) being the factor of the worst node
// accepted at order P: s = 1 for the Laplace S + D (the per-node bound stays
// that of order P at theta), s = 1/10 for the Stokes single layer, whose
// eight channels add the truncation errors of more terms.
//
// Per apply: leaf multipoles from the FP32 sources (FP32 per warp with TwoSum
// compensation for the orders n < 4 that carry most of the far field, FP64
// across warps), translations up the tree for the nodes the lists read (FP64
// for the orders n < 8, FP32 above, where a coefficient weighs at most
// theta^n of the field), conversion to FP32, then
// the direct part and the multipole evaluations (FP32, per-node sums folded
// by TwoSum), each added atomically into the FP64 outputs.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "sbio_internal.cuh"

namespace sbio {

constexpr int kTreeGroup = 2 * kFarTile;   // most targets per group (direct kernel: 2 per thread)
constexpr int kTreeChunkNodes = 16;        // multipole nodes per evaluation CTA
constexpr int kTreeChunkTiles = 32;        // direct source tiles per CTA
constexpr double kInv4PiTree = 0.07957747154594767;

struct TreeNodeH {
  double c[3];
  double r;
  int first, count;   // particle range in tree order
  int child[2];
  int level;
};

struct TreeFar {
  int order = 16;
  double theta = 0.5;
  int n_nodes = 0, n_levels = 0, n_groups = 0;
  std::vector<TreeNodeH> nodes;
  std::vector<int> perm;                     // tree position -> particle
  std::vector<int> pos;                      // particle -> tree position
  std::vector<std::vector<int>> levels;      // internal node ids per level
  int64_t m2p_pairs = 0, direct_pairs = 0, m2p_entries = 0, direct_tiles = 0;
  int64_t m2p_source_pairs = 0;   // (target, source node) pairs the accepted nodes stand for
  int n_translated = 0;            // internal nodes whose multipoles are formed per apply
  // device
  double* d_geo = nullptr;        // n_nodes x 4: centre, radius
  float4* d_c32 = nullptr;        // n_nodes x 2: hi, lo parts of the centre
  int* d_child = nullptr;         // n_nodes x 2
  int* d_leaf = nullptr;          // particle -> node id
  int* d_levels = nullptr;        // internal node ids, level by level (deepest last)
  std::vector<int> level_off;     // offsets into d_levels
  double2* d_M = nullptr;         // n_nodes x 2 x NM: FP64 multipoles (S, D)
  float2* d_M32 = nullptr;        // n_nodes x 2 x NM: FP32, m > 0 doubled
  // Stokes single layer: 4 channel planes of n_nodes x 2 x NM (charges F_1,
  // F_2, F_3, 0 with dipoles F, (y-c)_x F, (y-c)_y F, (y-c)_z F)
  double2* d_SM = nullptr;
  float2* d_SM32 = nullptr;
  int2* d_groups = nullptr;       // target range [first, end) of every group
  int4* d_tiles = nullptr;        // direct source tiles, group after group
  int4* d_ditems = nullptr;       // (group, first tile, end tile, 0)
  int n_ditems = 0;
  // evaluation lists, one per operator (0 Laplace, 1 Stokes: the orders
  // differ, the accepted nodes do not)
  struct EvalLists {
    int* d_mlist = nullptr;          // accepted node ids, group after group, by order class
    int4* d_mitems = nullptr;        // (group, first entry, end entry, order class), by class
    int off[4] = {0, 0, 0, 0};       // items of evaluation order 8 + 4 c: [off[c], off[c + 1])
    int64_t evals_by_order[3] = {0, 0, 0};
  } ev_lists[2];
  // host images of the uploaded tables (kept until the tree is dropped, so
  // that an upload queued on a stream may read them after the build returns)
  std::vector<std::vector<char>> host_images;
  // phase events of the last apply while the geometry's timing is on:
  // leaf multipoles | translations + FP32 copy | direct part | evaluations
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // the direct part runs on its own stream beside the multipole phases (it
  // needs no multipoles); null when the geometry runs its phases in order
  cudaStream_t side = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
  ~TreeFar() {
    for (cudaEvent_t& e : ev)
      if (e) cudaEventDestroy(e);
    if (side_fork) cudaEventDestroy(side_fork);
    if (side_join) cudaEventDestroy(side_join);
    if (side) cudaStreamDestroy(side);
  }
};

void tree_free(TreeFar* t) { delete t; }

__host__ __device__ constexpr int tree_nm(int p) { return (p + 1) * (p + 2) / 2; }
__host__ __device__ inline int tree_idx(int n, int m) { return n * (n + 1) / 2 + m; }

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Leaf multipoles about each particle's centre from its nodes' FP32 sources
// (y - c, q), (d, 0).  One CTA (8 warps) per particle; lane m of a warp owns
// column m of the harmonics and all warps step through n together, so the
// dipole terms can take R_{n-1}^{m+-1} from the neighbouring lanes.
constexpr int kP2MWarps = 8;

// SRC = 0: the Laplace sources (y - c, q), (d, 0).  SRC = 1..4: channel
// SRC - 1 of the Stokes sources (y - c, F_1), (F_2, F_3, 0, 0), F = w f:
// charges F_1, F_2, F_3, 0 and dipoles F, (y - c)_x F, (y - c)_y F, (y - c)_z F.
template <int PF, int SRC>
__global__ void __launch_bounds__(32 * kP2MWarps) tree_p2m_kernel(int G, const float4* __restrict__ src32,
                                                       const int* __restrict__ leaf, double2* __restrict__ Mout) {
  constexpr int NM = tree_nm(PF);
  constexpr int NC = 4;   // orders n < NC carry TwoSum compensation (they dominate the far field)
  __shared__ float red[kP2MWarps][PF + 1][PF + 1][4];   // [warp][column m][order n]
  __shared__ float redc[kP2MWarps][PF + 1][NC][4];
  const int i = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = lane;
  float aSr[PF + 1], aSi[PF + 1], aDr[PF + 1], aDi[PF + 1];
  float cSr[NC], cSi[NC], cDr[NC], cDi[NC];
#pragma unroll
  for (int n = 0; n <= PF; ++n) aSr[n] = aSi[n] = aDr[n] = aDi[n] = 0.f;
#pragma unroll
  for (int n = 0; n < NC; ++n) cSr[n] = cSi[n] = cDr[n] = cDi[n] = 0.f;
  for (int j = warp; j < G; j += kP2MWarps) {
    const float4 A = src32[((int64_t)i * G + j) * 2 + 0];
    const float4 B = src32[((int64_t)i * G + j) * 2 + 1];
    const float x = A.x, y = A.y, z = A.z;
    float q, ddx, ddy, ddz;
    if (SRC == 0) {
      q = A.w;
      ddx = B.x;
      ddy = B.y;
      ddz = B.z;
    } else {
      const float w = SRC == 1 ? 1.f : (SRC == 2 ? x : (SRC == 3 ? y : z));
      q = SRC == 1 ? A.w : (SRC == 2 ? B.x : (SRC == 3 ? B.y : 0.f));
      ddx = w * A.w;
      ddy = w * B.x;
      ddz = w * B.y;
    }
    const float r2 = fmaf(z, z, fmaf(y, y, x * x));
    const float dr = 0.5f * ddx, di = 0.5f * ddy, dz = ddz;   // delta = (d_x + i d_y) / 2
    // R_m^m = (-(x + i y) / 2)^m / m!
    float mr = 1.f, mi = 0.f;
#pragma unroll
    for (int k = 1; k <= PF; ++k) {
      if (k <= m) {
        const float s = -0.5f / (float)k;
        const float tr = s * (x * mr - y * mi), ti = s * (x * mi + y * mr);
        mr = tr;
        mi = ti;
      }
    }
    float r1r = 0.f, r1i = 0.f, r2r = 0.f, r2i = 0.f;   // R_{n-1}^m, R_{n-2}^m of this lane's column
#pragma unroll
    for (int n = 0; n <= PF; ++n) {
      float cr, ci;
      if (n < m) {
        cr = ci = 0.f;
      } else if (n == m) {
        cr = mr;
        ci = mi;
      } else if (n == m + 1) {
        cr = z * r1r;
        ci = z * r1i;
      } else {
        const float f = 1.f / (float)((n - m) * (n + m));
        const float a = (float)(2 * n - 1) * z;
        cr = (a * r1r - r2 * r2r) * f;
        ci = (a * r1i - r2 * r2i) * f;
      }
      // R_{n-1} of the neighbouring columns (zero where the column has not started)
      const float upr = __shfl_down_sync(0xffffffffu, r1r, 1), upi = __shfl_down_sync(0xffffffffu, r1i, 1);
      const float dnr = __shfl_up_sync(0xffffffffu, r1r, 1), dni = __shfl_up_sync(0xffffffffu, r1i, 1);
      if (m <= PF && n >= m) {
        if (n < NC) {
          float s2, e2;
          two_sum_f32(aSr[n], q * cr, s2, e2);
          aSr[n] = s2;
          cSr[n] += e2;
          two_sum_f32(aSi[n], -q * ci, s2, e2);
          aSi[n] = s2;
          cSi[n] += e2;
        } else {
          aSr[n] = fmaf(q, cr, aSr[n]);
          aSi[n] = fmaf(-q, ci, aSi[n]);
        }
        if (n >= 1) {
          float er = dz * r1r, ei = -dz * r1i;                   // d_z conj R_{n-1}^m
          er += dr * upr + di * upi;                              // delta conj R_{n-1}^{m+1}
          ei += di * upr - dr * upi;
          if (m >= 1) {                                           // - conj(delta) conj R_{n-1}^{m-1}
            er -= dr * dnr - di * dni;
            ei += dr * dni + di * dnr;
          } else {                                                // m = 0: + conj(delta) R_{n-1}^{1}
            er += dr * upr + di * upi;
            ei += dr * upi - di * upr;
          }
          if (n < NC) {
            float s2, e2;
            two_sum_f32(aDr[n], er, s2, e2);
            aDr[n] = s2;
            cDr[n] += e2;
            two_sum_f32(aDi[n], ei, s2, e2);
            aDi[n] = s2;
            cDi[n] += e2;
          } else {
            aDr[n] += er;
            aDi[n] += ei;
          }
        }
      }
      r2r = r1r;
      r2i = r1i;
      r1r = cr;
      r1i = ci;
    }
  }
  if (lane <= PF) {
#pragma unroll
    for (int n = 0; n <= PF; ++n) {
      red[warp][lane][n][0] = aSr[n];
      red[warp][lane][n][1] = aSi[n];
      red[warp][lane][n][2] = aDr[n];
      red[warp][lane][n][3] = aDi[n];
    }
#pragma unroll
    for (int n = 0; n < NC; ++n) {
      redc[warp][lane][n][0] = cSr[n];
      redc[warp][lane][n][1] = cSi[n];
      redc[warp][lane][n][2] = cDr[n];
      redc[warp][lane][n][3] = cDi[n];
    }
  }
  __syncthreads();
  const int node = leaf[i];
  for (int k = threadIdx.x; k < NM; k += blockDim.x) {
    int n = 0;
    while (tree_idx(n + 1, 0) <= k) ++n;
    const int mm = k - tree_idx(n, 0);
    double sr = 0, si = 0, er = 0, ei = 0;
#pragma unroll
    for (int w = 0; w < kP2MWarps; ++w) {
      sr += red[w][mm][n][0];
      si += red[w][mm][n][1];
      er += red[w][mm][n][2];
      ei += red[w][mm][n][3];
      if (n < NC) {
        sr += redc[w][mm][n][0];
        si += redc[w][mm][n][1];
        er += redc[w][mm][n][2];
        ei += redc[w][mm][n][3];
      }
    }
    Mout[((int64_t)node * 2 + 0) * NM + k] = make_double2(sr, si);
    Mout[((int64_t)node * 2 + 1) * NM + k] = make_double2(er, ei);
  }
}

// value of a stored (n, m >= 0) table at order l of either sign, for tables
// of real sources: T_n^{-l} = (-1)^l conj(T_n^l)
__device__ __forceinline__ double2 signed_order(const double2* T, int n, int l) {
  if (l >= 0) return T[tree_idx(n, l)];
  const double2 v = T[tree_idx(n, -l)];
  return (l & 1) ? make_double2(-v.x, v.y) : make_double2(v.x, -v.y);
}

__device__ __forceinline__ float2 signed_order32(const float2* T, int n, int l) {
  if (l >= 0) return T[tree_idx(n, l)];
  const float2 v = T[tree_idx(n, -l)];
  return (l & 1) ? make_float2(-v.x, v.y) : make_float2(v.x, -v.y);
}

// One tree level: each internal node's multipoles from its two children's.
// The 2 NM outputs of a node are spread over gridDim.y CTAs of kM2MThreads
// threads (one output per thread), so that the short top levels still use
// many SMs: the translation is FP64 and the FP64 pipe is the bound.
constexpr int kM2MThreads = 64;
constexpr int kM2MExactOrders = 8;   // output orders n below this are translated in FP64

// Several channel planes at once (blockIdx.z, planes `plane` double2 apart,
// as the Stokes channels): a plane z >= 1 with `shifted` set carries dipoles
// weighted by (y - c)_{z-1} of its own node's centre, so before translation
// each child's dipole part gets (c_child - c_parent)_{z-1} times plane 0's
// dipole part (the weight moves with the expansion centre).
template <int PF>
__global__ void __launch_bounds__(kM2MThreads) tree_m2m_kernel(const int* __restrict__ ids,
                                                               const int* __restrict__ child,
                                                               const double* __restrict__ geo,
                                                               double2* __restrict__ Mbase, int64_t plane,
                                                               int shifted) {
  constexpr int NM = tree_nm(PF);
  __shared__ double2 Rb[2][NM];
  __shared__ double2 Mc[2][2][NM];
  __shared__ float2 Rb32[2][NM];       // FP32 copies for the high orders (converted once:
  __shared__ float2 Mc32[2][2][NM];    // double-to-float conversions run at the FP64 rate)
  const int node = ids[blockIdx.x];
  const int ch0 = child[node * 2 + 0], ch1 = child[node * 2 + 1];
  double2* __restrict__ Mt = Mbase + blockIdx.z * plane;
  const int axis = (shifted && blockIdx.z > 0) ? (int)blockIdx.z - 1 : -1;
  // R_k^l of the two child offsets, one column l per thread (lanes 0..PF of
  // warp 0 for the first child, of warp 1 for the second): the FP64 pipe
  // issues at 1/64 of the FP32 rate, so a serial recurrence by one thread
  // would set the time of the whole level
  {
    const int k = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l <= PF) {
      const int c = k ? ch1 : ch0;
      const double x = geo[c * 4 + 0] - geo[node * 4 + 0], y = geo[c * 4 + 1] - geo[node * 4 + 1],
                   z = geo[c * 4 + 2] - geo[node * 4 + 2];
      const double r2 = x * x + y * y + z * z;
      double mr = 1.0, mi = 0.0;   // R_l^l = (-(x + i y) / 2)^l / l!
      for (int q = 1; q <= l; ++q) {
        const double sc = -0.5 / q;
        const double tr = sc * (x * mr - y * mi), ti = sc * (x * mi + y * mr);
        mr = tr;
        mi = ti;
      }
      double2* R = Rb[k];
      R[tree_idx(l, l)] = make_double2(mr, mi);
      double ar = mr, ai = mi, br = 0.0, bi = 0.0;   // R_{n-1}^l, R_{n-2}^l
      for (int n = l + 1; n <= PF; ++n) {
        const double f = 1.0 / ((double)(n - l) * (n + l));
        const double cr = ((2 * n - 1) * z * ar - r2 * br) * f, ci = ((2 * n - 1) * z * ai - r2 * bi) * f;
        R[tree_idx(n, l)] = make_double2(cr, ci);
        br = ar;
        bi = ai;
        ar = cr;
        ai = ci;
      }
    }
  }
  for (int k = threadIdx.x; k < 4 * NM; k += blockDim.x) {
    const int c = k / (2 * NM), rest = k - c * 2 * NM;
    const int cn = c ? ch1 : ch0;
    double2 v = Mt[((int64_t)cn * 2 + rest / NM) * NM + rest % NM];
    if (axis >= 0 && rest >= NM) {
      const double b = geo[cn * 4 + axis] - geo[node * 4 + axis];
      const double2 v0 = Mbase[((int64_t)cn * 2 + 1) * NM + rest % NM];
      v = make_double2(fma(b, v0.x, v.x), fma(b, v0.y, v.y));
    }
    Mc[c][rest / NM][rest % NM] = v;
    Mc32[c][rest / NM][rest % NM] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * NM; k += blockDim.x) {
    const double2 v = Rb[k / NM][k % NM];
    Rb32[k / NM][k % NM] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (k >= 2 * NM) return;
  const int kind = k / NM, idx = k - kind * NM;
  int n = 0;
  while (tree_idx(n + 1, 0) <= idx) ++n;
  const int m = idx - tree_idx(n, 0);
  double ar = 0.0, ai = 0.0;
  if (n < kM2MExactOrders) {
    for (int c = 0; c < 2; ++c) {
      for (int kk = 0; kk <= n; ++kk) {
        const int nn = n - kk;
        // |m - l| <= nn and |l| <= kk
        const int l_lo = max(-kk, m - nn), l_hi = min(kk, m + nn);
        for (int l = l_lo; l <= l_hi; ++l) {
          const double2 r = signed_order(Rb[c], kk, l);
          const double2 v = signed_order(Mc[c][kind], nn, m - l);
          // conj(r) * v
          ar = fma(r.x, v.x, fma(r.y, v.y, ar));
          ai = fma(r.x, v.y, fma(-r.y, v.x, ai));
        }
      }
    }
  } else {
    // orders n >= kM2MExactOrders hold most of the terms but weigh at most
    // theta^n of the node's field at any accepted target: FP32 products and
    // sums (their rounding is below 1e-9 of the field) at 64x the FP64 rate
    float fr = 0.f, fi = 0.f;
    for (int c = 0; c < 2; ++c) {
      for (int kk = 0; kk <= n; ++kk) {
        const int nn = n - kk;
        const int l_lo = max(-kk, m - nn), l_hi = min(kk, m + nn);
        for (int l = l_lo; l <= l_hi; ++l) {
          const float2 r = signed_order32(Rb32[c], kk, l);
          const float2 v = signed_order32(Mc32[c][kind], nn, m - l);
          fr = fmaf(r.x, v.x, fmaf(r.y, v.y, fr));
          fi = fmaf(r.x, v.y, fmaf(-r.y, v.x, fi));
        }
      }
    }
    ar = fr;
    ai = fi;
  }
  Mt[((int64_t)node * 2 + kind) * NM + idx] = make_double2(ar, ai);
}

// FP32 copy of every node's multipoles with the m > 0 terms doubled, so the
// evaluation is sum_{n, m >= 0} Re(M I)
template <int PF>
__global__ void tree_to_f32_kernel(int64_t total, const double2* __restrict__ Mt, float2* __restrict__ M32) {
  constexpr int NM = tree_nm(PF);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int idx = (int)(k % NM);
    int n = 0;
    while (tree_idx(n + 1, 0) <= idx) ++n;
    const double w = (idx - tree_idx(n, 0)) > 0 ? 2.0 : 1.0;
    const double2 v = Mt[k];
    M32[k] = make_float2((float)(w * v.x), (float)(w * v.y));
  }
}

// Multipole evaluation: one CTA per (group of at most 256 targets, up to
// kTreeChunkNodes accepted nodes), two targets per thread packed into one
// f32x2 lane pair (sm_100+ packed FP32), so each recurrence and contraction
// step issues once for both.  The node's coefficients are staged in shared
// memory already broadcast to lane pairs: (re, re, -im, -im).
template <int PF, int PE>
__global__ void __launch_bounds__(kFarTile) tree_m2p_kernel(const int4* __restrict__ items, const int2* __restrict__ groups,
                                                            const int* __restrict__ mlist,
                                                            const float4* __restrict__ c32,
                                                            const float2* __restrict__ M32,
                                                            const float4* __restrict__ tgt32,
                                                            double* __restrict__ S_out, double* __restrict__ D_out) {
  constexpr int NMF = tree_nm(PF);   // stored coefficients per node and operator
  constexpr int NM = tree_nm(PE);    // evaluated ones (orders n <= PE)
  __shared__ float4 cf[2 * NM];
  __shared__ float4 cc[2];
  const int4 it = items[blockIdx.x];
  const int2 grp = groups[it.x];
  const int64_t N = grp.y;
  const int tid = threadIdx.x;
  int64_t t[2];
  float4 xh[2], xl[2];
  float hS[2], lS[2], hD[2], lD[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    t[q] = (int64_t)grp.x + q * kFarTile + tid;
    xh[q] = xl[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t[q] < N) {
      xh[q] = tgt32[t[q] * 2 + 0];
      xl[q] = tgt32[t[q] * 2 + 1];
    }
    hS[q] = lS[q] = hD[q] = lD[q] = 0.f;
  }
  for (int e = it.y; e < it.z; ++e) {
    const int node = mlist[e];
    __syncthreads();
    for (int k = tid; k < 2 * NM; k += kFarTile) {
      const int op = k >= NM ? 1 : 0;
      const float2 v = M32[((int64_t)node * 2 + op) * NMF + (k - op * NM)];
      cf[k] = make_float4(v.x, v.x, -v.y, -v.y);
    }
    if (tid < 2) cc[tid] = c32[node * 2 + tid];
    __syncthreads();
    const float4 ch = cc[0], cl = cc[1];
    float Xs[2], Ys[2], Zs[2], I2[2], R0[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float X = (xh[q].x - ch.x) + (xl[q].x - cl.x);
      const float Y = (xh[q].y - ch.y) + (xl[q].y - cl.y);
      const float Z = (xh[q].z - ch.z) + (xl[q].z - cl.z);
      const float r2 = fmaf(Z, Z, fmaf(Y, Y, X * X));
      const float ri = rsqrt_f32(r2);
      I2[q] = ri * ri;
      Xs[q] = X * I2[q];
      Ys[q] = Y * I2[q];
      Zs[q] = Z * I2[q];
      R0[q] = ri;
    }
    const float2 xs = make_float2(Xs[0], Xs[1]), ys = make_float2(Ys[0], Ys[1]);
    const float2 zs = make_float2(Zs[0], Zs[1]), ir2 = make_float2(I2[0], I2[1]);
    float2 Ir = make_float2(R0[0], R0[1]), Ii = make_float2(0.f, 0.f);   // I_m^m, from I_0^0 = 1 / r
    float2 sS = make_float2(0.f, 0.f), sD = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m <= PE; ++m) {
      if (m > 0) {
        // I_m^m = -(2m - 1) (x + i y) / r^2 I_{m-1}^{m-1}
        const float2 s2 = make_float2(-(float)(2 * m - 1), -(float)(2 * m - 1));
        const float2 wr = __fmul2_rn(s2, xs), wi = __fmul2_rn(s2, ys);
        const float2 tr = __ffma2_rn(wr, Ir, __fmul2_rn(make_float2(-wi.x, -wi.y), Ii));
        const float2 ti = __ffma2_rn(wr, Ii, __fmul2_rn(wi, Ir));
        Ir = tr;
        Ii = ti;
      }
      {
        const float4 a = cf[tree_idx(m, m)], b = cf[NM + tree_idx(m, m)];
        sS = __ffma2_rn(make_float2(a.x, a.y), Ir, __ffma2_rn(make_float2(a.z, a.w), Ii, sS));
        sD = __ffma2_rn(make_float2(b.x, b.y), Ir, __ffma2_rn(make_float2(b.z, b.w), Ii, sD));
      }
      float2 ar = Ir, ai = Ii, br = make_float2(0.f, 0.f), bi = make_float2(0.f, 0.f);   // I_{n-1}^m, I_{n-2}^m
#pragma unroll
      for (int n = m + 1; n <= PE; ++n) {
        // I_n^m = ((2n - 1) z I_{n-1}^m - (n-1-m)(n-1+m) I_{n-2}^m) / r^2
        const float kz = (float)(2 * n - 1), kb = -(float)((n - 1 - m) * (n - 1 + m));
        const float2 u = __fmul2_rn(make_float2(kz, kz), zs), v = __fmul2_rn(make_float2(kb, kb), ir2);
        const float2 cr = __ffma2_rn(u, ar, __fmul2_rn(v, br)), ci = __ffma2_rn(u, ai, __fmul2_rn(v, bi));
        const float4 a = cf[tree_idx(n, m)], b = cf[NM + tree_idx(n, m)];
        sS = __ffma2_rn(make_float2(a.x, a.y), cr, __ffma2_rn(make_float2(a.z, a.w), ci, sS));
        sD = __ffma2_rn(make_float2(b.x, b.y), cr, __ffma2_rn(make_float2(b.z, b.w), ci, sD));
        br = ar;
        bi = ai;
        ar = cr;
        ai = ci;
      }
    }
    const float pS[2] = {sS.x, sS.y}, pD[2] = {sD.x, sD.y};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float s, e;
      two_sum_f32(hS[q], pS[q], s, e);
      hS[q] = s;
      lS[q] += e;
      two_sum_f32(hD[q], pD[q], s, e);
      hD[q] = s;
      lD[q] += e;
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (t[q] < N) {
      atomicAdd(S_out + t[q], ((double)hS[q] + (double)lS[q]) * kInv4PiTree);
      atomicAdd(D_out + t[q], ((double)hD[q] + (double)lD[q]) * kInv4PiTree);
    }
}

// Stokes single layer from the four channel planes: per target
//   8 pi u_i = S[F_i] + (x - c)_i D[F] - D[(y - c)_i F]
// (the Stokeslet f/r + (r.f) r/r^3 written through Laplace charges and
// dipoles about the node's centre c), two targets per thread packed in f32x2.
template <int PF, int PE>
__global__ void __launch_bounds__(kFarTile, 4) tree_m2p_stokes_kernel(
    const int4* __restrict__ items, const int2* __restrict__ groups, const int* __restrict__ mlist,
    const float4* __restrict__ c32, const float2* __restrict__ M32, int64_t plane, const float4* __restrict__ tgt32,
    double* __restrict__ u_out) {
  constexpr int NMF = tree_nm(PF);   // stored coefficients per node, plane and kind
  constexpr int NM = tree_nm(PE);    // evaluated ones (orders n <= PE)
  constexpr double kInv8Pi = 0.039788735772973836;
  // blocks b = 0..6 of NM coefficients: (plane z, kind k) = (b / 2, b % 2); the
  // charges of plane 3 are zero and not read (its dipoles are block 6)
  __shared__ float4 cf[7 * NM];
  __shared__ float4 cc[2];
  const int4 it = items[blockIdx.x];
  const int2 grp = groups[it.x];
  const int64_t N = grp.y;
  const int tid = threadIdx.x;
  int64_t t[2];
  float4 xh[2], xl[2];
  float hU[2][3], lU[2][3];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    t[q] = (int64_t)grp.x + q * kFarTile + tid;
    xh[q] = xl[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t[q] < N) {
      xh[q] = tgt32[t[q] * 2 + 0];
      xl[q] = tgt32[t[q] * 2 + 1];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) hU[q][c] = lU[q][c] = 0.f;
  }
  for (int e = it.y; e < it.z; ++e) {
    const int node = mlist[e];
    __syncthreads();
    for (int k = tid; k < 7 * NM; k += kFarTile) {
      const int b = k / NM, idx = k - b * NM;
      const int blk = b < 6 ? b : 7;   // 2 z + kind
      const float2 v = M32[(blk >> 1) * plane + ((int64_t)node * 2 + (blk & 1)) * NMF + idx];
      cf[k] = make_float4(v.x, v.x, -v.y, -v.y);
    }
    if (tid < 2) cc[tid] = c32[node * 2 + tid];
    __syncthreads();
    const float4 ch = cc[0], cl = cc[1];
    float Xr[2], Yr[2], Zr[2], Xs[2], Ys[2], Zs[2], I2[2], R0[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      Xr[q] = (xh[q].x - ch.x) + (xl[q].x - cl.x);
      Yr[q] = (xh[q].y - ch.y) + (xl[q].y - cl.y);
      Zr[q] = (xh[q].z - ch.z) + (xl[q].z - cl.z);
      const float r2 = fmaf(Zr[q], Zr[q], fmaf(Yr[q], Yr[q], Xr[q] * Xr[q]));
      const float ri = rsqrt_f32(r2);
      I2[q] = ri * ri;
      Xs[q] = Xr[q] * I2[q];
      Ys[q] = Yr[q] * I2[q];
      Zs[q] = Zr[q] * I2[q];
      R0[q] = ri;
    }
    const float2 xs = make_float2(Xs[0], Xs[1]), ys = make_float2(Ys[0], Ys[1]);
    const float2 zs = make_float2(Zs[0], Zs[1]), ir2 = make_float2(I2[0], I2[1]);
    float2 Ir = make_float2(R0[0], R0[1]), Ii = make_float2(0.f, 0.f);
    float2 acc[7];
#pragma unroll
    for (int b = 0; b < 7; ++b) acc[b] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m <= PE; ++m) {
      if (m > 0) {
        const float2 s2 = make_float2(-(float)(2 * m - 1), -(float)(2 * m - 1));
        const float2 wr = __fmul2_rn(s2, xs), wi = __fmul2_rn(s2, ys);
        const float2 tr = __ffma2_rn(wr, Ir, __fmul2_rn(make_float2(-wi.x, -wi.y), Ii));
        const float2 ti = __ffma2_rn(wr, Ii, __fmul2_rn(wi, Ir));
        Ir = tr;
        Ii = ti;
      }
#pragma unroll
      for (int b = 0; b < 7; ++b) {
        const float4 a = cf[b * NM + tree_idx(m, m)];
        acc[b] = __ffma2_rn(make_float2(a.x, a.y), Ir, __ffma2_rn(make_float2(a.z, a.w), Ii, acc[b]));
      }
      float2 ar = Ir, ai = Ii, br = make_float2(0.f, 0.f), bi = make_float2(0.f, 0.f);
#pragma unroll
      for (int n = m + 1; n <= PE; ++n) {
        const float kz = (float)(2 * n - 1), kb = -(float)((n - 1 - m) * (n - 1 + m));
        const float2 u = __fmul2_rn(make_float2(kz, kz), zs), v = __fmul2_rn(make_float2(kb, kb), ir2);
        const float2 cr = __ffma2_rn(u, ar, __fmul2_rn(v, br)), ci = __ffma2_rn(u, ai, __fmul2_rn(v, bi));
#pragma unroll
        for (int b = 0; b < 7; ++b) {
          const float4 a = cf[b * NM + tree_idx(n, m)];
          acc[b] = __ffma2_rn(make_float2(a.x, a.y), cr, __ffma2_rn(make_float2(a.z, a.w), ci, acc[b]));
        }
        br = ar;
        bi = ai;
        ar = cr;
        ai = ci;
      }
    }
    // acc[2 z] = S of plane z < 3 (charges F_1, F_2, F_3), acc[2 z + 1] = D of
    // plane z < 3, acc[6] = D of plane 3
    const float Sx[2] = {acc[0].x, acc[0].y}, Sy[2] = {acc[2].x, acc[2].y}, Sz[2] = {acc[4].x, acc[4].y};
    const float D0[2] = {acc[1].x, acc[1].y}, Dx[2] = {acc[3].x, acc[3].y}, Dy[2] = {acc[5].x, acc[5].y},
                Dz[2] = {acc[6].x, acc[6].y};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float uv[3] = {fmaf(Xr[q], D0[q], Sx[q] - Dx[q]), fmaf(Yr[q], D0[q], Sy[q] - Dy[q]),
                           fmaf(Zr[q], D0[q], Sz[q] - Dz[q])};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float s2, e2;
        two_sum_f32(hU[q][c], uv[c], s2, e2);
        hU[q][c] = s2;
        lU[q][c] += e2;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (t[q] < N)
#pragma unroll
      for (int c = 0; c < 3; ++c) atomicAdd(u_out + t[q] * 3 + c, ((double)hU[q][c] + (double)lU[q][c]) * kInv8Pi);
}

// ---------------------------------------------------------------------------
// host: tree, lists, launches
// ---------------------------------------------------------------------------

static int build_nodes(TreeFar& T, const GeomHost& h, int lo, int hi, int level) {
  const int id = (int)T.nodes.size();
  T.nodes.push_back(TreeNodeH());
  double bmin[3] = {1e300, 1e300, 1e300}, bmax[3] = {-1e300, -1e300, -1e300};
  for (int k = lo; k < hi; ++k) {
    const PartGeom& P = h.parts[T.perm[k]];
    const double R = std::max(P.A, P.C);
    for (int c = 0; c < 3; ++c) {
      bmin[c] = std::min(bmin[c], P.c[c] - R);
      bmax[c] = std::max(bmax[c], P.c[c] + R);
    }
  }
  TreeNodeH nd;
  double r = 0.0;
  for (int c = 0; c < 3; ++c) nd.c[c] = 0.5 * (bmin[c] + bmax[c]);
  for (int k = lo; k < hi; ++k) {
    const PartGeom& P = h.parts[T.perm[k]];
    const double d = std::sqrt((P.c[0] - nd.c[0]) * (P.c[0] - nd.c[0]) + (P.c[1] - nd.c[1]) * (P.c[1] - nd.c[1]) +
                               (P.c[2] - nd.c[2]) * (P.c[2] - nd.c[2]));
    r = std::max(r, d + std::max(P.A, P.C));
  }
  nd.r = r;
  nd.first = lo;
  nd.count = hi - lo;
  nd.child[0] = nd.child[1] = -1;
  nd.level = level;
  T.n_levels = std::max(T.n_levels, level + 1);
  if (hi - lo > 1) {
    double cmin[3] = {1e300, 1e300, 1e300}, cmax[3] = {-1e300, -1e300, -1e300};
    for (int k = lo; k < hi; ++k)
      for (int c = 0; c < 3; ++c) {
        cmin[c] = std::min(cmin[c], h.parts[T.perm[k]].c[c]);
        cmax[c] = std::max(cmax[c], h.parts[T.perm[k]].c[c]);
      }
    int ax = 0;
    for (int c = 1; c < 3; ++c)
      if (cmax[c] - cmin[c] > cmax[ax] - cmin[ax]) ax = c;
    std::stable_sort(T.perm.begin() + lo, T.perm.begin() + hi,
                     [&](int a, int b) { return h.parts[a].c[ax] < h.parts[b].c[ax]; });
    const int mid = lo + (hi - lo) / 2;
    T.nodes[id] = nd;
    const int c0 = build_nodes(T, h, lo, mid, level + 1);
    const int c1 = build_nodes(T, h, mid, hi, level + 1);
    T.nodes[id].child[0] = c0;
    T.nodes[id].child[1] = c1;
    return id;
  }
  T.nodes[id] = nd;
  return id;
}

// Device copy of a host table, ordered on `st`; the host bytes are kept in
// the tree until it is dropped.
template <typename V>
static int upload_vec(sbio_geom* g, TreeFar& T, V** dst, const std::vector<V>& v, const char* what,
                      cudaStream_t st) {
  if (v.empty()) {
    *dst = nullptr;
    return SBIO_OK;
  }
  int rc = dev_alloc(g, (void**)dst, v.size() * sizeof(V), what);
  if (rc) return rc;
  T.host_images.emplace_back(reinterpret_cast<const char*>(v.data()),
                             reinterpret_cast<const char*>(v.data()) + v.size() * sizeof(V));
  SBIO_CUDA_TRY(cudaMemcpyAsync(*dst, T.host_images.back().data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, st));
  return SBIO_OK;
}

static int build_tree(sbio_geom* g, TreeFar& T, cudaStream_t st) {
  const GeomHost& h = g->h;
  const int M = h.M, G = h.G;
  T.perm.resize(M);
  for (int i = 0; i < M; ++i) T.perm[i] = i;
  T.nodes.clear();
  T.nodes.reserve(2 * M);
  T.n_levels = 0;
  build_nodes(T, h, 0, M, 0);
  T.n_nodes = (int)T.nodes.size();
  T.pos.assign(M, 0);
  for (int k = 0; k < M; ++k) T.pos[T.perm[k]] = k;
  std::vector<int> leaf(M, -1);
  T.levels.assign(T.n_levels, {});
  for (int id = 0; id < T.n_nodes; ++id) {
    const TreeNodeH& nd = T.nodes[id];
    if (nd.count == 1) leaf[T.perm[nd.first]] = id;
    else T.levels[nd.level].push_back(id);
  }
  // per group: own and near particles (the far sum skips them for the
  // targets concerned; a multipole node may hold none of them)
  // groups never straddle particles (a group's bounding sphere is then a
  // part of one surface): each particle's G nodes in ceil(G / 256) runs of
  // nearly equal length
  const int chunks = (G + kTreeGroup - 1) / kTreeGroup;
  const int cs = (G + chunks - 1) / chunks;
  const int n_groups = M * chunks;
  T.n_groups = n_groups;
  std::vector<int2> groups(n_groups);
  for (int i = 0; i < M; ++i)
    for (int c = 0; c < chunks; ++c) {
      const int64_t t0 = (int64_t)i * G + (int64_t)c * cs;
      const int64_t t1 = std::min<int64_t>((int64_t)(i + 1) * G, t0 + cs);
      groups[(size_t)i * chunks + c] = make_int2((int)t0, (int)std::max(t0, t1));
    }
  auto group_of = [&](int64_t t) { return (int)((t / G) * chunks + (t % G) / cs); };
  std::vector<std::vector<int>> excl(n_groups);
  std::vector<std::vector<std::pair<int, int>>> excl_cnt(n_groups);   // (particle, targets of the group skipping it)
  for (int gi = 0; gi < n_groups; ++gi)
    for (int64_t t = groups[gi].x; t < groups[gi].y; ++t) excl[gi].push_back((int)(t / G));
  for (size_t k = 0; k < h.pair_t.size(); ++k) excl[group_of(h.pair_t[k])].push_back(h.pair_s[k]);
  for (int gi = 0; gi < n_groups; ++gi) {
    std::vector<int>& e = excl[gi];
    std::sort(e.begin(), e.end());
    for (size_t k = 0; k < e.size();) {
      size_t j = k;
      while (j < e.size() && e[j] == e[k]) ++j;
      excl_cnt[gi].push_back({e[k], (int)(j - k)});
      k = j;
    }
    e.erase(std::unique(e.begin(), e.end()), e.end());
  }
  const int tiles_per_part = (G + kFarTile - 1) / kFarTile;
  std::vector<int4> dtiles, ditems, mitems[2];
  std::vector<int> mlist[2];
  T.m2p_pairs = T.direct_pairs = T.m2p_source_pairs = 0;
  std::vector<int> stack, dlist, epos, accepted;
  std::vector<int> cls[2][3];   // accepted nodes of a group by operator and evaluation order 8, 12, 16
  const double worst = std::pow(T.theta, T.order + 1);
  const double margin[2] = {1.0, 0.1};
  for (auto& L : T.ev_lists)
    for (int64_t& v : L.evals_by_order) v = 0;
  for (int gi = 0; gi < n_groups; ++gi) {
    const int64_t t0 = groups[gi].x, t1 = groups[gi].y;
    if (t1 <= t0) continue;
    double bmin[3] = {1e300, 1e300, 1e300}, bmax[3] = {-1e300, -1e300, -1e300};
    for (int64_t t = t0; t < t1; ++t)
      for (int c = 0; c < 3; ++c) {
        bmin[c] = std::min(bmin[c], h.xyz[t * 3 + c]);
        bmax[c] = std::max(bmax[c], h.xyz[t * 3 + c]);
      }
    double cg[3], rg = 0.0;
    for (int c = 0; c < 3; ++c) cg[c] = 0.5 * (bmin[c] + bmax[c]);
    for (int64_t t = t0; t < t1; ++t) {
      double d2 = 0.0;
      for (int c = 0; c < 3; ++c) d2 += (h.xyz[t * 3 + c] - cg[c]) * (h.xyz[t * 3 + c] - cg[c]);
      rg = std::max(rg, std::sqrt(d2));
    }
    epos.clear();
    for (int e : excl[gi]) epos.push_back(T.pos[e]);
    std::sort(epos.begin(), epos.end());
    dlist.clear();
    accepted.clear();
    for (auto& op : cls)
      for (auto& v : op) v.clear();
    stack.assign(1, 0);
    while (!stack.empty()) {
      const int id = stack.back();
      stack.pop_back();
      const TreeNodeH& nd = T.nodes[id];
      const double dist = std::sqrt((nd.c[0] - cg[0]) * (nd.c[0] - cg[0]) + (nd.c[1] - cg[1]) * (nd.c[1] - cg[1]) +
                                    (nd.c[2] - cg[2]) * (nd.c[2] - cg[2]));
      const auto it = std::lower_bound(epos.begin(), epos.end(), nd.first);
      const bool holds_excluded = it != epos.end() && *it < nd.first + nd.count;
      if (!holds_excluded && dist >= rg + nd.r / T.theta) {
        const double rho = nd.r / (dist - rg);
        accepted.push_back(id);
        for (int op = 0; op < 2; ++op) {
          int c = 0;
          while (8 + 4 * c < T.order && std::pow(rho, 9 + 4 * c) > margin[op] * worst) ++c;
          cls[op][c].push_back(id);
        }
      } else if (nd.count == 1) {
        dlist.push_back(T.perm[nd.first]);
      } else {
        stack.push_back(nd.child[1]);
        stack.push_back(nd.child[0]);
      }
    }
    for (int op = 0; op < 2; ++op)
      for (int c = 0; c < 3; ++c) {
        std::vector<int>& ml = mlist[op];
        const size_t k0 = ml.size();
        ml.insert(ml.end(), cls[op][c].begin(), cls[op][c].end());
        for (size_t k = k0; k < ml.size(); k += kTreeChunkNodes)
          mitems[op].push_back(make_int4(gi, (int)k, (int)std::min(ml.size(), k + kTreeChunkNodes), c));
        T.ev_lists[op].evals_by_order[c] += (int64_t)cls[op][c].size() * (t1 - t0);
      }
    T.m2p_pairs += (int64_t)accepted.size() * (t1 - t0);
    for (int id : accepted) T.m2p_source_pairs += (int64_t)T.nodes[id].count * G * (t1 - t0);
    // direct list in ascending particle order (the kernel's skip-list walk needs it)
    std::sort(dlist.begin(), dlist.end());
    const int d0 = (int)dtiles.size();
    for (int i : dlist) {
      for (int k = 0; k < tiles_per_part; ++k) dtiles.push_back(h.tiles[(size_t)i * tiles_per_part + k]);
      const auto ec = std::lower_bound(excl_cnt[gi].begin(), excl_cnt[gi].end(), std::make_pair(i, -1));
      const int skipped = (ec != excl_cnt[gi].end() && ec->first == i) ? ec->second : 0;
      T.direct_pairs += (int64_t)((t1 - t0) - skipped) * G;
    }
    for (int k = d0; k < (int)dtiles.size(); k += kTreeChunkTiles)
      ditems.push_back(make_int4(gi, k, std::min((int)dtiles.size(), k + kTreeChunkTiles), 0));
  }
  T.m2p_entries = (int64_t)mlist[0].size();
  T.direct_tiles = (int64_t)dtiles.size();
  // longest items first (the tail of the grid is then short), within each order class
  std::stable_sort(ditems.begin(), ditems.end(), [](const int4& a, const int4& b) { return a.z - a.y > b.z - b.y; });
  for (int op = 0; op < 2; ++op) {
    std::vector<int4>& mi = mitems[op];
    std::stable_sort(mi.begin(), mi.end(), [](const int4& a, const int4& b) {
      return a.w != b.w ? a.w < b.w : a.z - a.y > b.z - b.y;
    });
    for (int c = 0; c <= 3; ++c)
      T.ev_lists[op].off[c] =
          (int)(std::lower_bound(mi.begin(), mi.end(), c, [](const int4& a, int cc) { return a.w < cc; }) - mi.begin());
  }
  // device tables
  std::vector<double> geo(T.n_nodes * 4);
  std::vector<float4> c32(T.n_nodes * 2);
  std::vector<int> child(T.n_nodes * 2), lev;
  for (int id = 0; id < T.n_nodes; ++id) {
    const TreeNodeH& nd = T.nodes[id];
    float hi[3], lo[3];
    for (int c = 0; c < 3; ++c) {
      geo[id * 4 + c] = nd.c[c];
      split_f32(nd.c[c], hi[c], lo[c]);
    }
    geo[id * 4 + 3] = nd.r;
    c32[id * 2 + 0] = make_float4(hi[0], hi[1], hi[2], 0.f);
    c32[id * 2 + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    child[id * 2 + 0] = nd.child[0];
    child[id * 2 + 1] = nd.child[1];
  }
  // translations only where a list reads the result: a node is needed if it
  // is accepted somewhere or lies below an accepted node (nodes come in
  // depth-first pre-order, so a parent precedes its children); the top
  // levels, whose nodes are too large to be accepted, are skipped
  std::vector<char> needed(T.n_nodes, 0);
  for (int id : mlist[0]) needed[id] = 1;
  for (int id = 0; id < T.n_nodes; ++id)
    if (needed[id])
      for (int c : T.nodes[id].child)
        if (c >= 0) needed[c] = 1;
  T.n_translated = 0;
  T.level_off.assign(1, 0);
  for (int l = T.n_levels - 1; l >= 0; --l) {   // deepest level first
    for (int id : T.levels[l])
      if (needed[id]) {
        lev.push_back(id);
        ++T.n_translated;
      }
    T.level_off.push_back((int)lev.size());
  }
  const int NM = tree_nm(T.order);
  int rc;
  if ((rc = upload_vec(g, T, &T.d_geo, geo, "tree nodes", st))) return rc;
  if ((rc = upload_vec(g, T, &T.d_c32, c32, "tree centres", st))) return rc;
  if ((rc = upload_vec(g, T, &T.d_child, child, "tree children", st))) return rc;
  if ((rc = upload_vec(g, T, &T.d_leaf, leaf, "tree leaves", st))) return rc;
  if ((rc = upload_vec(g, T, &T.d_levels, lev, "tree levels", st))) return rc;
  if ((rc = upload_vec(g, T, &T.d_groups, groups, "tree target groups", st))) return rc;
  if ((rc = upload_vec(g, T, &T.d_tiles, dtiles, "tree direct tiles", st))) return rc;
  if ((rc = upload_vec(g, T, &T.d_ditems, ditems, "tree direct items", st))) return rc;
  for (int op = 0; op < 2; ++op) {
    if ((rc = upload_vec(g, T, &T.ev_lists[op].d_mlist, mlist[op], "tree multipole lists", st))) return rc;
    if ((rc = upload_vec(g, T, &T.ev_lists[op].d_mitems, mitems[op], "tree multipole items", st))) return rc;
  }
  T.n_ditems = (int)ditems.size();
  if ((rc = dev_alloc(g, (void**)&T.d_M, sizeof(double2) * 2 * NM * (size_t)T.n_nodes, "tree multipoles"))) return rc;
  if ((rc = dev_alloc(g, (void**)&T.d_M32, sizeof(float2) * 2 * NM * (size_t)T.n_nodes, "tree multipoles (FP32)")))
    return rc;
  if ((rc = dev_alloc(g, (void**)&T.d_SM, sizeof(double2) * 8 * NM * (size_t)T.n_nodes, "tree Stokes multipoles")))
    return rc;
  if ((rc = dev_alloc(g, (void**)&T.d_SM32, sizeof(float2) * 8 * NM * (size_t)T.n_nodes,
                      "tree Stokes multipoles (FP32)")))
    return rc;
  return SBIO_OK;
}

template <int PF>
static int tree_apply(sbio_geom* g, TreeFar& T, double* S, double* D, cudaStream_t st) {
  const GeomHost& h = g->h;
  const DevGeom& d = g->d;
  constexpr int NM = tree_nm(PF);
  const bool timed = g->timing && T.ev[0];
  if (timed) cudaEventRecord(T.ev[0], st);
  // untimed: the direct part first, on the side stream, beside the multipole
  // phases (both add into S and D atomically)
  SideFork sf;
  const bool forked = !timed && T.side && g->overlap;
  if (forked) {
    SBIO_CUDA_TRY(sf.fork_on(st, T.side, T.side_fork, T.side_join));
    launch_far_tile_items(d, T.d_groups, T.d_tiles, T.d_ditems, T.n_ditems, S, D, T.side);
  }
  tree_p2m_kernel<PF, 0><<<h.M, 32 * kP2MWarps, 0, st>>>(h.G, d.src32, T.d_leaf, T.d_M);
  count_launch();
  if (timed) cudaEventRecord(T.ev[1], st);
  for (size_t l = 0; l + 1 < T.level_off.size(); ++l) {
    const int n = T.level_off[l + 1] - T.level_off[l];
    if (n <= 0) continue;
    const dim3 grid((unsigned)n, (unsigned)((2 * NM + kM2MThreads - 1) / kM2MThreads));
    tree_m2m_kernel<PF><<<grid, kM2MThreads, 0, st>>>(T.d_levels + T.level_off[l], T.d_child, T.d_geo, T.d_M, 0, 0);
    count_launch();
  }
  const int64_t total = (int64_t)T.n_nodes * 2 * NM;
  tree_to_f32_kernel<PF><<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(total, T.d_M, T.d_M32);
  count_launch();
  if (timed) cudaEventRecord(T.ev[2], st);
  if (!forked) launch_far_tile_items(d, T.d_groups, T.d_tiles, T.d_ditems, T.n_ditems, S, D, st);
  if (timed) cudaEventRecord(T.ev[3], st);
  // the evaluations, one launch per evaluation order (8, 12, 16 up to PF)
  const TreeFar::EvalLists& L = T.ev_lists[0];
  auto m2p = [&](auto pe, int c) {
    constexpr int PE = decltype(pe)::value;
    const int n = L.off[c + 1] - L.off[c];
    if (n <= 0) return;
    tree_m2p_kernel<PF, PE><<<n, kFarTile, 0, st>>>(L.d_mitems + L.off[c], T.d_groups, L.d_mlist, T.d_c32, T.d_M32,
                                                    d.tgt32, S, D);
    count_launch();
  };
  m2p(std::integral_constant<int, 8>(), 0);
  if constexpr (PF >= 12) m2p(std::integral_constant<int, 12>(), 1);
  if constexpr (PF >= 16) m2p(std::integral_constant<int, 16>(), 2);
  if (timed) cudaEventRecord(T.ev[4], st);
  SBIO_CUDA_TRY(cudaGetLastError());
  SBIO_CUDA_TRY(sf.join());
  return SBIO_OK;
}

// Builds and attaches a treecode to a geometry that has none, uploading its
// lists in order on `st` without synchronising the device (used by the
// serving engine, whose other slots keep running meanwhile).
int tree_attach_async(sbio_geom* g, int order, double theta, cudaStream_t st) {
  if (g->tree) return set_error(SBIO_EINVAL, "the geometry already has a treecode");
  TreeFar* t = new TreeFar();
  t->order = order;
  t->theta = theta;
  int rc = SBIO_OK;
  for (cudaEvent_t& e : t->ev)
    if (!rc && cudaEventCreate(&e) != cudaSuccess) rc = set_error(SBIO_ECUDA, "treecode event creation failed");
  if (!rc) rc = build_tree(g, *t, st);
  if (rc) {
    delete t;
    return rc;
  }
  g->tree = t;
  return SBIO_OK;
}

template <int PF>
static int tree_apply_stokes(sbio_geom* g, TreeFar& T, double* u, cudaStream_t st) {
  const GeomHost& h = g->h;
  const DevGeom& d = g->d;
  constexpr int NM = tree_nm(PF);
  const int64_t plane = (int64_t)T.n_nodes * 2 * NM;
  const bool timed = g->timing && T.ev[0];
  if (timed) cudaEventRecord(T.ev[0], st);
  SideFork sf;   // the direct part beside the multipole phases, as for Laplace
  const bool forked = !timed && T.side && g->overlap;
  if (forked) {
    SBIO_CUDA_TRY(sf.fork_on(st, T.side, T.side_fork, T.side_join));
    launch_stokes_far_tile_items(d, T.d_groups, T.d_tiles, T.d_ditems, T.n_ditems, u, T.side);
  }
  tree_p2m_kernel<PF, 1><<<h.M, 32 * kP2MWarps, 0, st>>>(h.G, d.st_src32, T.d_leaf, T.d_SM + 0 * plane);
  tree_p2m_kernel<PF, 2><<<h.M, 32 * kP2MWarps, 0, st>>>(h.G, d.st_src32, T.d_leaf, T.d_SM + 1 * plane);
  tree_p2m_kernel<PF, 3><<<h.M, 32 * kP2MWarps, 0, st>>>(h.G, d.st_src32, T.d_leaf, T.d_SM + 2 * plane);
  tree_p2m_kernel<PF, 4><<<h.M, 32 * kP2MWarps, 0, st>>>(h.G, d.st_src32, T.d_leaf, T.d_SM + 3 * plane);
  count_launch(4);
  if (timed) cudaEventRecord(T.ev[1], st);
  for (size_t l = 0; l + 1 < T.level_off.size(); ++l) {
    const int n = T.level_off[l + 1] - T.level_off[l];
    if (n <= 0) continue;
    const dim3 grid((unsigned)n, (unsigned)((2 * NM + kM2MThreads - 1) / kM2MThreads), 4);
    tree_m2m_kernel<PF><<<grid, kM2MThreads, 0, st>>>(T.d_levels + T.level_off[l], T.d_child, T.d_geo, T.d_SM, plane,
                                                      1);
    count_launch();
  }
  const int64_t total = 4 * plane;
  tree_to_f32_kernel<PF><<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(total, T.d_SM,
                                                                                                 T.d_SM32);
  count_launch();
  if (timed) cudaEventRecord(T.ev[2], st);
  if (!forked) launch_stokes_far_tile_items(d, T.d_groups, T.d_tiles, T.d_ditems, T.n_ditems, u, st);
  if (timed) cudaEventRecord(T.ev[3], st);
  const TreeFar::EvalLists& L = T.ev_lists[1];
  auto m2p = [&](auto pe, int c) {
    constexpr int PE = decltype(pe)::value;
    const int n = L.off[c + 1] - L.off[c];
    if (n <= 0) return;
    tree_m2p_stokes_kernel<PF, PE><<<n, kFarTile, 0, st>>>(L.d_mitems + L.off[c], T.d_groups, L.d_mlist, T.d_c32,
                                                           T.d_SM32, plane, d.tgt32, u);
    count_launch();
  };
  m2p(std::integral_constant<int, 8>(), 0);
  if constexpr (PF >= 12) m2p(std::integral_constant<int, 12>(), 1);
  if constexpr (PF >= 16) m2p(std::integral_constant<int, 16>(), 2);
  if (timed) cudaEventRecord(T.ev[4], st);
  SBIO_CUDA_TRY(cudaGetLastError());
  SBIO_CUDA_TRY(sf.join());
  return SBIO_OK;
}

int launch_tree_stokes_far(sbio_geom* g, double* u, cudaStream_t st) {
  TreeFar& T = *g->tree;
  switch (T.order) {
    case 8: return tree_apply_stokes<8>(g, T, u, st);
    case 12: return tree_apply_stokes<12>(g, T, u, st);
    default: return tree_apply_stokes<16>(g, T, u, st);
  }
}

int launch_tree_far(sbio_geom* g, double* S, double* D, cudaStream_t st) {
  TreeFar& T = *g->tree;
  switch (T.order) {
    case 8: return tree_apply<8>(g, T, S, D, st);
    case 12: return tree_apply<12>(g, T, S, D, st);
    default: return tree_apply<16>(g, T, S, D, st);
  }
}

}  // namespace sbio

using namespace sbio;

extern "C" {

int sbio_geom_set_far_method(sbio_geom* g, int32_t method, double theta, int32_t order) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (method == SBIO_FAR_DIRECT) {
    if (g->tree) {
      cudaSetDevice(g->ctx->device);
      cudaDeviceSynchronize();   // no apply may still read the lists being dropped
      tree_free(g->tree);
      g->tree = nullptr;
    }
    return SBIO_OK;
  }
  if (method != SBIO_FAR_TREE) return set_error(SBIO_EINVAL, "far method %d unknown", method);
  if (!(theta > 0.05 && theta < 1.0)) return set_error(SBIO_EINVAL, "theta = %g must be in (0.05, 1)", theta);
  if (order != 8 && order != 12 && order != 16)
    return set_error(SBIO_EINVAL, "treecode order %d: 8, 12 or 16", order);
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  SBIO_CUDA_TRY(cudaDeviceSynchronize());
  // a new setting rebuilds the lists (their device arrays stay with the
  // geometry until it is destroyed)
  TreeFar* t = new TreeFar();
  t->order = order;
  t->theta = theta;
  int rc = SBIO_OK;
  for (cudaEvent_t& e : t->ev)
    if (!rc && cudaEventCreate(&e) != cudaSuccess) rc = set_error(SBIO_ECUDA, "treecode event creation failed");
  if (!rc && g->overlap &&
      (cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking) != cudaSuccess ||
       cudaEventCreateWithFlags(&t->side_fork, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&t->side_join, cudaEventDisableTiming) != cudaSuccess))
    rc = set_error(SBIO_ECUDA, "treecode stream creation failed");
  if (!rc) rc = build_tree(g, *t, nullptr);
  if (!rc && cudaStreamSynchronize(nullptr) != cudaSuccess) rc = set_error(SBIO_ECUDA, "treecode upload failed");
  if (rc) {
    delete t;
    return rc;
  }
  tree_free(g->tree);
  g->tree = t;
  // the near kernels' CTA cap beside the treecode's phases, by whole applies
  // of zero densities (the apply writes finite sources first)
  if (g->overlap && g->near_stream && !g->timing && !g->h.pair_t.empty()) {
    const size_t nc = (size_t)(g->h.p + 1) * (g->h.p + 1) * g->h.M;
    SBIO_CUDA_TRY(cudaMemsetAsync(g->d.host_in, 0, 2 * nc * sizeof(double), nullptr));
    TuneOps ops;
    ops.far = nullptr;
    ops.whole = [](sbio_geom* gg, double* out, cudaStream_t s) {
      const size_t n = (size_t)(gg->h.p + 1) * (gg->h.p + 1) * gg->h.M;
      return launch_laplace(gg, gg->d.host_in, gg->d.host_in + n, out, out + gg->h.N, SBIO_PART_ALL, s);
    };
    ops.tt = nullptr;
    ops.splits = nullptr;
    ops.cap = &g->h.tree_near_ctas_per_sm;
    rc = tune_near_cap(g, ops, g->d.host_out, nullptr);
    if (!rc && cudaStreamSynchronize(nullptr) != cudaSuccess) rc = set_error(SBIO_ECUDA, "near cap tuning failed");
    if (rc) return rc;
  }
  return SBIO_OK;
}

int sbio_geom_set_tree_near_cap(sbio_geom* g, int32_t ctas_per_sm) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (ctas_per_sm < 0) return set_error(SBIO_EINVAL, "ctas_per_sm must be >= 0");
  g->h.tree_near_ctas_per_sm = ctas_per_sm;
  return SBIO_OK;
}

int sbio_geom_get_tree_near_cap(const sbio_geom* g, int32_t* ctas_per_sm) {
  clear_error();
  if (!g || !ctas_per_sm) return set_error(SBIO_EINVAL, "null argument");
  *ctas_per_sm = g->h.tree_near_ctas_per_sm;
  return SBIO_OK;
}

int sbio_geom_tree_phase_times(sbio_geom* g, double* ms) {
  clear_error();
  if (!g || !ms) return set_error(SBIO_EINVAL, "null argument");
  if (!g->tree) return set_error(SBIO_EINVAL, "the geometry's far field is the direct sum");
  if (!g->timing) return set_error(SBIO_EINVAL, "phase timing is off (sbio_geom_enable_timing)");
  SBIO_CUDA_TRY(cudaEventSynchronize(g->tree->ev[4]));
  for (int k = 0; k < 4; ++k) {
    float t = 0.f;
    SBIO_CUDA_TRY(cudaEventElapsedTime(&t, g->tree->ev[k], g->tree->ev[k + 1]));
    ms[k] = t;
  }
  return SBIO_OK;
}

int sbio_geom_tree_order_counts(const sbio_geom* g, int32_t op, int64_t* evals) {
  clear_error();
  if (!g || !evals) return set_error(SBIO_EINVAL, "null argument");
  if (op != SBIO_OP_LAPLACE && op != SBIO_OP_STOKES) return set_error(SBIO_EINVAL, "operator %d unknown", op);
  if (!g->tree) return set_error(SBIO_EINVAL, "the geometry's far field is the direct sum");
  const TreeFar::EvalLists& L = g->tree->ev_lists[op == SBIO_OP_STOKES ? 1 : 0];
  for (int c = 0; c < 3; ++c) evals[c] = L.evals_by_order[c];
  return SBIO_OK;
}

int sbio_geom_tree_info(const sbio_geom* g, int64_t* n_nodes, int64_t* n_groups, int64_t* m2p_pairs,
                        int64_t* m2p_source_pairs, int64_t* direct_pairs) {
  clear_error();
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (!g->tree) return set_error(SBIO_EINVAL, "the geometry's far field is the direct sum");
  if (n_nodes) *n_nodes = g->tree->n_nodes;
  if (n_groups) *n_groups = g->tree->n_groups;
  if (m2p_pairs) *m2p_pairs = g->tree->m2p_pairs;
  if (m2p_source_pairs) *m2p_source_pairs = g->tree->m2p_source_pairs;
  if (direct_pairs) *direct_pairs = g->tree->direct_pairs;
  return SBIO_OK;
}

}  // extern "C"
