// Host-side internal state of the library (context, geometry) and the kernel
// launch interface between the set-up code and the kernel translation units.
#pragma once

#include <atomic>
#include <cstdarg>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "sbio_common.cuh"

struct sbio_ctx {
  int device = 0;
  size_t budget = 0;                 // 0 = unbounded
  std::atomic<size_t> used{0};
  std::atomic<int> n_geoms{0};
};

namespace sbio {

constexpr int kFarTile = 128;        // sources per far-field tile (= threads per CTA)

// Per-apply device workspaces and per-geometry device tables.
struct DevGeom {
  PartGeom* parts = nullptr;     // M
  double* xyz = nullptr;         // N x 3 global node positions
  double* nrm = nullptr;         // N x 3 outward unit normals
  double* w = nullptr;           // N quadrature weights
  double* ptab = nullptr;        // (p+1) x nm_count(p): N_n^m Pbar_n^m(v_j)
  double* glw = nullptr;         // p+1 Gauss-Legendre weights of the v nodes
  double* trig = nullptr;        // n_phi x (p+1) x 2: cos(m phi_k), sin(m phi_k)
  double* sqrtw = nullptr;       // M x (p+1): sqrt(u0^2 + sgn v_j^2)
  double* mult = nullptr;        // M x 4 x nm_count(p): extS, extD, selfS, selfD
  double* dmult = nullptr;       // M x 4 x nm_count(p): extS, extD, S' (principal value), D' (d/du at u0)
  double* normc = nullptr;       // (p+1)^2: N_n^|m| (sqrt 2 for m != 0) per coefficient
  int32_t* pair_t = nullptr;     // near pairs: target node
  int32_t* pair_s = nullptr;     // near pairs: source particle
  int32_t* skip_ptr = nullptr;   // N+1 CSR of per-target skipped particles (own + near), ascending
  int32_t* skip_idx = nullptr;
  int4* tiles = nullptr;         // far source tiles (particle, first node, count, -)
  double* inv = nullptr;         // 1/k for k >= 1; entry 0 holds the table length (sized per geometry)
  int near_grid_cap = 0;         // > 0: at most this many near CTAs (grid-stride), set while overlapping
  int near_block = 128;          // threads per CTA of the S + D near kernel (64 or 128; tunable)
  float4* tgt32 = nullptr;       // N x 2: hi, lo parts of the global node position
  float4* cen32 = nullptr;       // M x 2: hi, lo parts of the centres
  // workspaces written by every apply
  double* src64 = nullptr;       // N x 8: y - c_own (3), q, d (3), 0
  float4* src32 = nullptr;       // N x 2: (y - c_own, q), (d, 0)
  double* alpha = nullptr;       // M x (p+1)^2 folded exterior S coefficients
  double* beta = nullptr;        // M x (p+1)^2 folded exterior D coefficients
  float* alpha32 = nullptr;      // M x (p+1)^2: sigma (the mixed near form's S coefficients)
  float* beta32 = nullptr;       // M x (p+1)^2: mu extD / extS (its D coefficients)
  double* host_in = nullptr;     // 2 x M x (p+1)^2 staging for the host-memory entry point
  double* host_out = nullptr;    // 2 x N
  // Stokes single layer (Sec. 4.3): tables, pairs and workspaces
  double* st_ext = nullptr;      // M x nm_count(p+1): exterior S factor up to order p+1
  double* st_normc = nullptr;    // (p+2)^2 normalisation up to order p+1
  double* st_qv = nullptr;       // n_q GL nodes of the y.f transform grid
  double* st_qw = nullptr;       // n_q GL weights
  double* st_qptab = nullptr;    // n_q x nm_count(p+1): N_n^m Pbar_n^m(v_q)
  double* st_qtrig = nullptr;    // n_f x (p+2) x 2: cos / sin (m phi_l)
  double* st_qu0 = nullptr;      // M x nm_count(p+1): q_n^m(u0) (self term)
  double* st_dqu0 = nullptr;     // M x nm_count(p+1): dq_n^m/du (u0)
  double* st_fP = nullptr;       // (p+1) x nm_count(p+1): Pbar_n^m(v_j), unnormalised
  double* st_fV = nullptr;       //   sqrt(1-v_j^2) dPbar/dv
  double* st_fF = nullptr;       //   m Pbar / sqrt(1-v_j^2)
  double* st_trig1 = nullptr;    // n_phi x (p+2) x 2: cos / sin (m phi_k), m <= p+1
  double* st_glv = nullptr;      // p+1 GL nodes v_j of the surface grid
  double* st_coef = nullptr;     // M x 4 x (p+2)^2 folded coefficients (f1, f2, f3, y.f)
  double* st_src64 = nullptr;    // N x 8: y - c_own (3), w f (3), 0, 0
  float4* st_src32 = nullptr;    // N x 2: (y - c_own, w f_1), (w f_2, w f_3, 0, 0)
  // Stokes double layer: exterior D factor to order p+1, FP32 normals, 13
  // folded expansions per particle (q_1..3, y_i q_j, q.nu)
  double* sdl_ext = nullptr;     // M x nm_count(p+1)
  float4* nrm32 = nullptr;       // N: outward normal (FP32)
  double* sdl_coef = nullptr;    // M x 13 x (p+2)^2
};

struct GeomHost {
  int M = 0, p = 0, n_v = 0, n_phi = 0, G = 0;
  int64_t N = 0;
  double near_factor = 1.0;
  int precision = SBIO_FP64;
  std::vector<PartGeom> parts;
  std::vector<double> xyz, nrm, w;
  std::vector<int32_t> pair_t, pair_s;   // sorted by (kind, source, target)
  int64_t n_pairs_prolate = 0;           // pairs [0, n_pairs_prolate) have prolate sources
  int64_t far_pairs = 0;
  std::vector<int4> tiles;
  int n_q = 0, n_f = 0;                      // y.f transform grid
  // launch shape of the far field (tunable): targets per thread of the mixed
  // kernel and number of source splits (0 = chosen from the device size)
  int far_tt = 2;
  int far_splits = 0;
  int near_block = 128;                      // threads per CTA of the near kernels
  int near_ctas_per_sm = 2;                  // near CTAs per SM while overlapping with the far field (0 = no cap)
  int tree_near_ctas_per_sm = 2;             // the same while the treecode computes the far field
  // the same three settings for the Stokes single layer (its own kernels)
  int st_far_tt = 2;
  int st_far_splits = 0;
  int st_near_ctas_per_sm = 0;
};

}  // namespace sbio

namespace sbio {
struct TreeFar;   // particle treecode far field (sbio_tree.cu)
void tree_free(TreeFar* t);
}  // namespace sbio

struct sbio_geom {
  sbio_ctx* ctx = nullptr;
  sbio::GeomHost h;
  sbio::DevGeom d;
  size_t bytes = 0;
  std::vector<void*> allocs;
  cudaStream_t setup_stream = nullptr;
  // optional phase timing: events recorded on the launch stream around the
  // synth, near and far phases of the last apply
  bool timing = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // stream-ordered allocation on setup_stream (used by the serving engine so
  // that creating / releasing one request's geometry does not synchronise the
  // device)
  bool async_alloc = false;
  // near/far overlap: the FP64 near kernels run on a high-priority stream
  // forked from the caller's stream, beside the FP32 far kernel
  bool overlap = true;
  double setup_ms[3] = {0.0, 0.0, 0.0};   // host geometry, near sets, device tables + upload
  cudaStream_t near_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::atomic<int> n_target_sets{0};       // live sbio_targets of this geometry
  // far field by the particle treecode instead of the direct sum (mixed
  // precision applies at the nodes only); null = direct
  sbio::TreeFar* tree = nullptr;
};

namespace sbio {

// error reporting (thread-local message)
int set_error(int code, const char* fmt, ...);
void clear_error();
void count_launch(int n = 1);
int64_t launch_counter();

// host set-up helpers shared by the translation units (defined in sbio_geom.cu)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void ferrers(double v, int N, double* P);
double kfact(int n, int m);
int validate(const sbio_spheroid* sph, int32_t M, const sbio_options* o);
int build_host(GeomHost& h, const sbio_spheroid* sph, int32_t M, const sbio_options* o);

// geometry creation / release with stream-ordered allocation on `st`
int geom_create_async(sbio_ctx* ctx, const sbio_spheroid* sph, int32_t M, const sbio_options* opts,
                      cudaStream_t st, sbio_geom** out);
void geom_destroy_async(sbio_geom* g, cudaStream_t st);

// device allocation tracked against the context budget
int dev_alloc(sbio_geom* g, void** ptr, size_t bytes, const char* what);

struct DevGeom;
// mixed: the FP32-contraction form (SBIO_MIXED geometries), else plain FP64
typedef void (*near_launcher)(const DevGeom&, int64_t, int64_t, const double*, double*, double*, bool, cudaStream_t);
near_launcher near_lookup_a(int p);
near_launcher near_lookup_b(int p);
near_launcher near_lookup_c(int p);
near_launcher near_lookup_d(int p);
inline near_launcher near_for_p(int p) {
  near_launcher f = near_lookup_a(p);
  if (!f) f = near_lookup_b(p);
  if (!f) f = near_lookup_c(p);
  if (!f) f = near_lookup_d(p);
  return f;
}

// Far-field view of one suspension for the persistent batched kernel.
struct FarDesc {
  const int4* tiles;
  const float4* src32;
  const float4* tgt32;
  const float4* cen32;
  const int32_t* skip_ptr;
  const int32_t* skip_idx;
  int64_t N;
  double* S;
  double* D;
};
int launch_far_persistent(const FarDesc* descs, const int4* items, int n_items, int* counter, int tt, int grid,
                          cudaStream_t st);
// Direct part of the treecode far field: items (target group, first tile,
// end tile) over a tile list, groups = [first, end) target ranges of at most
// 256 targets; the geometry's mixed far pair sum (2 packed targets per
// thread) with its skip lists; defined in sbio_laplace.cu.
void launch_far_tile_items(const DevGeom& d, const int2* groups, const int4* tiles, const int4* items, int n_items,
                           double* S, double* D, cudaStream_t st);
// the treecode far field of one apply (sbio_tree.cu)
int launch_tree_far(sbio_geom* g, double* S, double* D, cudaStream_t st);
// build and attach a treecode (order, theta) with its uploads ordered on st
int tree_attach_async(sbio_geom* g, int order, double theta, cudaStream_t st);
// the Stokes single layer's far field by the treecode (sbio_tree.cu) and its
// direct part (sbio_stokes.cu)
int launch_tree_stokes_far(sbio_geom* g, double* u, cudaStream_t st);
void launch_stokes_far_tile_items(const DevGeom& d, const int2* groups, const int4* tiles, const int4* items,
                                  int n_items, double* u, cudaStream_t st);

// record phase event k (0..3) when timing is enabled
inline void phase_mark(sbio_geom* g, int k, cudaStream_t st) {
  if (g->timing && g->ev[k]) cudaEventRecord(g->ev[k], st);
}

// Near-field work forked from the caller's stream onto the geometry's
// high-priority stream, joined back on every exit path: if an apply returns
// an error after the fork, the caller's stream still waits for the kernels
// already queued on the side stream, so the next call on that stream cannot
// overwrite the workspaces they read or race their atomic adds.
struct SideFork {
  cudaStream_t main = nullptr, side = nullptr;
  cudaEvent_t join_ev = nullptr;
  bool open = false;
  cudaError_t fork(sbio_geom* g, cudaStream_t caller) { return fork_on(caller, g->near_stream, g->ev_fork, g->ev_join); }
  cudaError_t fork_on(cudaStream_t caller, cudaStream_t to, cudaEvent_t fork_ev, cudaEvent_t join_with) {
    main = caller;
    side = to;
    join_ev = join_with;
    cudaError_t e = cudaEventRecord(fork_ev, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork_ev, 0);
    open = (e == cudaSuccess);
    return e;
  }
  cudaError_t join() {
    if (!open) return cudaSuccess;
    open = false;
    cudaError_t e = cudaEventRecord(join_ev, side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(main, join_ev, 0);
    return e;
  }
  ~SideFork() { join(); }
};

// kernel entry points (defined in the kernel translation units)
// side (on the own surface): 0 the principal value of D, +1 / -1 the exterior
// / interior limit D +- mu/2 (for S' in derivative mode: S' -+ sigma/2)
int launch_laplace(sbio_geom* g, const double* sigma, const double* mu, double* S, double* D,
                   uint32_t parts, cudaStream_t st, int side = 0);
int launch_synth(sbio_geom* g, const double* sigma, const double* mu, double* S, double* D, bool write_self,
                 cudaStream_t st);
// Near sets on the device for n targets at device positions xyz: the
// geometry's nodes (G nodes per particle) or points (G = 0); see sbio_geom.cu.
int device_near_sets(sbio_geom* g, const double* xyz, int64_t n, int G, double inside_tol,
                     const std::vector<int32_t>* order_host, cudaStream_t st,
                     const std::function<int(const std::vector<int32_t>&, int32_t**, int32_t**)>& alloc_skip,
                     std::vector<int32_t>& pair_t, std::vector<int32_t>& pair_s, int64_t* n_pro,
                     std::vector<int32_t>& cnt, int64_t* inside);

// A target set's view of its geometry: the geometry's device tables with the
// set's points as targets (xyz, tgt32, near pairs, skip lists; nrm null),
// the point count and the near pairs (the first n_pro on prolate sources).
int targets_view(sbio_targets* ts, sbio_geom** g, const DevGeom** view, int64_t* T, int64_t* n_pro,
                 int64_t* n_pairs);

int launch_synth_mode(sbio_geom* g, const double* sigma, const double* mu, double* S, double* D, int self_mode,
                      cudaStream_t st, int side = 0);
int launch_near(sbio_geom* g, double* S, double* D, cudaStream_t st);
int launch_stokes(sbio_geom* g, const double* f, double* u, cudaStream_t st);
// far field of the geometry's sources at the NT targets of `d` (d.xyz,
// d.tgt32, d.skip_ptr, d.skip_idx; the node targets of the geometry itself
// when d is g->d and NT = N), in the geometry's precision and launch shape
void launch_far_on(const DevGeom& d, const GeomHost& h, int64_t NT, double* S, double* D, cudaStream_t st);
// host geometry helpers shared by the set-up code
void split_f32(double v, float& hi, float& lo);
int launch_stokes_far(sbio_geom* g, double* u, cudaStream_t st);
int launch_stokes_far_on(const DevGeom& d, const GeomHost& h, int64_t NT, double* u, double* pr, cudaStream_t st);
int launch_stokes_prep(sbio_geom* g, const double* f, cudaStream_t st);
int launch_laplace_deriv(sbio_geom* g, const double* sigma, const double* mu, double* Sp, double* Dp,
                         cudaStream_t st, int side = 0);

// Launch-shape search shared by the Laplace and Stokes autotuners: times
// far(g, out, st) for every targets-per-thread form and a ladder of source
// splits (writing *tt / *splits before each launch), keeps the fastest, then,
// if whole(...) is given and the near field overlaps the far field, times
// whole applies for a few near CTA caps written to *cap.  `out` is the
// launch's output workspace.
struct TuneOps {
  int (*far)(sbio_geom* g, double* out, cudaStream_t st);
  int (*whole)(sbio_geom* g, double* out, cudaStream_t st);
  int* tt;
  int* splits;
  int* cap;
  int min_cap = 1;   // smallest near cap tried (besides uncapped)
};
int tune_launch_shape(sbio_geom* g, const TuneOps& ops, double* out, cudaStream_t st, double* best_far_ms);
// the near CTA cap alone (*ops.cap) by whole applies, with the far field as set
int tune_near_cap(sbio_geom* g, const TuneOps& ops, double* out, cudaStream_t st);

// source splits of the far-field grid (gridDim.y) for `target_blocks` target
// CTAs; `requested` > 0 forces the count
int far_split_count(int64_t target_blocks, int n_tiles, int requested);
int sm_count();   // multiprocessors of the current device (cached)

}  // namespace sbio

#define SBIO_CUDA_TRY(call)                                                                   \
  do {                                                                                        \
    cudaError_t err_ = (call);                                                                \
    if (err_ != cudaSuccess)                                                                  \
      return ::sbio::set_error(SBIO_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(err_), \
                               __FILE__, __LINE__);                                           \
  } while (0)
