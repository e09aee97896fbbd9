// Particle-to-target evaluation (Sec. 4.1, "Particle-to-target algorithm"):
// S[sigma] and D[mu] of every spheroid at arbitrary points in the fluid.
//
// Creation uploads the point coordinates (FP64 and hi/lo FP32) and classifies
// each (point, spheroid) pair on the device by the exact point-to-surface
// distance (near iff below near_factor x major semi-axis, the rule used for
// surface nodes), with the geometry's near-set kernel: the near pairs (sorted
// by source kind, source, point) and the per-point skip lists of near
// spheroids.  Evaluation reuses the
// geometry's kernels through a view of its device tables in which the
// targets are the points: the synthesis kernel writes the far sources and
// near coefficients of the given densities (no self output: no point lies on
// a surface in the sense of the self term), the near kernel evaluates the
// exterior expansions at the near pairs and the far kernel sums the smooth
// quadrature over all other spheroids.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sbio_internal.cuh"

struct sbio_targets {
  sbio_geom* g = nullptr;
  int64_t T = 0;
  int64_t n_pro = 0, n_pairs = 0, far_pairs = 0;
  // the geometry's tables with the points as targets: xyz, tgt32, the near
  // pairs and the skip lists are the points'; nrm is null (points carry no
  // normal), so kernels that need source normals take them from the geometry
  sbio::DevGeom view;
  std::vector<void*> allocs;
  size_t bytes = 0;
};

namespace sbio {

static int ts_alloc(sbio_targets* ts, void** ptr, size_t bytes, const char* what) {
  *ptr = nullptr;
  if (bytes == 0) return SBIO_OK;
  sbio_ctx* c = ts->g->ctx;
  const size_t prev = c->used.fetch_add(bytes);
  if (c->budget && prev + bytes > c->budget) {
    c->used.fetch_sub(bytes);
    return set_error(SBIO_ENOMEM, "device budget exceeded allocating %s (%zu bytes)", what, bytes);
  }
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->used.fetch_sub(bytes);
    *ptr = nullptr;
    return set_error(SBIO_ENOMEM, "cudaMalloc of %s (%zu bytes) failed", what, bytes);
  }
  ts->allocs.push_back(*ptr);
  ts->bytes += bytes;
  return SBIO_OK;
}

template <typename T>
static int ts_upload(sbio_targets* ts, T** dst, const T* src, size_t count, const char* what, cudaStream_t st) {
  int rc = ts_alloc(ts, (void**)dst, count * sizeof(T), what);
  if (rc) return rc;
  if (count) SBIO_CUDA_TRY(cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, st));
  return SBIO_OK;
}

static void ts_free(sbio_targets* ts) {
  for (void* p : ts->allocs) cudaFree(p);
  if (ts->g) ts->g->ctx->used.fetch_sub(ts->bytes);
  ts->allocs.clear();
  ts->bytes = 0;
}

// Processing order of the points for the near-set kernel: a counting sort by
// cell of a 32 x 32 x 32 grid over the points' bounding box, so that the
// threads of a warp hold nearby points (alike candidate spheroids).
static void spatial_order(const double* xyz, int64_t T, std::vector<int32_t>& order) {
  constexpr int kCells = 32;
  double lo[3] = {xyz[0], xyz[1], xyz[2]}, hi[3] = {xyz[0], xyz[1], xyz[2]};
  for (int64_t t = 1; t < T; ++t)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], xyz[t * 3 + c]);
      hi[c] = std::max(hi[c], xyz[t * 3 + c]);
    }
  double sc[3];
  for (int c = 0; c < 3; ++c) sc[c] = hi[c] > lo[c] ? (kCells - 1e-9) / (hi[c] - lo[c]) : 0.0;
  std::vector<int32_t> cell(T);
  std::vector<int64_t> start(kCells * kCells * kCells + 1, 0);
  for (int64_t t = 0; t < T; ++t) {
    int q[3];
    for (int c = 0; c < 3; ++c) q[c] = std::min(kCells - 1, std::max(0, (int)((xyz[t * 3 + c] - lo[c]) * sc[c])));
    cell[t] = (q[2] * kCells + q[1]) * kCells + q[0];
    start[cell[t] + 1]++;
  }
  for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
  order.assign(T, 0);
  for (int64_t t = 0; t < T; ++t) order[start[cell[t]]++] = (int32_t)t;
}

int targets_view(sbio_targets* ts, sbio_geom** g, const DevGeom** view, int64_t* T, int64_t* n_pro,
                 int64_t* n_pairs) {
  if (!ts) return set_error(SBIO_EINVAL, "null target set");
  *g = ts->g;
  *view = &ts->view;
  *T = ts->T;
  *n_pro = ts->n_pro;
  *n_pairs = ts->n_pairs;
  return SBIO_OK;
}

}  // namespace sbio

using namespace sbio;

extern "C" {

int sbio_targets_create(sbio_geom* g, const double* xyz_host, int64_t T, void* stream, sbio_targets** out) {
  clear_error();
  if (!g || !out || (T > 0 && !xyz_host)) return set_error(SBIO_EINVAL, "null argument");
  *out = nullptr;
  if (T < 0 || T > (int64_t)INT32_MAX / 2) return set_error(SBIO_EINVAL, "bad number of points %lld", (long long)T);
  for (int64_t k = 0; k < 3 * T; ++k)
    if (!std::isfinite(xyz_host[k])) return set_error(SBIO_EINVAL, "point %lld is not finite", (long long)(k / 3));
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const GeomHost& h = g->h;
  sbio_targets* ts = new sbio_targets();
  ts->g = g;
  ts->T = T;
  ts->view = g->d;
  std::vector<float4> tgt(T * 2);
  for (int64_t t = 0; t < T; ++t) {
    float hi[3], lo[3];
    for (int c = 0; c < 3; ++c) split_f32(xyz_host[t * 3 + c], hi[c], lo[c]);
    tgt[t * 2 + 0] = make_float4(hi[0], hi[1], hi[2], 0.f);
    tgt[t * 2 + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
  }
  DevGeom& v = ts->view;
  int rc = SBIO_OK;
  if (!rc) rc = ts_upload(ts, &v.xyz, xyz_host, (size_t)T * 3, "target points", st);
  if (!rc) rc = ts_upload(ts, &v.tgt32, tgt.data(), tgt.size(), "target points (fp32)", st);
  // near pairs and skip lists on the device; a point inside a spheroid (the
  // ellipsoid form below 1 - 1e-11, so that points on a surface are outside)
  // is refused
  std::vector<int32_t> pt, ps, cnt;
  int64_t inside = -1;
  if (!rc) {
    auto alloc_skip = [&](const std::vector<int32_t>& sptr, int32_t** sp, int32_t** si) -> int {
      int r = ts_upload(ts, &v.skip_ptr, sptr.data(), sptr.size(), "target skip lists", st);
      if (!r) r = ts_alloc(ts, (void**)&v.skip_idx, (size_t)sptr.back() * sizeof(int32_t), "target skip lists");
      *sp = v.skip_ptr;
      *si = v.skip_idx;
      return r;
    };
    std::vector<int32_t> order;
    if (T > 0) spatial_order(xyz_host, T, order);
    rc = device_near_sets(g, v.xyz, T, 0, 1e-11, T > 0 ? &order : nullptr, st, alloc_skip, pt, ps, &ts->n_pro, cnt,
                          &inside);
    if (rc == SBIO_EINVAL && inside >= 0) rc = set_error(SBIO_EINVAL, "point %lld lies inside a spheroid", (long long)inside);
  }
  ts->n_pairs = (int64_t)pt.size();
  ts->far_pairs = (T * (int64_t)h.M - ts->n_pairs) * h.G;
  if (!rc) rc = ts_upload(ts, &v.pair_t, pt.data(), pt.size(), "target near pairs", st);
  if (!rc) rc = ts_upload(ts, &v.pair_s, ps.data(), ps.size(), "target near pairs", st);
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = set_error(SBIO_ECUDA, "target upload failed");
  if (rc) {
    ts_free(ts);
    delete ts;
    return rc;
  }
  v.nrm = nullptr;   // points carry no normal
  v.near_grid_cap = 0;
  g->n_target_sets.fetch_add(1);
  *out = ts;
  return SBIO_OK;
}

int sbio_targets_destroy(sbio_targets* ts) {
  if (!ts) return SBIO_OK;
  cudaSetDevice(ts->g->ctx->device);
  cudaDeviceSynchronize();
  ts_free(ts);
  ts->g->n_target_sets.fetch_sub(1);
  delete ts;
  return SBIO_OK;
}

int sbio_targets_info(const sbio_targets* ts, int64_t* n_points, int64_t* n_near_pairs, int64_t* n_far_pairs,
                      size_t* device_bytes) {
  if (!ts) return set_error(SBIO_EINVAL, "null target set");
  if (n_points) *n_points = ts->T;
  if (n_near_pairs) *n_near_pairs = ts->n_pairs;
  if (n_far_pairs) *n_far_pairs = ts->far_pairs;
  if (device_bytes) *device_bytes = ts->bytes;
  return SBIO_OK;
}

int sbio_eval_targets(sbio_targets* ts, const double* sigma_tilde, const double* mu_hat, double* S_out,
                      double* D_out, void* stream) {
  clear_error();
  if (!ts) return set_error(SBIO_EINVAL, "null target set");
  if ((sigma_tilde == nullptr) != (S_out == nullptr) || (mu_hat == nullptr) != (D_out == nullptr))
    return set_error(SBIO_EINVAL, "each output must be given exactly when its input is");
  if (!sigma_tilde && !mu_hat) return set_error(SBIO_EINVAL, "nothing to evaluate");
  sbio_geom* g = ts->g;
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const GeomHost& h = g->h;
  if (ts->T == 0) return SBIO_OK;
  if (S_out) SBIO_CUDA_TRY(cudaMemsetAsync(S_out, 0, ts->T * sizeof(double), st));
  if (D_out) SBIO_CUDA_TRY(cudaMemsetAsync(D_out, 0, ts->T * sizeof(double), st));
  // far sources and near coefficients of these densities (no self output)
  int rc = launch_synth_mode(g, sigma_tilde, mu_hat, nullptr, nullptr, 0, st);
  if (rc) return rc;
  near_launcher nl = near_for_p(h.p);
  if (ts->n_pairs > 0 && !nl) return set_error(SBIO_ENOTSUP, "no near-field kernel for p = %d", h.p);
  // the FP64 near pairs run beside the FP32 far field on the geometry's
  // high-priority stream (capped CTAs per SM), as in the on-surface apply
  const bool fork = g->overlap && !g->timing && g->near_stream && ts->n_pairs > 0;
  SideFork sf;
  if (fork) {
    SBIO_CUDA_TRY(sf.fork(g, st));
    ts->view.near_grid_cap = h.near_ctas_per_sm > 0 ? h.near_ctas_per_sm * sm_count() : 0;
    nl(ts->view, ts->n_pro, ts->n_pairs, ts->view.inv, S_out, D_out, h.precision == SBIO_MIXED, g->near_stream);
    ts->view.near_grid_cap = 0;
    SBIO_CUDA_TRY(cudaGetLastError());
  } else if (ts->n_pairs > 0) {
    nl(ts->view, ts->n_pro, ts->n_pairs, ts->view.inv, S_out, D_out, h.precision == SBIO_MIXED, st);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  launch_far_on(ts->view, h, ts->T, S_out, D_out, st);
  SBIO_CUDA_TRY(cudaGetLastError());
  SBIO_CUDA_TRY(sf.join());
  return SBIO_OK;
}

}  // extern "C"
