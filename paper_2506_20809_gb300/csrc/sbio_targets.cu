// Particle-to-target evaluation (Sec. 4.1, "Particle-to-target algorithm"):
// S[sigma] and D[mu] of every spheroid at arbitrary points in the fluid.
//
// Creation classifies each (point, spheroid) pair on the host by the exact
// point-to-surface distance (near iff below near_factor x major semi-axis,
// the rule used for surface nodes), and uploads the point coordinates (FP64
// and hi/lo FP32), the near pairs (sorted by source kind, source, point) and
// the per-point skip lists of near spheroids.  Evaluation reuses the
// geometry's kernels through a view of its device tables in which the
// targets are the points: the synthesis kernel writes the far sources and
// near coefficients of the given densities (no self output: no point lies on
// a surface in the sense of the self term), the near kernel evaluates the
// exterior expansions at the near pairs and the far kernel sums the smooth
// quadrature over all other spheroids.
#include <algorithm>
#include <thread>
#include <utility>
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

// Per-point near spheroids; returns the index of a point inside a spheroid
// (or -1) through `inside_point`.
static void classify(const GeomHost& h, const double* xyz, int64_t T, std::vector<std::pair<int32_t, int32_t>>& pairs,
                     int64_t* inside_point, int* inside_part) {
  const int M = h.M;
  std::vector<double> rmax(M), thr(M);
  for (int i = 0; i < M; ++i) {
    rmax[i] = std::max(h.parts[i].A, h.parts[i].C);
    thr[i] = h.near_factor * rmax[i];
  }
  const unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::vector<std::pair<int32_t, int32_t>>> local(nth);
  std::vector<int64_t> bad_t(nth, -1);
  std::vector<int> bad_i(nth, -1);
  auto work = [&](unsigned tid) {
    for (int64_t t = tid; t < T; t += nth) {
      const double* x = xyz + t * 3;
      for (int i = 0; i < M; ++i) {
        const PartGeom& P = h.parts[i];
        const double d0 = x[0] - P.c[0], d1 = x[1] - P.c[1], d2 = x[2] - P.c[2];
        const double dc = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        if (dc - rmax[i] >= thr[i]) continue;
        const double xl = P.R[0] * d0 + P.R[3] * d1 + P.R[6] * d2;
        const double yl = P.R[1] * d0 + P.R[4] * d1 + P.R[7] * d2;
        const double zl = P.R[2] * d0 + P.R[5] * d1 + P.R[8] * d2;
        bool inside = false;
        const double d = spheroid_distance_local(P, xl, yl, zl, 1e-11, &inside);
        if (inside) {
          bad_t[tid] = t;
          bad_i[tid] = i;
          return;
        }
        if (d < thr[i]) local[tid].push_back({(int32_t)t, (int32_t)i});
      }
    }
  };
  std::vector<std::thread> th;
  for (unsigned k = 0; k < nth; ++k) th.emplace_back(work, k);
  for (auto& t : th) t.join();
  *inside_point = -1;
  for (unsigned k = 0; k < nth; ++k)
    if (bad_t[k] >= 0) {
      *inside_point = bad_t[k];
      *inside_part = bad_i[k];
      return;
    }
  pairs.clear();
  for (auto& v : local) pairs.insert(pairs.end(), v.begin(), v.end());
  std::sort(pairs.begin(), pairs.end(), [&](const std::pair<int32_t, int32_t>& a, const std::pair<int32_t, int32_t>& b) {
    const int ka = h.parts[a.second].kind, kb = h.parts[b.second].kind;
    if (ka != kb) return ka < kb;
    if (a.second != b.second) return a.second < b.second;
    return a.first < b.first;
  });
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
  std::vector<std::pair<int32_t, int32_t>> pairs;
  int64_t bad = -1;
  int bad_i = -1;
  classify(h, xyz_host, T, pairs, &bad, &bad_i);
  if (bad >= 0) return set_error(SBIO_EINVAL, "point %lld lies inside spheroid %d", (long long)bad, bad_i);
  sbio_targets* ts = new sbio_targets();
  ts->g = g;
  ts->T = T;
  ts->view = g->d;
  std::vector<int32_t> pt(pairs.size()), ps(pairs.size());
  std::vector<std::vector<int32_t>> skip(T);
  for (size_t k = 0; k < pairs.size(); ++k) {
    pt[k] = pairs[k].first;
    ps[k] = pairs[k].second;
    if (h.parts[ps[k]].kind == SBIO_PROLATE) ts->n_pro++;
    skip[pt[k]].push_back(ps[k]);
  }
  ts->n_pairs = (int64_t)pairs.size();
  ts->far_pairs = (T * (int64_t)h.M - ts->n_pairs) * h.G;
  std::vector<int32_t> sptr(T + 1, 0), sidx;
  for (int64_t t = 0; t < T; ++t) {
    std::sort(skip[t].begin(), skip[t].end());
    skip[t].push_back(INT32_MAX);   // sentinel
    sptr[t + 1] = sptr[t] + (int32_t)skip[t].size();
    sidx.insert(sidx.end(), skip[t].begin(), skip[t].end());
  }
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
  if (!rc) rc = ts_upload(ts, &v.pair_t, pt.data(), pt.size(), "target near pairs", st);
  if (!rc) rc = ts_upload(ts, &v.pair_s, ps.data(), ps.size(), "target near pairs", st);
  if (!rc) rc = ts_upload(ts, &v.skip_ptr, sptr.data(), sptr.size(), "target skip lists", st);
  if (!rc) rc = ts_upload(ts, &v.skip_idx, sidx.data(), sidx.size(), "target skip lists", st);
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
  if (fork) {
    SBIO_CUDA_TRY(cudaEventRecord(g->ev_fork, st));
    SBIO_CUDA_TRY(cudaStreamWaitEvent(g->near_stream, g->ev_fork, 0));
    ts->view.near_grid_cap = h.near_ctas_per_sm > 0 ? h.near_ctas_per_sm * sm_count() : 0;
    nl(ts->view, ts->n_pro, ts->n_pairs, ts->view.inv, S_out, D_out, g->near_stream);
    ts->view.near_grid_cap = 0;
    SBIO_CUDA_TRY(cudaGetLastError());
    SBIO_CUDA_TRY(cudaEventRecord(g->ev_join, g->near_stream));
  } else if (ts->n_pairs > 0) {
    nl(ts->view, ts->n_pro, ts->n_pairs, ts->view.inv, S_out, D_out, st);
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  launch_far_on(ts->view, h, ts->T, S_out, D_out, st);
  SBIO_CUDA_TRY(cudaGetLastError());
  if (fork) SBIO_CUDA_TRY(cudaStreamWaitEvent(st, g->ev_join, 0));
  return SBIO_OK;
}

}  // extern "C"
