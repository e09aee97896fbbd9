// Batched Laplace S+D apply over many independent suspensions of uneven size
// and order p (mixed precision).  One apply of the batch is a CUDA graph:
//   branch A: the synthesis/self kernel of every suspension, then one
//             persistent far-field kernel whose CTAs pull (suspension, target
//             block, tile range) work items from an atomic counter, longest
//             first, until all suspensions' far fields are done;
//   branch B: after all syntheses, the near-field kernels of every suspension
//             (FP64) spread over several streams, so that their small grids
//             run side by side when SM slots are free.
// The graph is captured on the first apply and replayed while the caller
// passes the same buffers; the per-suspension far descriptors live in device
// memory and are refreshed before every replay.
#include <algorithm>
#include <vector>

#include "sbio_internal.cuh"

struct sbio_batch {
  sbio_ctx* ctx = nullptr;
  std::vector<sbio_geom*> geoms;
  std::vector<sbio::FarDesc> h_desc;
  sbio::FarDesc* d_desc = nullptr;
  int4* d_items = nullptr;
  int n_items = 0;
  int* d_counter = nullptr;
  int far_tt = 2;
  int grid = 0;
  int ctas_per_sm = 6;                 // persistent far grid = SMs x this
  int n_tree = 0;                      // suspensions whose far field is the treecode
  int64_t far_pairs = 0;
  cudaStream_t sa = nullptr, sb = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_near = nullptr;
  // near branch: the suspensions' near kernels spread over several streams so
  // that their small grids run side by side in the far kernel's spare slots
  static constexpr int kNearStreams = 8;
  cudaStream_t sn[kNearStreams] = {};
  cudaEvent_t ev_nj[kNearStreams] = {};
  // the same streams run the suspensions' synthesis kernels (small grids, one
  // per suspension) side by side first; the far kernel waits for all of them
  cudaEvent_t ev_sj[kNearStreams] = {};
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> captured;   // buffers baked into the graph
  int kernels_per_apply = 0;           // kernel nodes of the captured graph
};

namespace sbio {

static int build_items(sbio_batch* b) {
  struct Item {
    int4 v;
    int64_t cost;
  };
  std::vector<Item> items;
  const int tt = b->far_tt < 0 ? -b->far_tt : b->far_tt;
  for (size_t s = 0; s < b->geoms.size(); ++s) {
    if (b->geoms[s]->tree) continue;   // its far field runs as treecode launches in the graph
    const GeomHost& h = b->geoms[s]->h;
    const int nt = (int)h.tiles.size();
    const int64_t tb = (h.N + (int64_t)kFarTile * tt - 1) / ((int64_t)kFarTile * tt);
    // about 64 source tiles (8k source nodes) per item keeps items uniform
    const int per = std::max(1, std::min(nt, 64));
    for (int64_t t = 0; t < tb; ++t)
      for (int lo = 0; lo < nt; lo += per) {
        const int hi = std::min(nt, lo + per);
        const int64_t ntg = std::min<int64_t>((int64_t)kFarTile * tt, h.N - t * kFarTile * tt);
        items.push_back({make_int4((int)s, (int)t, lo, hi), ntg * (hi - lo)});
      }
  }
  std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& c) { return a.cost > c.cost; });
  std::vector<int4> v(items.size());
  for (size_t k = 0; k < items.size(); ++k) v[k] = items[k].v;
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  b->n_items = (int)v.size();
  if (!v.empty()) {
    SBIO_CUDA_TRY(cudaMalloc(&b->d_items, v.size() * sizeof(int4)));
    SBIO_CUDA_TRY(cudaMemcpy(b->d_items, v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // at least as many CTAs as fit: the far field holds the SMs until its item
  // queue is empty (running the FP64 near kernels in slots left beside it
  // measured slower); the near kernels of the suspensions then run side by
  // side on their streams
  b->grid = std::max(1, std::min(b->n_items, sms * b->ctas_per_sm));
  return SBIO_OK;
}

static void drop_graph(sbio_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->captured.clear();
}

static int capture(sbio_batch* b, const double* const* sigma, const double* const* mu, double* const* S,
                   double* const* D) {
  drop_graph(b);
  cudaGraph_t graph = nullptr;
  const int64_t launches_before = launch_counter();
  SBIO_CUDA_TRY(cudaStreamBeginCapture(b->sa, cudaStreamCaptureModeThreadLocal));
  int rc = SBIO_OK;
  cudaEventRecord(b->ev_fork, b->sa);
  cudaStreamWaitEvent(b->sb, b->ev_fork, 0);
  for (int k = 0; k < sbio_batch::kNearStreams; ++k) cudaStreamWaitEvent(b->sn[k], b->ev_fork, 0);
  // branch of each suspension: longest first to the least loaded stream, by
  // a cost of M (p + 1)^2 (the synthesis and near work both grow with it)
  const size_t ns_count = b->geoms.size();
  std::vector<int> branch(ns_count, 0), order(ns_count);
  for (size_t s = 0; s < ns_count; ++s) order[s] = (int)s;
  auto cost = [&](int s) { const GeomHost& h = b->geoms[s]->h; return (double)h.M * (h.p + 1) * (h.p + 1); };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  double load[sbio_batch::kNearStreams] = {};
  for (int s : order) {
    int k = 0;
    for (int j = 1; j < sbio_batch::kNearStreams; ++j)
      if (load[j] < load[k]) k = j;
    branch[s] = k;
    load[k] += cost(s);
  }
  // synthesis of every suspension on its branch, then the far kernel waits
  // for all branches' synthesis
  for (size_t s = 0; s < ns_count && !rc; ++s)
    rc = launch_synth(b->geoms[s], sigma[s], mu[s], S[s], D[s], true, b->sn[branch[s]]);
  for (int k = 0; k < sbio_batch::kNearStreams; ++k) {
    cudaEventRecord(b->ev_sj[k], b->sn[k]);
    cudaStreamWaitEvent(b->sa, b->ev_sj[k], 0);
  }
  // suspensions with a treecode far field run it on their branch, beside the
  // persistent direct kernel of the others, followed by their near field
  for (size_t s = 0; s < ns_count && !rc; ++s) {
    cudaStream_t ns = b->sn[branch[s]];
    if (b->geoms[s]->tree) rc = launch_tree_far(b->geoms[s], S[s], D[s], ns);
    if (!rc) rc = launch_near(b->geoms[s], S[s], D[s], ns);
  }
  for (int k = 0; k < sbio_batch::kNearStreams; ++k) cudaEventRecord(b->ev_nj[k], b->sn[k]);
  cudaEventRecord(b->ev_near, b->sb);
  if (!rc) cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->sa);
  if (!rc && b->n_items > 0)
    rc = launch_far_persistent(b->d_desc, b->d_items, b->n_items, b->d_counter, b->far_tt, b->grid, b->sa);
  for (int k = 0; k < sbio_batch::kNearStreams; ++k) cudaStreamWaitEvent(b->sa, b->ev_nj[k], 0);
  cudaStreamWaitEvent(b->sa, b->ev_near, 0);
  cudaError_t e = cudaStreamEndCapture(b->sa, &graph);
  // capture records launches without running them: count them per replay instead
  b->kernels_per_apply = (int)(launch_counter() - launches_before);
  count_launch(-b->kernels_per_apply);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return set_error(SBIO_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return set_error(SBIO_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  for (size_t s = 0; s < b->geoms.size(); ++s) {
    b->captured.push_back(sigma[s]);
    b->captured.push_back(mu[s]);
    b->captured.push_back(S[s]);
    b->captured.push_back(D[s]);
  }
  return SBIO_OK;
}

}  // namespace sbio

using namespace sbio;

extern "C" {

int sbio_batch_apply(sbio_batch* b, const double* const* sigma, const double* const* mu, double* const* S_out,
                     double* const* D_out, void* stream);

int sbio_batch_create(sbio_ctx* ctx, sbio_geom* const* geoms, int32_t n, sbio_batch** out) {
  clear_error();
  if (!ctx || !geoms || !out || n < 1) return set_error(SBIO_EINVAL, "bad batch arguments");
  *out = nullptr;
  for (int k = 0; k < n; ++k) {
    if (!geoms[k] || geoms[k]->ctx != ctx) return set_error(SBIO_EINVAL, "geometry %d missing or of another context", k);
    if (geoms[k]->h.precision != SBIO_MIXED)
      return set_error(SBIO_EINVAL, "geometry %d: the batched apply runs the mixed-precision path", k);
  }
  SBIO_CUDA_TRY(cudaSetDevice(ctx->device));
  sbio_batch* b = new sbio_batch();
  b->ctx = ctx;
  b->geoms.assign(geoms, geoms + n);
  b->h_desc.resize(n);
  for (int k = 0; k < n; ++k) {
    const sbio_geom* g = geoms[k];
    b->far_pairs += g->h.far_pairs;
    if (g->tree) ++b->n_tree;
    b->h_desc[k] = FarDesc{g->d.tiles, g->d.src32, g->d.tgt32, g->d.cen32, g->d.skip_ptr, g->d.skip_idx, g->h.N,
                           nullptr, nullptr};
  }
  cudaError_t e = cudaMalloc(&b->d_desc, n * sizeof(FarDesc));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->sa, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->sb, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_near, cudaEventDisableTiming);
  for (int k = 0; k < sbio_batch::kNearStreams && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->sn[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_nj[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_sj[k], cudaEventDisableTiming);
  }
  int rc = (e == cudaSuccess) ? build_items(b) : set_error(SBIO_ENOMEM, "batch allocation failed: %s", cudaGetErrorString(e));
  if (rc) {
    sbio_batch_destroy(b);
    return rc;
  }
  *out = b;
  return SBIO_OK;
}

int sbio_batch_destroy(sbio_batch* b) {
  if (!b) return SBIO_OK;
  cudaSetDevice(b->ctx->device);
  if (b->sa) cudaStreamSynchronize(b->sa);
  drop_graph(b);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->sa) cudaStreamDestroy(b->sa);
  if (b->sb) cudaStreamDestroy(b->sb);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_near) cudaEventDestroy(b->ev_near);
  for (int k = 0; k < sbio_batch::kNearStreams; ++k) {
    if (b->sn[k]) cudaStreamDestroy(b->sn[k]);
    if (b->ev_nj[k]) cudaEventDestroy(b->ev_nj[k]);
    if (b->ev_sj[k]) cudaEventDestroy(b->ev_sj[k]);
  }
  delete b;
  return SBIO_OK;
}

int sbio_batch_info(const sbio_batch* b, int64_t* n_items, int64_t* far_pairs, int32_t* far_tt, int32_t* grid) {
  if (!b) return set_error(SBIO_EINVAL, "null batch");
  if (n_items) *n_items = b->n_items;
  if (far_pairs) *far_pairs = b->far_pairs;
  if (far_tt) *far_tt = b->far_tt;
  if (grid) *grid = b->grid;
  return SBIO_OK;
}

int sbio_batch_set_far_tt(sbio_batch* b, int32_t tt) {
  clear_error();
  if (!b) return set_error(SBIO_EINVAL, "null batch");
  if (tt != 1 && tt != 2 && tt != 4 && tt != 8 && tt != -2 && tt != -4 && tt != -8)
    return set_error(SBIO_EINVAL, "far_tt must be 1, 2, 4, 8 or -2, -4, -8 (packed)");
  SBIO_CUDA_TRY(cudaSetDevice(b->ctx->device));
  SBIO_CUDA_TRY(cudaStreamSynchronize(b->sa));
  b->far_tt = tt;
  drop_graph(b);
  return build_items(b);
}

int sbio_batch_autotune(sbio_batch* b, const double* const* sigma, const double* const* mu, double* const* S_out,
                        double* const* D_out, void* stream, int32_t* far_tt, int32_t* near_block,
                        int32_t* ctas_per_sm, double* step_ms) {
  clear_error();
  if (!b || !sigma || !mu || !S_out || !D_out) return set_error(SBIO_EINVAL, "null argument");
  SBIO_CUDA_TRY(cudaSetDevice(b->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SBIO_CUDA_TRY(cudaEventCreate(&e0));
  SBIO_CUDA_TRY(cudaEventCreate(&e1));
  // one warm replay, then the best of two timed replays of the whole step
  auto time_step = [&](double* ms) -> int {
    int rc = sbio_batch_apply(b, sigma, mu, S_out, D_out, stream);
    if (rc) return rc;
    double best = 1e300;
    for (int r = 0; r < 2; ++r) {
      SBIO_CUDA_TRY(cudaEventRecord(e0, st));
      rc = sbio_batch_apply(b, sigma, mu, S_out, D_out, stream);
      if (rc) return rc;
      SBIO_CUDA_TRY(cudaEventRecord(e1, st));
      SBIO_CUDA_TRY(cudaEventSynchronize(e1));
      float t = 0.f;
      SBIO_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
      best = std::min(best, (double)t);
    }
    *ms = best;
    return SBIO_OK;
  };
  auto set_near_block = [&](int nb) {
    for (sbio_geom* g : b->geoms) g->d.near_block = nb;
  };
  auto configure = [&](int tt, int nb, int cps) -> int {
    SBIO_CUDA_TRY(cudaStreamSynchronize(st));
    SBIO_CUDA_TRY(cudaStreamSynchronize(b->sa));
    set_near_block(nb);
    b->far_tt = tt;
    b->ctas_per_sm = cps;
    drop_graph(b);   // the launch shapes are baked into the captured graph
    return build_items(b);
  };
  int best_tt = b->far_tt, best_nb = b->geoms[0]->d.near_block, best_cps = b->ctas_per_sm;
  double best = 1e300;
  int rc = SBIO_OK;
  // targets per thread of the persistent far kernel (scalar and packed)
  for (int tt : {1, 2, 4, 8, -2, -4, -8}) {
    double ms = 0.0;
    if ((rc = configure(tt, best_nb, best_cps)) || (rc = time_step(&ms))) break;
    if (ms < best) {
      best = ms;
      best_tt = tt;
    }
  }
  // near thread-group size, then the persistent grid (fewer far CTAs per SM
  // leave slots for the near kernels of the other graph branch)
  for (int nb : {64, 128}) {
    double ms = 0.0;
    if (rc || (rc = configure(best_tt, nb, best_cps)) || (rc = time_step(&ms))) break;
    if (ms < best) {
      best = ms;
      best_nb = nb;
    }
  }
  for (int cps : {2, 3, 4, 5, 6, 8}) {
    double ms = 0.0;
    if (rc || (rc = configure(best_tt, best_nb, cps)) || (rc = time_step(&ms))) break;
    if (ms < best) {
      best = ms;
      best_cps = cps;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = configure(best_tt, best_nb, best_cps))) return rc;
  if (far_tt) *far_tt = best_tt;
  if (near_block) *near_block = best_nb;
  if (ctas_per_sm) *ctas_per_sm = best_cps;
  if (step_ms) *step_ms = best;
  return SBIO_OK;
}

int sbio_batch_apply(sbio_batch* b, const double* const* sigma, const double* const* mu, double* const* S_out,
                     double* const* D_out, void* stream) {
  clear_error();
  if (!b || !sigma || !mu || !S_out || !D_out) return set_error(SBIO_EINVAL, "null argument");
  const size_t n = b->geoms.size();
  for (size_t s = 0; s < n; ++s)
    if (!sigma[s] || !mu[s] || !S_out[s] || !D_out[s]) return set_error(SBIO_EINVAL, "suspension %zu: null buffer", s);
  SBIO_CUDA_TRY(cudaSetDevice(b->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  bool same = b->exec && b->captured.size() == 4 * n;
  for (size_t s = 0; same && s < n; ++s)
    same = b->captured[4 * s] == sigma[s] && b->captured[4 * s + 1] == mu[s] && b->captured[4 * s + 2] == S_out[s] &&
           b->captured[4 * s + 3] == D_out[s];
  // no replay may still be queued while the executable graph is replaced
  if (!same) {
    SBIO_CUDA_TRY(cudaStreamSynchronize(st));
    int rc = capture(b, sigma, mu, S_out, D_out);
    if (rc) return rc;
  }
  for (size_t s = 0; s < n; ++s) {
    b->h_desc[s].S = S_out[s];
    b->h_desc[s].D = D_out[s];
  }
  // pageable source: staged before the call returns
  SBIO_CUDA_TRY(cudaMemcpyAsync(b->d_desc, b->h_desc.data(), n * sizeof(FarDesc), cudaMemcpyHostToDevice, st));
  SBIO_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  count_launch(b->kernels_per_apply);
  return SBIO_OK;
}

}  // extern "C"
