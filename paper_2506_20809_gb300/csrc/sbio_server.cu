// Request-serving engine for BIO applies with continuous batching.
//
// A request carries a suspension, an operator (Laplace S+D or Stokes single
// layer) and n_applies coefficient sets in host memory.  The scheduler admits
// requests first-in first-out whenever a slot is free and the request's
// estimated device footprint fits the remaining memory budget; requests that
// arrive while others run are admitted as soon as slots and memory free up.
// Each slot is a host thread with its own CUDA stream: it builds the resident
// geometry once (host set-up + upload), runs the n_applies applies back to
// back with the geometry and near lists resident, copies every result to the
// request's host buffer, releases the geometry and reports completion.  Work of
// different slots overlaps on the device.  Waits on the host are bounded by the
// caller's timeout.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "sbio_internal.cuh"

namespace {

using clock_type = std::chrono::steady_clock;

struct Job {
  int64_t ticket;
  sbio_request req;
  std::vector<sbio_spheroid> sph;     // owned copy of the descriptors
  clock_type::time_point t_submit;
  size_t estimate = 0;
  int status = 1;                    // 1 queued/running, 0 done, < 0 error
  double latency_ms = 0.0;
  double service_ms = 0.0;
  std::string error;                 // message of a failed request
};

}  // namespace

struct sbio_server {
  sbio_ctx* ctx = nullptr;
  int n_slots = 0;
  size_t budget = 0;
  size_t reserved = 0;
  int running = 0;
  bool stop = false;
  std::mutex mu;
  std::condition_variable cv_sched;   // wakes the workers
  std::condition_variable cv_done;    // wakes waiters
  std::deque<Job*> queue;
  std::map<int64_t, Job*> jobs;
  int64_t next_ticket = 1;
  std::vector<std::thread> workers;
  int64_t completed = 0, applies_done = 0;
};

namespace sbio {

// Conservative device footprint of a request (geometry + staging).
static size_t estimate_bytes(int32_t M, const sbio_options& o) {
  const int64_t G = (int64_t)(o.p + 1) * (o.n_phi ? o.n_phi : 2 * (o.p + 1));
  const int64_t N = G * M;
  const int64_t nc1 = (int64_t)(o.p + 2) * (o.p + 2);
  return (size_t)(N * 420 + (int64_t)M * (nc1 * 8 * 12 + 4096) + (4 << 20));
}

constexpr int64_t kServeTreeMinNodes = 50000;

static int run_job(sbio_server* s, Job* j, cudaStream_t st) {
  const sbio_request& r = j->req;
  sbio_geom* g = nullptr;
  sbio_options o = r.opts;
  int rc = geom_create_async(s->ctx, j->sph.data(), r.M, &o, st, &g);
  if (rc) return rc;
  const int64_t N = g->h.N;
  const size_t nc = (size_t)(o.p + 1) * (o.p + 1) * r.M;
  const bool stokes = r.op == SBIO_OP_STOKES;
  // the treecode far field for mixed requests that ask for it and are large
  // enough to gain from it (below about 50,000 nodes its fixed costs make it
  // slower than the direct sum)
  if ((r.flags & SBIO_REQ_TREE) && o.precision == SBIO_MIXED && r.M > 1 && N >= kServeTreeMinNodes) {
    rc = tree_attach_async(g, 16, 0.5, st);
    if (rc) {
      geom_destroy_async(g, st);
      return rc;
    }
  }
  const size_t in_per = stokes ? 3 * nc : 2 * nc;
  const size_t out_per = stokes ? 3 * (size_t)N : 2 * (size_t)N;
  double *din = nullptr, *dout = nullptr;
  rc = dev_alloc(g, (void**)&din, in_per * sizeof(double), "request input");
  if (!rc) rc = dev_alloc(g, (void**)&dout, out_per * sizeof(double), "request output");
  for (int a = 0; a < r.n_applies && !rc; ++a) {
    cudaError_t e = cudaMemcpyAsync(din, r.coef_host + a * in_per, in_per * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = set_error(SBIO_ECUDA, "request input copy: %s", cudaGetErrorString(e));
    if (!rc) {
      if (stokes)
        rc = launch_stokes(g, din, dout, st);
      else
        rc = launch_laplace(g, din, din + nc, dout, dout + N, SBIO_PART_ALL, st);
    }
    if (!rc) {
      e = cudaMemcpyAsync(r.out_host + a * out_per, dout, out_per * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) rc = set_error(SBIO_ECUDA, "request output copy: %s", cudaGetErrorString(e));
    }
  }
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = set_error(SBIO_ECUDA, "request stream: %s", cudaGetErrorString(e));
  }
  geom_destroy_async(g, st);
  return rc;
}

static void worker_main(sbio_server* s) {
  cudaSetDevice(s->ctx->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Job* j = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_sched.wait(lk, [&] {
        if (s->stop && s->queue.empty()) return true;
        if (s->queue.empty()) return false;
        // first-in first-out admission by memory
        Job* h = s->queue.front();
        return s->budget == 0 || s->reserved + h->estimate <= s->budget || s->running == 0;
      });
      if (s->queue.empty()) break;
      j = s->queue.front();
      s->queue.pop_front();
      s->reserved += j->estimate;
      s->running++;
    }
    const auto t0 = clock_type::now();
    int rc = run_job(s, j, st);
    const auto t1 = clock_type::now();
    const std::string msg = rc ? std::string(sbio_last_error(nullptr)) : std::string();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->reserved -= j->estimate;
      s->running--;
      j->status = rc;
      j->error = msg;
      j->latency_ms = std::chrono::duration<double, std::milli>(t1 - j->t_submit).count();
      j->service_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
      if (!rc) {
        s->completed++;
        s->applies_done += j->req.n_applies;
      }
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace sbio

using namespace sbio;

extern "C" {

int sbio_server_create(sbio_ctx* ctx, int32_t n_slots, size_t mem_budget_bytes, sbio_server** out) {
  clear_error();
  if (!ctx || !out || n_slots < 1 || n_slots > 64) return set_error(SBIO_EINVAL, "bad server arguments");
  sbio_server* s = new sbio_server();
  s->ctx = ctx;
  s->n_slots = n_slots;
  s->budget = mem_budget_bytes;
  for (int k = 0; k < n_slots; ++k) s->workers.emplace_back(worker_main, s);
  *out = s;
  return SBIO_OK;
}

int sbio_server_submit(sbio_server* s, const sbio_request* r, int64_t* ticket) {
  clear_error();
  if (!s || !r || !ticket || !r->sph || r->M < 1 || r->n_applies < 1 || !r->coef_host || !r->out_host)
    return set_error(SBIO_EINVAL, "bad request");
  if (r->op != SBIO_OP_LAPLACE && r->op != SBIO_OP_STOKES) return set_error(SBIO_EINVAL, "unknown operator %d", r->op);
  int rc = validate(r->sph, r->M, &r->opts);
  if (rc) return rc;
  Job* j = new Job();
  j->req = *r;
  j->sph.assign(r->sph, r->sph + r->M);
  j->req.sph = j->sph.data();
  j->t_submit = clock_type::now();
  j->estimate = estimate_bytes(r->M, r->opts);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete j;
      return set_error(SBIO_EINVAL, "server is shutting down");
    }
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
  }
  s->cv_sched.notify_all();
  *ticket = j->ticket;
  return SBIO_OK;
}

int sbio_server_wait(sbio_server* s, int64_t ticket, double timeout_s, int32_t* status, double* latency_ms,
                     double* service_ms) {
  clear_error();
  if (!s) return set_error(SBIO_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return set_error(SBIO_EINVAL, "unknown ticket %lld", (long long)ticket);
  Job* j = it->second;
  const bool done = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return j->status <= 0; });
  if (!done) return set_error(SBIO_ETIMEOUT, "ticket %lld not finished within %.3f s", (long long)ticket, timeout_s);
  if (status) *status = j->status;
  if (j->status) set_error(j->status, "request %lld failed: %s", (long long)ticket, j->error.c_str());
  if (latency_ms) *latency_ms = j->latency_ms;
  if (service_ms) *service_ms = j->service_ms;
  s->jobs.erase(it);
  delete j;
  return SBIO_OK;
}

int sbio_server_stats(sbio_server* s, int64_t* completed, int64_t* applies, int32_t* running, int32_t* queued,
                      size_t* reserved) {
  if (!s) return set_error(SBIO_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (applies) *applies = s->applies_done;
  if (running) *running = s->running;
  if (queued) *queued = (int32_t)s->queue.size();
  if (reserved) *reserved = s->reserved;
  return SBIO_OK;
}

int sbio_server_destroy(sbio_server* s) {
  if (!s) return SBIO_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
  return SBIO_OK;
}

}  // extern "C"
