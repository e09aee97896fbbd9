// Forward spheroidal transform and the exterior Laplace boundary-value solves
// of the numerical section (Sec. 5.1), on the device.
//
// Forward transform: the real-basis coefficients of node values f,
//     f^_nm = sum_j w_j (2 pi / n_phi) sum_k f_jk Y_nm(v_j, phi_k),
// separable (Fourier sums in phi per GL row, then Legendre sums in v), exact
// for band-limited f of degree <= p; the modified-basis coefficients are
// those of f sqrt(u0^2 -+ v^2).
//
// Dirichlet (completed double layer): 1/2 sigma + D[sigma] + C[sigma] = f,
// Neumann (single layer): -1/2 rho + S'[rho] = g, both in coefficient space:
// the unknown is the density's coefficient vector, one operator application
// is the apply on the geometry followed by the forward transform of its node
// values, and the identity term acts on the coefficients exactly.  The
// completions: C_I (charges int sigma_i dS at the centres, kernel 1/|x - c_i|
// as printed), eta C_I, S and eta S with eta_i from the paper's table.
//
// The linear systems are solved by restarted GMRES driven from the host:
// Arnoldi with classical Gram-Schmidt applied twice (one projection kernel and
// one update kernel per pass, deterministic two-stage reductions), the small
// Hessenberg least-squares problem by Givens rotations on the host.
#include <chrono>
#include <cmath>
#include <vector>

#include "sbio_internal.cuh"

namespace sbio {
namespace {

constexpr double kTwoPi = 6.283185307179586;

// One CTA per particle: out[i][k] = alpha * x[i][k] + (T f)_k, with f the
// node values (f0 + f1, f1 optional), times sqrt(u0^2 + sgn v^2) when
// `modified`.  Shared memory: n_v x (2p+1) Fourier sums.
__global__ void __launch_bounds__(256) analysis_kernel(int p, int n_v, int n_phi, const double* __restrict__ f0,
                                                       const double* __restrict__ f1, int modified,
                                                       const double* __restrict__ sqrtw,
                                                       const double* __restrict__ glw,
                                                       const double* __restrict__ ptab,
                                                       const double* __restrict__ trig, double alpha,
                                                       const double* __restrict__ x, double* __restrict__ out) {
  extern __shared__ double Fs[];   // n_v x (2p+1)
  const int i = blockIdx.x, nmw = 2 * p + 1, nm = nm_count(p), nc = (p + 1) * (p + 1);
  const int64_t base = (int64_t)i * n_v * n_phi;
  const double dphi = kTwoPi / n_phi;
  for (int idx = threadIdx.x; idx < n_v * nmw; idx += blockDim.x) {
    const int j = idx / nmw, ms = idx - j * nmw, m = ms - p, am = m < 0 ? -m : m;
    double s = 0.0;
    for (int k = 0; k < n_phi; ++k) {
      const int64_t t = base + (int64_t)j * n_phi + k;
      const double v = f1 ? f0[t] + f1[t] : f0[t];
      s = fma(v, trig[((size_t)k * (p + 1) + am) * 2 + (m < 0 ? 1 : 0)], s);
    }
    const double wj = glw[j] * dphi * (modified ? sqrtw[(size_t)i * n_v + j] : 1.0);
    Fs[idx] = s * wj;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const int n = (int)sqrt((double)k);
    const int m = k - n * n - n, am = m < 0 ? -m : m;
    const double s2 = m ? 1.4142135623730951 : 1.0;
    double s = 0.0;
    for (int j = 0; j < n_v; ++j) s = fma(Fs[j * nmw + m + p], ptab[(size_t)j * nm + nm_index(n, am)], s);
    const double a = x ? alpha * x[(size_t)i * nc + k] : 0.0;
    out[(size_t)i * nc + k] = a + s2 * s;
  }
}

// One CTA per particle: node values sigma = sum mu^ Y of the plain
// coefficients, then (S completions) st_i = eta_i T_mod(sigma) or (C_I
// completions) q_i = eta_i sum_t w_t sigma_t.  Shared memory: G node values
// + n_v x (2p+1) sums.
__global__ void __launch_bounds__(256) completion_kernel(int p, int n_v, int n_phi, const double* __restrict__ mu,
                                                         const double* __restrict__ eta, int want_st,
                                                         const double* __restrict__ w,
                                                         const double* __restrict__ sqrtw,
                                                         const double* __restrict__ glw,
                                                         const double* __restrict__ ptab,
                                                         const double* __restrict__ trig, double* __restrict__ st,
                                                         double* __restrict__ q) {
  extern __shared__ double sm[];
  const int i = blockIdx.x, nmw = 2 * p + 1, nm = nm_count(p), nc = (p + 1) * (p + 1), G = n_v * n_phi;
  double* vals = sm;               // G
  double* Fs = sm + G;             // n_v x nmw
  __shared__ double red[256];
  const double* c = mu + (size_t)i * nc;
  // Legendre sums per (row, m), then Fourier sums per node
  for (int idx = threadIdx.x; idx < n_v * nmw; idx += blockDim.x) {
    const int j = idx / nmw, ms = idx - j * nmw, m = ms - p, am = m < 0 ? -m : m;
    const double s2 = m ? 1.4142135623730951 : 1.0;
    double s = 0.0;
    for (int n = am; n <= p; ++n) s = fma(c[n * n + n + m], ptab[(size_t)j * nm + nm_index(n, am)], s);
    Fs[idx] = s2 * s;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < G; l += blockDim.x) {
    const int j = l / n_phi, k = l - j * n_phi;
    const double* tr = trig + (size_t)k * (p + 1) * 2;
    const double* F = Fs + j * nmw + p;
    double v = F[0];
    for (int m = 1; m <= p; ++m) v = fma(F[m], tr[2 * m], fma(F[-m], tr[2 * m + 1], v));
    vals[l] = v;
  }
  __syncthreads();
  if (want_st) {
    const double dphi = kTwoPi / n_phi;
    for (int idx = threadIdx.x; idx < n_v * nmw; idx += blockDim.x) {
      const int j = idx / nmw, ms = idx - j * nmw, m = ms - p, am = m < 0 ? -m : m;
      double s = 0.0;
      for (int k = 0; k < n_phi; ++k) s = fma(vals[j * n_phi + k], trig[((size_t)k * (p + 1) + am) * 2 + (m < 0 ? 1 : 0)], s);
      Fs[idx] = s * glw[j] * dphi * sqrtw[(size_t)i * n_v + j];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
      const int n = (int)sqrt((double)k);
      const int m = k - n * n - n, am = m < 0 ? -m : m;
      double s = 0.0;
      for (int j = 0; j < n_v; ++j) s = fma(Fs[j * nmw + m + p], ptab[(size_t)j * nm + nm_index(n, am)], s);
      st[(size_t)i * nc + k] = eta[i] * (m ? 1.4142135623730951 : 1.0) * s;
    }
  } else {
    double s = 0.0;
    for (int l = threadIdx.x; l < G; l += blockDim.x) s = fma(w[(int64_t)i * G + l], vals[l], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) q[i] = eta[i] * red[0];
  }
}

// u[t] += sum_i q_i / |x_t - c_i| (the C_I field at the nodes).
__global__ void __launch_bounds__(256) charges_field_kernel(int M, const PartGeom* __restrict__ parts,
                                                            const double* __restrict__ q,
                                                            const double* __restrict__ xyz, int64_t N,
                                                            double* __restrict__ u) {
  __shared__ double sc[4 * 256];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double x0 = 0, x1 = 0, x2 = 0, acc = 0.0;
  if (t < N) {
    x0 = xyz[t * 3 + 0];
    x1 = xyz[t * 3 + 1];
    x2 = xyz[t * 3 + 2];
  }
  for (int i0 = 0; i0 < M; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    if (i < M) {
      sc[threadIdx.x * 4 + 0] = parts[i].c[0];
      sc[threadIdx.x * 4 + 1] = parts[i].c[1];
      sc[threadIdx.x * 4 + 2] = parts[i].c[2];
      sc[threadIdx.x * 4 + 3] = q[i];
    }
    __syncthreads();
    const int cnt = min((int)blockDim.x, M - i0);
    for (int k = 0; k < cnt; ++k) {
      const double d0 = x0 - sc[k * 4 + 0], d1 = x1 - sc[k * 4 + 1], d2 = x2 - sc[k * 4 + 2];
      acc = fma(sc[k * 4 + 3], rsqrt(d0 * d0 + d1 * d1 + d2 * d2), acc);
    }
    __syncthreads();
  }
  if (t < N) u[t] += acc;
}

// ---- Krylov vector kernels (deterministic two-stage reductions) ----------
constexpr int kRedBlocks = 240;     // partial sums per projection
constexpr int kRedThreads = 256;

// partial[j][b] = sum over block b's share of e of V[j][e] * w[e], j < k1
__global__ void __launch_bounds__(kRedThreads) proj_kernel(const double* __restrict__ V, int64_t ldv,
                                                            const double* __restrict__ w, int64_t n,
                                                            double* __restrict__ partial) {
  __shared__ double red[kRedThreads];
  const int j = blockIdx.y;
  const double* v = V + (int64_t)j * ldv;
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s = fma(v[e], w[e], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = red[0];
}

// h[j] = sum_b partial[j][b]
__global__ void __launch_bounds__(kRedThreads) reduce_partials_kernel(const double* __restrict__ partial, int nb,
                                                                       double* __restrict__ h) {
  __shared__ double red[kRedThreads];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(int64_t)blockIdx.x * nb + b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) h[blockIdx.x] = red[0];
}

// w[e] += sgn * sum_{j < k1} h[j] V[j][e]
__global__ void __launch_bounds__(256) combine_kernel(const double* __restrict__ V, int64_t ldv, int k1,
                                                      const double* __restrict__ h, double sgn,
                                                      double* __restrict__ w, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k1; ++j) s = fma(h[j], V[(int64_t)j * ldv + e], s);
    w[e] = fma(sgn, s, w[e]);
  }
}

// y[e] = a * x[e] + b * y[e]
__global__ void __launch_bounds__(256) axpby_kernel(double a, const double* __restrict__ x, double b,
                                                    double* __restrict__ y, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a * x[e] + (b == 0.0 ? 0.0 : b * y[e]);
}

}  // namespace

namespace {

double eta_of(const PartGeom& P, int completion) {
  const double R = std::max(P.A, P.C) / std::min(P.A, P.C), eps = 1.0 / R;
  const bool prolate = P.kind == SBIO_PROLATE;
  if (completion == SBIO_COMPLETION_CI || completion == SBIO_COMPLETION_S) return 1.0;
  if (completion == SBIO_COMPLETION_ETA_CI) {
    if (!prolate && R > 3.0) return 0.06;
    // eps / area of the spheroid with major semi-axis 1 and aspect ratio R
    double area = 4.0 * kPi;
    if (eps < 1.0) {
      const double e = std::sqrt(1.0 - eps * eps);
      area = prolate ? 2.0 * kPi * eps * eps * (1.0 + std::asin(e) / (eps * e))
                     : 2.0 * kPi * (1.0 + eps * eps / e * std::atanh(e));
    }
    return eps / area;
  }
  if (prolate) return R <= 3.0 ? 0.5 : 1.0 / (2.0 * eps * std::log(1.0 / eps));
  return R <= 3.0 ? 1.0 / (4.0 * eps) + 0.25 : 1.0;
}

struct Solver {
  sbio_geom* g = nullptr;
  cudaStream_t st = nullptr;
  bool dirichlet = true;
  int completion = SBIO_COMPLETION_ETA_S;
  int64_t n = 0;                      // M (p+1)^2 unknowns
  double *eta = nullptr, *nodesA = nullptr, *nodesB = nullptr, *stc = nullptr, *q = nullptr;
  double *V = nullptr, *w = nullptr, *b = nullptr, *x = nullptr, *partial = nullptr, *h = nullptr;
  std::vector<void*> mem;
  size_t bytes = 0;

  int alloc(void** p, size_t sz) {
    sbio_ctx* c = g->ctx;
    const size_t prev = c->used.fetch_add(sz);
    if (c->budget && prev + sz > c->budget) {
      c->used.fetch_sub(sz);
      return set_error(SBIO_ENOMEM, "device budget exceeded by the solver workspace (%zu bytes)", sz);
    }
    if (cudaMallocAsync(p, sz, st) != cudaSuccess) {
      cudaGetLastError();
      c->used.fetch_sub(sz);
      return set_error(SBIO_ENOMEM, "solver workspace allocation (%zu bytes) failed", sz);
    }
    mem.push_back(*p);
    bytes += sz;
    return SBIO_OK;
  }
  void release() {
    for (void* p : mem) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    g->ctx->used.fetch_sub(bytes);
    mem.clear();
    bytes = 0;
  }

  void analysis(const double* f0, const double* f1, bool modified, double alpha, const double* xin, double* out) {
    const GeomHost& hh = g->h;
    const size_t smem = (size_t)hh.n_v * (2 * hh.p + 1) * sizeof(double);
    analysis_kernel<<<hh.M, 256, smem, st>>>(hh.p, hh.n_v, hh.n_phi, f0, f1, modified ? 1 : 0, g->d.sqrtw, g->d.glw,
                                             g->d.ptab, g->d.trig, alpha, xin, out);
    count_launch();
  }

  // y = K x
  int apply(const double* xin, double* y) {
    const GeomHost& hh = g->h;
    const DevGeom& d = g->d;
    int rc;
    if (!dirichlet) {
      if ((rc = launch_laplace_deriv(g, xin, nullptr, nodesA, nullptr, st))) return rc;
      analysis(nodesA, nullptr, true, -0.5, xin, y);
      SBIO_CUDA_TRY(cudaGetLastError());
      return SBIO_OK;
    }
    const bool has_s = completion == SBIO_COMPLETION_S || completion == SBIO_COMPLETION_ETA_S;
    const size_t smem = (size_t)(hh.G + hh.n_v * (2 * hh.p + 1)) * sizeof(double);
    completion_kernel<<<hh.M, 256, smem, st>>>(hh.p, hh.n_v, hh.n_phi, xin, eta, has_s ? 1 : 0, d.w, d.sqrtw, d.glw,
                                               d.ptab, d.trig, stc, q);
    count_launch();
    SBIO_CUDA_TRY(cudaGetLastError());
    if (has_s) {
      if ((rc = launch_laplace(g, stc, xin, nodesA, nodesB, SBIO_PART_ALL, st))) return rc;
      analysis(nodesA, nodesB, false, 0.5, xin, y);
    } else {
      if ((rc = launch_laplace(g, nullptr, xin, nullptr, nodesB, SBIO_PART_ALL, st))) return rc;
      charges_field_kernel<<<(unsigned)((hh.N + 255) / 256), 256, 0, st>>>(hh.M, d.parts, q, d.xyz, hh.N, nodesB);
      count_launch();
      analysis(nodesB, nullptr, false, 0.5, xin, y);
    }
    SBIO_CUDA_TRY(cudaGetLastError());
    return SBIO_OK;
  }

  // hv[j] = <V_j, v> for j < k1 (host copy); V rows of length n
  int project(const double* Vb, int k1, const double* v, std::vector<double>& hv) {
    proj_kernel<<<dim3(kRedBlocks, k1), kRedThreads, 0, st>>>(Vb, n, v, n, partial);
    reduce_partials_kernel<<<k1, kRedThreads, 0, st>>>(partial, kRedBlocks, h);
    count_launch(2);
    hv.resize(k1);
    SBIO_CUDA_TRY(cudaMemcpyAsync(hv.data(), h, k1 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SBIO_CUDA_TRY(cudaStreamSynchronize(st));
    return SBIO_OK;
  }

  // v += sgn * V[0..k1) hv
  int combine(const double* Vb, int k1, const std::vector<double>& hv, double sgn, double* v) {
    SBIO_CUDA_TRY(cudaMemcpyAsync(h, hv.data(), k1 * sizeof(double), cudaMemcpyHostToDevice, st));
    combine_kernel<<<2 * sm_count(), 256, 0, st>>>(Vb, n, k1, h, sgn, v, n);
    count_launch();
    SBIO_CUDA_TRY(cudaGetLastError());
    return SBIO_OK;
  }

  void axpby(double a, const double* xin, double bb, double* y) {
    axpby_kernel<<<2 * sm_count(), 256, 0, st>>>(a, xin, bb, y, n);
    count_launch();
  }
};

}  // namespace

// Restarted GMRES on K x = b (x0 = 0).  V holds restart+1 basis vectors.
static int gmres(Solver& S, double tol, int max_iter, int restart, sbio_solve_info* info) {
  const int64_t n = S.n;
  std::vector<double> hv, hv2;
  int rc = S.project(S.b, 1, S.b, hv);
  if (rc) return rc;
  const double bnorm = std::sqrt(hv[0]);
  SBIO_CUDA_TRY(cudaMemsetAsync(S.x, 0, n * sizeof(double), S.st));
  int iters = 0, restarts = 0;
  bool converged = bnorm == 0.0;
  double est = 0.0;
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), gv(restart + 1), y(restart);
  // r = b (x = 0) on the first cycle, b - K x afterwards
  SBIO_CUDA_TRY(cudaMemcpyAsync(S.w, S.b, n * sizeof(double), cudaMemcpyDeviceToDevice, S.st));
  double beta = bnorm;
  while (!converged && iters < max_iter) {
    S.axpby(1.0 / beta, S.w, 0.0, S.V);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k_end = 0;
    for (int k = 0; k < restart && iters < max_iter; ++k) {
      double* vk1 = S.V + (int64_t)(k + 1) * n;
      if ((rc = S.apply(S.V + (int64_t)k * n, vk1))) return rc;
      // classical Gram-Schmidt, twice
      if ((rc = S.project(S.V, k + 1, vk1, hv))) return rc;
      if ((rc = S.combine(S.V, k + 1, hv, -1.0, vk1))) return rc;
      if ((rc = S.project(S.V, k + 1, vk1, hv2))) return rc;
      if ((rc = S.combine(S.V, k + 1, hv2, -1.0, vk1))) return rc;
      std::vector<double> nn;
      if ((rc = S.project(vk1, 1, vk1, nn))) return rc;
      const double hk1 = std::sqrt(std::max(nn[0], 0.0));
      for (int j = 0; j <= k; ++j) H[(size_t)j * restart + k] = hv[j] + hv2[j];
      H[(size_t)(k + 1) * restart + k] = hk1;
      if (hk1 > 0.0) S.axpby(1.0 / hk1, vk1, 0.0, vk1);
      // previous rotations, then a new one zeroing H[k+1][k]
      for (int j = 0; j < k; ++j) {
        const double a = H[(size_t)j * restart + k], c = H[(size_t)(j + 1) * restart + k];
        H[(size_t)j * restart + k] = cs[j] * a + sn[j] * c;
        H[(size_t)(j + 1) * restart + k] = -sn[j] * a + cs[j] * c;
      }
      const double a = H[(size_t)k * restart + k], c = H[(size_t)(k + 1) * restart + k];
      const double r = std::hypot(a, c);
      cs[k] = r > 0.0 ? a / r : 1.0;
      sn[k] = r > 0.0 ? c / r : 0.0;
      H[(size_t)k * restart + k] = r;
      H[(size_t)(k + 1) * restart + k] = 0.0;
      gv[k + 1] = -sn[k] * gv[k];
      gv[k] = cs[k] * gv[k];
      ++iters;
      k_end = k + 1;
      est = std::fabs(gv[k + 1]) / bnorm;
      if (est <= tol || hk1 == 0.0) break;
    }
    // y = H^-1 g (upper triangular), x += V y
    for (int i = k_end - 1; i >= 0; --i) {
      double s = gv[i];
      for (int j = i + 1; j < k_end; ++j) s -= H[(size_t)i * restart + j] * y[j];
      y[i] = s / H[(size_t)i * restart + i];
    }
    std::vector<double> yk(y.begin(), y.begin() + k_end);
    if ((rc = S.combine(S.V, k_end, yk, 1.0, S.x))) return rc;
    // true residual r = b - K x
    if ((rc = S.apply(S.x, S.w))) return rc;
    S.axpby(1.0, S.b, -1.0, S.w);
    if ((rc = S.project(S.w, 1, S.w, hv))) return rc;
    beta = std::sqrt(std::max(hv[0], 0.0));
    est = beta / bnorm;
    converged = est <= tol;
    if (!converged) ++restarts;
  }
  if (info) {
    info->iterations = iters;
    info->restarts = restarts;
    info->rel_residual = bnorm > 0.0 ? est : 0.0;
    info->converged = converged ? 1 : 0;
  }
  return SBIO_OK;
}

}  // namespace sbio

using namespace sbio;

static int solve_common(sbio_geom* g, const double* rhs_nodes, bool dirichlet, int completion, double tol,
                        int32_t max_iter, int32_t restart, double* coef_out, double* st_out, double* q_out,
                        sbio_solve_info* info, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const GeomHost& hh = g->h;
  const int64_t nc = (int64_t)(hh.p + 1) * (hh.p + 1);
  Solver S;
  S.g = g;
  S.st = st;
  S.dirichlet = dirichlet;
  S.completion = completion;
  S.n = (int64_t)hh.M * nc;
  const int64_t n = S.n;
  int rc = SBIO_OK;
  auto A = [&](double** p, size_t cnt) {
    if (!rc) rc = S.alloc((void**)p, cnt * sizeof(double));
  };
  A(&S.eta, hh.M);
  A(&S.nodesA, hh.N);
  A(&S.nodesB, hh.N);
  A(&S.stc, n);
  A(&S.q, hh.M);
  A(&S.V, (size_t)(restart + 1) * n);
  A(&S.w, n);
  A(&S.b, n);
  A(&S.x, n);
  A(&S.partial, (size_t)kRedBlocks * (restart + 1));
  A(&S.h, restart + 1);
  if (!rc) {
    std::vector<double> eta(hh.M);
    for (int i = 0; i < hh.M; ++i) eta[i] = eta_of(hh.parts[i], completion);
    if (cudaMemcpyAsync(S.eta, eta.data(), hh.M * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
      rc = set_error(SBIO_ECUDA, "eta upload failed");
    if (!rc) cudaStreamSynchronize(st);   // eta is a pageable host vector
  }
  if (!rc) {
    S.analysis(rhs_nodes, nullptr, !dirichlet, 0.0, nullptr, S.b);
    if (cudaGetLastError() != cudaSuccess) rc = set_error(SBIO_ECUDA, "right-hand side transform failed");
  }
  if (!rc) rc = gmres(S, tol, max_iter, restart, info);
  if (!rc) {
    cudaMemcpyAsync(coef_out, S.x, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (dirichlet && (st_out || q_out)) {
      const bool has_s = completion == SBIO_COMPLETION_S || completion == SBIO_COMPLETION_ETA_S;
      const size_t smem = (size_t)(hh.G + hh.n_v * (2 * hh.p + 1)) * sizeof(double);
      completion_kernel<<<hh.M, 256, smem, st>>>(hh.p, hh.n_v, hh.n_phi, S.x, S.eta, has_s ? 1 : 0, g->d.w,
                                                 g->d.sqrtw, g->d.glw, g->d.ptab, g->d.trig, S.stc, S.q);
      count_launch();
      if (!has_s) cudaMemsetAsync(S.stc, 0, n * sizeof(double), st);
      if (has_s) cudaMemsetAsync(S.q, 0, hh.M * sizeof(double), st);
      if (st_out) cudaMemcpyAsync(st_out, S.stc, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
      if (q_out) cudaMemcpyAsync(q_out, S.q, hh.M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      rc = set_error(SBIO_ECUDA, "solver output copy failed");
  }
  S.release();
  if (info) info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

extern "C" {

int sbio_forward_transform(sbio_geom* g, const double* values, int32_t modified, double* coef_out, void* stream) {
  clear_error();
  if (!g || !values || !coef_out) return set_error(SBIO_EINVAL, "null argument");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  const GeomHost& hh = g->h;
  const size_t smem = (size_t)hh.n_v * (2 * hh.p + 1) * sizeof(double);
  analysis_kernel<<<hh.M, 256, smem, (cudaStream_t)stream>>>(hh.p, hh.n_v, hh.n_phi, values, nullptr,
                                                             modified ? 1 : 0, g->d.sqrtw, g->d.glw, g->d.ptab,
                                                             g->d.trig, 0.0, nullptr, coef_out);
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}

static int check_solve_args(sbio_geom* g, const double* rhs, const double* out, double tol, int32_t max_iter,
                            int32_t restart) {
  if (!g || !rhs || !out) return set_error(SBIO_EINVAL, "null argument");
  if (!(tol > 0.0) || max_iter < 1 || restart < 1 || restart > 1000)
    return set_error(SBIO_EINVAL, "tol must be > 0, max_iter >= 1, 1 <= restart <= 1000");
  return SBIO_OK;
}

int sbio_solve_dirichlet(sbio_geom* g, const double* f_nodes, int32_t completion, double tol, int32_t max_iter,
                         int32_t restart, double* mu_hat_out, double* sigma_tilde_out, double* charges_out,
                         sbio_solve_info* info, void* stream) {
  clear_error();
  int rc = check_solve_args(g, f_nodes, mu_hat_out, tol, max_iter, restart);
  if (rc) return rc;
  if (completion < SBIO_COMPLETION_CI || completion > SBIO_COMPLETION_ETA_S)
    return set_error(SBIO_EINVAL, "unknown completion %d", completion);
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  return solve_common(g, f_nodes, true, completion, tol, max_iter, restart, mu_hat_out, sigma_tilde_out,
                      charges_out, info, (cudaStream_t)stream);
}

int sbio_solve_neumann(sbio_geom* g, const double* g_nodes, double tol, int32_t max_iter, int32_t restart,
                       double* rho_tilde_out, sbio_solve_info* info, void* stream) {
  clear_error();
  int rc = check_solve_args(g, g_nodes, rho_tilde_out, tol, max_iter, restart);
  if (rc) return rc;
  if (g->h.p > 20) return set_error(SBIO_ENOTSUP, "the Neumann solve uses S', built for p <= 20");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  return solve_common(g, g_nodes, false, SBIO_COMPLETION_S, tol, max_iter, restart, rho_tilde_out, nullptr,
                      nullptr, info, (cudaStream_t)stream);
}

}  // extern "C"
