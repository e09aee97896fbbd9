// Context, error state and resident geometry of the spheroidal BIO library:
// host FP64 set-up (Sec. 2.1-2.2 geometry, Theorems 1-2 multipliers, Sec. 4.1
// near sets) and the upload of everything an apply reads.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>

#include <functional>

#include "sbio_internal.cuh"
#include "sbio_near.cuh"

namespace sbio {

static thread_local std::string t_err;
static std::atomic<int64_t> g_launches{0};

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

void clear_error() { t_err.clear(); }

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int64_t launch_counter() { return g_launches.load(); }

int dev_alloc(sbio_geom* g, void** ptr, size_t bytes, const char* what) {
  *ptr = nullptr;
  if (bytes == 0) return SBIO_OK;
  sbio_ctx* c = g->ctx;
  size_t prev = c->used.fetch_add(bytes);
  if (c->budget && prev + bytes > c->budget) {
    c->used.fetch_sub(bytes);
    return set_error(SBIO_ENOMEM, "device budget exceeded allocating %s (%zu bytes, %zu of %zu in use)", what,
                     bytes, prev, c->budget);
  }
  cudaError_t e = g->async_alloc ? cudaMallocAsync(ptr, bytes, g->setup_stream) : cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    c->used.fetch_sub(bytes);
    *ptr = nullptr;
    return set_error(SBIO_ENOMEM, "cudaMalloc of %s (%zu bytes) failed: %s", what, bytes, cudaGetErrorString(e));
  }
  g->bytes += bytes;
  g->allocs.push_back(*ptr);
  return SBIO_OK;
}

// ---------------------------------------------------------------------------
// numerical helpers of the set-up
// ---------------------------------------------------------------------------

// Gauss-Legendre nodes (ascending) and weights by Newton's method on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? z : p1, pm1 = (n == 1) ? 1.0 : p0;
    dp = n * (z * pn - pm1) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Ferrers functions Pbar_n^m(v) (no Condon-Shortley phase), [nm_index(n,m)].
void ferrers(double v, int N, double* P) {
  const double sv = std::sqrt(std::max(0.0, 1.0 - v * v));
  double pmm = 1.0;
  for (int m = 0; m <= N; ++m) {
    if (m > 0) pmm *= (2.0 * m - 1.0) * sv;
    P[nm_index(m, m)] = pmm;
    if (m + 1 <= N) P[nm_index(m + 1, m)] = (2.0 * m + 1.0) * v * pmm;
    for (int n = m + 1; n < N; ++n)
      P[nm_index(n + 1, m)] = ((2.0 * n + 1.0) * v * P[nm_index(n, m)] - (n + m) * P[nm_index(n - 1, m)]) / (n - m + 1.0);
  }
}

// (n-m)!/(n+m)!
double kfact(int n, int m) {
  double r = 1.0;
  for (int j = n - m + 1; j <= n + m; ++j) r /= j;
  return r;
}

static void quat_rot(const double* q, double* R) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

void split_f32(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// ---------------------------------------------------------------------------
// geometry construction
// ---------------------------------------------------------------------------

int validate(const sbio_spheroid* sph, int32_t M, const sbio_options* o) {
  if (!sph || !o) return set_error(SBIO_EINVAL, "null spheroid array or options");
  if (M < 1) return set_error(SBIO_EINVAL, "M = %d: need at least one spheroid", M);
  if (o->p < 1 || o->p > SBIO_MAX_P) return set_error(SBIO_EINVAL, "p = %d outside [1, %d]", o->p, SBIO_MAX_P);
  const int nphi = o->n_phi ? o->n_phi : 2 * (o->p + 1);
  if (nphi < 2 * o->p || nphi > 4096) return set_error(SBIO_EINVAL, "n_phi = %d must be in [2p, 4096]", nphi);
  if (!(o->near_factor > 0.0) || !std::isfinite(o->near_factor))
    return set_error(SBIO_EINVAL, "near_factor must be positive and finite");
  if (o->far_upsample != 1) return set_error(SBIO_ENOTSUP, "far_upsample = %d: only 1 is implemented", o->far_upsample);
  if (o->precision != SBIO_FP64 && o->precision != SBIO_MIXED)
    return set_error(SBIO_EINVAL, "precision %d unknown", o->precision);
  if ((int64_t)M * (o->p + 1) * nphi > (int64_t)INT32_MAX / 2)
    return set_error(SBIO_EINVAL, "too many nodes");
  for (int i = 0; i < M; ++i) {
    const sbio_spheroid& s = sph[i];
    if (s.kind != SBIO_PROLATE && s.kind != SBIO_OBLATE) return set_error(SBIO_EINVAL, "particle %d: kind %d", i, s.kind);
    if (!(s.A > 0.0) || !(s.C > 0.0) || !std::isfinite(s.A) || !std::isfinite(s.C))
      return set_error(SBIO_EINVAL, "particle %d: semi-axes must be positive", i);
    if (s.kind == SBIO_PROLATE && !(s.C > s.A * (1.0 + 1e-9)))
      return set_error(SBIO_EINVAL, "particle %d: prolate needs C > A (spheres are not supported)", i);
    if (s.kind == SBIO_OBLATE && !(s.C < s.A * (1.0 - 1e-9)))
      return set_error(SBIO_EINVAL, "particle %d: oblate needs C < A (spheres are not supported)", i);
    const double ar = std::max(s.A, s.C) / std::min(s.A, s.C);
    if (!(ar <= kMaxAspectRatio))
      return set_error(SBIO_EINVAL, "particle %d: aspect ratio %g above the supported %g", i, ar, kMaxAspectRatio);
    const double qn = std::sqrt(s.quat[0] * s.quat[0] + s.quat[1] * s.quat[1] + s.quat[2] * s.quat[2] + s.quat[3] * s.quat[3]);
    if (!(std::fabs(qn - 1.0) <= 1e-6)) return set_error(SBIO_EINVAL, "particle %d: quaternion norm %g", i, qn);
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(s.center[k])) return set_error(SBIO_EINVAL, "particle %d: centre not finite", i);
  }
  return SBIO_OK;
}

int build_host(GeomHost& h, const sbio_spheroid* sph, int32_t M, const sbio_options* o) {
  h.M = M;
  h.p = o->p;
  h.n_v = o->p + 1;
  h.n_phi = o->n_phi ? o->n_phi : 2 * (o->p + 1);
  h.G = h.n_v * h.n_phi;
  h.N = (int64_t)M * h.G;
  h.near_factor = o->near_factor;
  h.precision = o->precision;
  h.parts.resize(M);
  for (int i = 0; i < M; ++i) {
    const sbio_spheroid& s = sph[i];
    PartGeom& P = h.parts[i];
    std::memset(&P, 0, sizeof(P));
    P.kind = s.kind;
    P.A = s.A;
    P.C = s.C;
    P.sgn = (s.kind == SBIO_PROLATE) ? -1.0 : 1.0;
    P.a = (s.kind == SBIO_PROLATE) ? std::sqrt((s.C - s.A) * (s.C + s.A)) : std::sqrt((s.A - s.C) * (s.A + s.C));
    P.u0 = s.C / P.a;
    double q[4];
    const double qn = std::sqrt(s.quat[0] * s.quat[0] + s.quat[1] * s.quat[1] + s.quat[2] * s.quat[2] + s.quat[3] * s.quat[3]);
    for (int k = 0; k < 4; ++k) q[k] = s.quat[k] / qn;
    quat_rot(q, P.R);
    for (int k = 0; k < 3; ++k) P.c[k] = s.center[k];
  }
  // nodes
  std::vector<double> gv, gw;
  gauss_legendre(h.n_v, gv, gw);
  h.xyz.resize(h.N * 3);
  h.nrm.resize(h.N * 3);
  h.w.resize(h.N);
  for (int i = 0; i < M; ++i) {
    const PartGeom& P = h.parts[i];
    for (int j = 0; j < h.n_v; ++j) {
      const double v = gv[j], sv = std::sqrt(std::max(0.0, (1.0 - v) * (1.0 + v)));
      // dS = a^2 sqrt(u0^2 + sgn v^2) sqrt(u0^2 + sgn) dv dphi = A sqrt(C^2 + sgn a^2 v^2) dv dphi
      const double dsf = P.A * std::sqrt(P.C * P.C * (P.kind == SBIO_PROLATE ? (1.0 - v * v) : 1.0) +
                                         (P.kind == SBIO_PROLATE ? P.A * P.A * v * v : P.a * P.a * v * v));
      for (int k = 0; k < h.n_phi; ++k) {
        const double ph = 2.0 * kPi * k / h.n_phi;
        const double xl[3] = {P.A * sv * std::cos(ph), P.A * sv * std::sin(ph), P.C * v};
        double nl[3] = {xl[0] / (P.A * P.A), xl[1] / (P.A * P.A), xl[2] / (P.C * P.C)};
        const double nn = std::sqrt(nl[0] * nl[0] + nl[1] * nl[1] + nl[2] * nl[2]);
        for (int c = 0; c < 3; ++c) nl[c] /= nn;
        const int64_t t = (int64_t)i * h.G + (int64_t)j * h.n_phi + k;
        for (int r = 0; r < 3; ++r) {
          h.xyz[t * 3 + r] = P.c[r] + P.R[r * 3 + 0] * xl[0] + P.R[r * 3 + 1] * xl[1] + P.R[r * 3 + 2] * xl[2];
          h.nrm[t * 3 + r] = P.R[r * 3 + 0] * nl[0] + P.R[r * 3 + 1] * nl[1] + P.R[r * 3 + 2] * nl[2];
        }
        h.w[t] = gw[j] * (2.0 * kPi / h.n_phi) * dsf;
      }
    }
  }
  return SBIO_OK;
}

// Near sets on the device.  One thread per target loops over the particles
// in ascending order: an FP32 bounding-sphere prefilter, then the FP64 sphere
// test and (for candidates) the exact point-to-spheroid distance; near iff
// below near_factor x the source's major semi-axis (strict).  Targets are the
// geometry's nodes (G nodes per particle; a node's own particle is skipped and
// heads its skip list) or arbitrary points (G = 0: no own particle).  A target
// is inside a spheroid when the ellipsoid form is below 1 - inside_tol.
// Count pass: near particles per target and the smallest target lying inside
// a spheroid.  Fill pass: the target's near pairs at its offset (ascending
// source) and its far skip list (own and near particles ascending, then a
// sentinel) at its CSR offset.  `order` (may be null) maps thread k to target
// order[k]: spatially sorted points keep a warp's candidate particles alike.
__global__ void __launch_bounds__(128) near_sets_kernel(int M, int G, int64_t N, const PartGeom* __restrict__ parts,
                                                        const int32_t* __restrict__ order,
                                                        const float4* __restrict__ sph,
                                                        const double* __restrict__ xyz, double near_factor,
                                                        double inside_tol, int fill, int32_t* __restrict__ count,
                                                        unsigned long long* __restrict__ overlap_min,
                                                        const int64_t* __restrict__ pair_off,
                                                        int32_t* __restrict__ pair_t, int32_t* __restrict__ pair_s,
                                                        const int32_t* __restrict__ skip_ptr,
                                                        int32_t* __restrict__ skip_idx) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t t = order ? (int64_t)order[k] : k;
  const int own = G > 0 ? (int)(t / G) : -1;
  const double x0 = xyz[t * 3 + 0], x1 = xyz[t * 3 + 1], x2 = xyz[t * 3 + 2];
  const float y0 = (float)x0, y1 = (float)x1, y2 = (float)x2;
  int c = 0;
  const int64_t po = fill ? pair_off[t] : 0;
  int32_t so = fill ? skip_ptr[t] : 0;
  bool own_done = own < 0;
  for (int i = 0; i < M; ++i) {
    if (i == own) continue;
    // FP32 prefilter against a sphere enlarged by a relative 1e-4 and an
    // absolute 1e-3 over the FP64 test's radius (rmax + threshold): it only
    // drops particles the FP64 test below drops too
    const float4 b = sph[i];
    const float e0 = y0 - b.x, e1 = y1 - b.y, e2 = y2 - b.z;
    if (fmaf(e2, e2, fmaf(e1, e1, e0 * e0)) > b.w) continue;
    const PartGeom& P = parts[i];
    const double rmax = fmax(P.A, P.C), thr = near_factor * rmax;
    const double d0 = x0 - P.c[0], d1 = x1 - P.c[1], d2 = x2 - P.c[2];
    const double dc = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (dc - rmax >= thr) continue;
    const double xl = P.R[0] * d0 + P.R[3] * d1 + P.R[6] * d2;
    const double yl = P.R[1] * d0 + P.R[4] * d1 + P.R[7] * d2;
    const double zl = P.R[2] * d0 + P.R[5] * d1 + P.R[8] * d2;
    const double rho = hypot(xl, yl), az = fabs(zl);
    const double f = (rho / P.A) * (rho / P.A) + (az / P.C) * (az / P.C);
    if (f < 1.0 - inside_tol) {
      if (!fill) atomicMin(overlap_min, (unsigned long long)t);
      continue;
    }
    // the spheroid holds the ball of radius min(A, C), so an outside point is
    // at most dc - min(A, C) from it: below the threshold (with a relative
    // margin of 1e-12) the pair is near without the exact distance
    if (!(dc - fmin(P.A, P.C) < thr * (1.0 - 1e-12))) {
      const double dist =
          (P.C >= P.A) ? ellipse_distance_hd(P.C, P.A, az, rho) : ellipse_distance_hd(P.A, P.C, rho, az);
      if (!(dist < thr)) continue;
    }
    if (fill) {
      pair_t[po + c] = (int32_t)t;
      pair_s[po + c] = i;
      if (!own_done && own < i) {
        skip_idx[so++] = own;
        own_done = true;
      }
      skip_idx[so++] = i;
    }
    ++c;
  }
  if (fill) {
    if (!own_done) skip_idx[so++] = own;
    skip_idx[so] = INT32_MAX;   // sentinel
  } else {
    count[t] = c;
  }
}

// Near sets of n targets (device positions xyz, G nodes per particle or 0 for
// points; order_host: optional processing order of the targets) on `st`:
// runs the count pass, returns SBIO_EOVERLAP (nodes) or
// SBIO_EINVAL (points) with *inside the smallest target inside a spheroid,
// allocates the skip lists through alloc_skip (CSR offsets of n + 1 entries
// and the lists), runs the fill pass, and returns the pairs sorted by
// (source kind, source, target) with the number on prolate sources and the
// near count per target.  Synchronises `st`.
int device_near_sets(sbio_geom* g, const double* xyz, int64_t n, int G, double inside_tol,
                     const std::vector<int32_t>* order_host, cudaStream_t st,
                     const std::function<int(const std::vector<int32_t>&, int32_t**, int32_t**)>& alloc_skip,
                     std::vector<int32_t>& pair_t, std::vector<int32_t>& pair_s, int64_t* n_pro,
                     std::vector<int32_t>& cnt, int64_t* inside) {
  const GeomHost& h = g->h;
  const int M = h.M;
  *inside = -1;
  pair_t.clear();
  pair_s.clear();
  cnt.assign(n, 0);
  *n_pro = 0;
  if (n == 0) {
    int32_t *sp = nullptr, *si = nullptr;
    return alloc_skip(std::vector<int32_t>(1, 0), &sp, &si);
  }
  int rc = SBIO_OK;
  // transient buffers, freed on `st` before returning
  std::vector<void*> scratch;
  auto tmp = [&](void** ptr, size_t bytes) -> int {
    *ptr = nullptr;
    if (bytes == 0) return SBIO_OK;
    if (cudaMallocAsync(ptr, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return set_error(SBIO_ENOMEM, "near-set scratch (%zu bytes) failed", bytes);
    }
    scratch.push_back(*ptr);
    return SBIO_OK;
  };
  struct Release {
    std::vector<void*>& v;
    cudaStream_t s;
    ~Release() {
      for (void* q : v) cudaFreeAsync(q, s);
    }
  } release{scratch, st};
  int32_t* dcount = nullptr;
  unsigned long long* dovl = nullptr;
  if ((rc = tmp((void**)&dcount, (size_t)n * sizeof(int32_t)))) return rc;
  if ((rc = tmp((void**)&dovl, sizeof(unsigned long long)))) return rc;
  SBIO_CUDA_TRY(cudaMemsetAsync(dovl, 0xff, sizeof(unsigned long long), st));
  // per particle: FP32 centre and the squared prefilter radius
  std::vector<float4> sph_h(M);
  for (int i = 0; i < M; ++i) {
    const PartGeom& P = h.parts[i];
    const double rmax = std::max(P.A, P.C);
    const double rcut = (rmax + h.near_factor * rmax) * (1.0 + 1e-4) + 1e-3;
    sph_h[i] = make_float4((float)P.c[0], (float)P.c[1], (float)P.c[2], (float)(rcut * rcut));
  }
  float4* dsph = nullptr;
  if ((rc = tmp((void**)&dsph, (size_t)M * sizeof(float4)))) return rc;
  SBIO_CUDA_TRY(cudaMemcpyAsync(dsph, sph_h.data(), (size_t)M * sizeof(float4), cudaMemcpyHostToDevice, st));
  int32_t* dorder = nullptr;
  if (order_host) {
    if ((int64_t)order_host->size() != n) return set_error(SBIO_EINVAL, "near-set order of wrong length");
    if ((rc = tmp((void**)&dorder, (size_t)n * sizeof(int32_t)))) return rc;
    SBIO_CUDA_TRY(cudaMemcpyAsync(dorder, order_host->data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  }
  const unsigned blocks = (unsigned)((n + 127) / 128);
  const PartGeom* dparts = g->d.parts;
  near_sets_kernel<<<blocks, 128, 0, st>>>(M, G, n, dparts, dorder, dsph, xyz, h.near_factor, inside_tol, 0, dcount,
                                           dovl, nullptr, nullptr, nullptr, nullptr, nullptr);
  SBIO_CUDA_TRY(cudaGetLastError());
  unsigned long long ovl = 0;
  SBIO_CUDA_TRY(cudaMemcpyAsync(cnt.data(), dcount, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SBIO_CUDA_TRY(cudaMemcpyAsync(&ovl, dovl, sizeof(ovl), cudaMemcpyDeviceToHost, st));
  SBIO_CUDA_TRY(cudaStreamSynchronize(st));
  if (ovl != ~0ull) {
    *inside = (int64_t)ovl;
    return G > 0 ? SBIO_EOVERLAP : SBIO_EINVAL;
  }
  // offsets: pairs per target; skip lists (near [+ own] + sentinel) per target
  const int extra = G > 0 ? 2 : 1;
  std::vector<int64_t> poff(n + 1, 0);
  std::vector<int32_t> sptr(n + 1, 0);
  for (int64_t t = 0; t < n; ++t) {
    poff[t + 1] = poff[t] + cnt[t];
    if ((int64_t)sptr[t] + cnt[t] + extra > INT32_MAX) return set_error(SBIO_EINVAL, "skip lists exceed 2^31 entries");
    sptr[t + 1] = sptr[t] + cnt[t] + extra;
  }
  const int64_t P = poff[n];
  int64_t* dpoff = nullptr;
  int32_t *dpt = nullptr, *dps = nullptr, *skip_ptr = nullptr, *skip_idx = nullptr;
  if ((rc = tmp((void**)&dpoff, poff.size() * sizeof(int64_t)))) return rc;
  SBIO_CUDA_TRY(cudaMemcpyAsync(dpoff, poff.data(), poff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if ((rc = alloc_skip(sptr, &skip_ptr, &skip_idx))) return rc;
  if ((rc = tmp((void**)&dpt, (size_t)P * sizeof(int32_t)))) return rc;
  if ((rc = tmp((void**)&dps, (size_t)P * sizeof(int32_t)))) return rc;
  near_sets_kernel<<<blocks, 128, 0, st>>>(M, G, n, dparts, dorder, dsph, xyz, h.near_factor, inside_tol, 1, nullptr,
                                           nullptr, dpoff, dpt, dps, skip_ptr, skip_idx);
  SBIO_CUDA_TRY(cudaGetLastError());
  std::vector<int32_t> pt(P), ps(P);
  if (P > 0) {
    SBIO_CUDA_TRY(cudaMemcpyAsync(pt.data(), dpt, P * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SBIO_CUDA_TRY(cudaMemcpyAsync(ps.data(), dps, P * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  }
  SBIO_CUDA_TRY(cudaStreamSynchronize(st));
  // counting sort by (source kind, source); targets stay ascending per source
  std::vector<int64_t> num(M, 0);
  for (int64_t k = 0; k < P; ++k) num[ps[k]]++;
  std::vector<int64_t> base(M, 0);
  int64_t acc = 0;
  for (int kind = SBIO_PROLATE; kind <= SBIO_OBLATE; ++kind)
    for (int i = 0; i < M; ++i)
      if (h.parts[i].kind == kind) {
        base[i] = acc;
        acc += num[i];
        if (kind == SBIO_PROLATE) *n_pro += num[i];
      }
  pair_t.assign(P, 0);
  pair_s.assign(P, 0);
  for (int64_t k = 0; k < P; ++k) {
    const int64_t dst = base[ps[k]]++;
    pair_t[dst] = pt[k];
    pair_s[dst] = ps[k];
  }
  return SBIO_OK;
}

template <typename T>
static int upload(sbio_geom* g, T** dst, const T* src, size_t count, const char* what);

// Near pairs (sorted by source kind, source, target), far pair count,
// source tiles and the device skip lists.
static int build_near(sbio_geom* g) {
  GeomHost& h = g->h;
  DevGeom& d = g->d;
  const int M = h.M;
  const int64_t N = h.N;
  int rc;
  if (!d.parts && (rc = upload(g, &d.parts, h.parts.data(), M, "particles"))) return rc;
  if (!d.xyz && (rc = upload(g, &d.xyz, h.xyz.data(), N * 3, "node positions"))) return rc;
  auto alloc_skip = [&](const std::vector<int32_t>& sptr, int32_t** sp, int32_t** si) -> int {
    int r = upload(g, &d.skip_ptr, sptr.data(), sptr.size(), "skip lists");
    if (!r) r = dev_alloc(g, (void**)&d.skip_idx, (size_t)sptr.back() * sizeof(int32_t), "skip lists");
    *sp = d.skip_ptr;
    *si = d.skip_idx;
    return r;
  };
  std::vector<int32_t> cnt;
  int64_t inside = -1;
  // nodes in their natural order (particle-major) are already spatially coherent
  rc = device_near_sets(g, d.xyz, N, h.G, 0.0, nullptr, g->setup_stream, alloc_skip, h.pair_t, h.pair_s,
                        &h.n_pairs_prolate, cnt, &inside);
  if (rc == SBIO_EOVERLAP)
    return set_error(SBIO_EOVERLAP, "node %lld of particle %lld lies inside another spheroid", (long long)inside,
                     (long long)(inside / h.G));
  if (rc) return rc;
  h.far_pairs = 0;
  for (int64_t t = 0; t < N; ++t) h.far_pairs += (int64_t)(M - 1 - cnt[t]) * h.G;
  // far-field source tiles
  h.tiles.clear();
  for (int i = 0; i < M; ++i)
    for (int s0 = 0; s0 < h.G; s0 += kFarTile)
      h.tiles.push_back(make_int4(i, i * h.G + s0, std::min(kFarTile, h.G - s0), 0));
  return SBIO_OK;
}

template <typename T>
static int upload(sbio_geom* g, T** dst, const T* src, size_t count, const char* what) {
  int rc = dev_alloc(g, (void**)dst, count * sizeof(T), what);
  if (rc) return rc;
  if (count) SBIO_CUDA_TRY(cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, g->setup_stream));
  return SBIO_OK;
}

static int build_device(sbio_geom* g) {
  GeomHost& h = g->h;
  DevGeom& d = g->d;
  const int p = h.p, M = h.M, nm = nm_count(p), nc = (p + 1) * (p + 1);
  const int64_t N = h.N;
  int rc;
  if (!d.parts && (rc = upload(g, &d.parts, h.parts.data(), M, "particles"))) return rc;
  if (!d.xyz && (rc = upload(g, &d.xyz, h.xyz.data(), N * 3, "node positions"))) return rc;
  if ((rc = upload(g, &d.nrm, h.nrm.data(), N * 3, "node normals"))) return rc;
  if ((rc = upload(g, &d.w, h.w.data(), N, "node weights"))) return rc;
  // Legendre table at the GL nodes, trig table, modified-basis weights
  std::vector<double> gv, gw;
  gauss_legendre(h.n_v, gv, gw);
  std::vector<double> ptab((size_t)h.n_v * nm), tmp(nm_count(p + 2));
  for (int j = 0; j < h.n_v; ++j) {
    ferrers(gv[j], p, tmp.data());
    for (int n = 0; n <= p; ++n)
      for (int m = 0; m <= n; ++m)
        ptab[(size_t)j * nm + nm_index(n, m)] = std::sqrt((2.0 * n + 1.0) / (4.0 * kPi) * kfact(n, m)) * tmp[nm_index(n, m)];
  }
  if ((rc = upload(g, &d.ptab, ptab.data(), ptab.size(), "Legendre table"))) return rc;
  if ((rc = upload(g, &d.glw, gw.data(), gw.size(), "GL weights"))) return rc;
  std::vector<double> trig((size_t)h.n_phi * (p + 1) * 2);
  for (int k = 0; k < h.n_phi; ++k)
    for (int m = 0; m <= p; ++m) {
      const double ph = 2.0 * kPi * k / h.n_phi;
      trig[((size_t)k * (p + 1) + m) * 2 + 0] = std::cos(m * ph);
      trig[((size_t)k * (p + 1) + m) * 2 + 1] = std::sin(m * ph);
    }
  if ((rc = upload(g, &d.trig, trig.data(), trig.size(), "trig table"))) return rc;
  std::vector<double> sqrtw((size_t)M * h.n_v);
  for (int i = 0; i < M; ++i) {
    const PartGeom& P = h.parts[i];
    for (int j = 0; j < h.n_v; ++j) {
      const double v = gv[j];
      const double c2 = (P.kind == SBIO_PROLATE) ? P.C * P.C * (1.0 - v * v) + P.A * P.A * v * v
                                                 : P.C * P.C + P.a * P.a * v * v;
      sqrtw[(size_t)i * h.n_v + j] = std::sqrt(c2) / P.a;   // sqrt(u0^2 + sgn v^2)
    }
  }
  if ((rc = upload(g, &d.sqrtw, sqrtw.data(), sqrtw.size(), "modified-basis weights"))) return rc;
  // Theorems 1-2 multipliers per particle
  std::vector<double> mult((size_t)M * 4 * nm), dmult((size_t)M * 4 * nm);
  std::vector<double> Pr(nm_count(p + 1)), Qr(nm_count(p + 1));
  for (int i = 0; i < M; ++i) {
    const PartGeom& P = h.parts[i];
    const double u0 = P.u0, sgn = P.sgn, s0 = P.A / P.a, den = u0 * u0 + sgn;
    radial_P(u0, sgn, p + 1, Pr.data());
    radial_Q(u0, sgn, p + 1, Qr.data());
    for (int n = 0; n <= p; ++n)
      for (int m = 0; m <= n; ++m) {
        const double K = kfact(n, m) * ((m & 1) ? -1.0 : 1.0);
        const double pn = Pr[nm_index(n, m)], qn = Qr[nm_index(n, m)];
        const double pn1 = Pr[nm_index(n + 1, m)], qn1 = Qr[nm_index(n + 1, m)];
        const double dp = ((n - m + 1.0) * pn1 - (n + 1.0) * u0 * pn) / den;
        const double dq = (-sgn * (n - m + 1.0) * qn1 - (n + 1.0) * u0 * qn) / den;
        const double extS = P.a * K * s0 * pn;
        const double extD = K * s0 * s0 * dp;
        const double Dp = extD * qn, Dm = K * s0 * s0 * dq * pn;
        double* mm = &mult[(size_t)i * 4 * nm];
        mm[0 * nm + nm_index(n, m)] = extS;
        mm[1 * nm + nm_index(n, m)] = extD;
        mm[2 * nm + nm_index(n, m)] = extS * qn;
        mm[3 * nm + nm_index(n, m)] = 0.5 * (Dp + Dm);
        // normal derivatives on the surface (Theorem 3 and its D' analogue),
        // as d/du of the exterior / interior expansions at u0; the 1/h_u
        // factor is applied per node.  S' = (S'+ + S'-)/2, D' continuous.
        double* dd = &dmult[(size_t)i * 4 * nm];
        dd[0 * nm + nm_index(n, m)] = extS;
        dd[1 * nm + nm_index(n, m)] = extD;
        dd[2 * nm + nm_index(n, m)] = 0.5 * (extS * dq + P.a * K * s0 * qn * dp);
        dd[3 * nm + nm_index(n, m)] = extD * dq;
      }
  }
  if ((rc = upload(g, &d.mult, mult.data(), mult.size(), "multipliers"))) return rc;
  if ((rc = upload(g, &d.dmult, dmult.data(), dmult.size(), "derivative multipliers"))) return rc;
  std::vector<double> normc(nc);
  for (int n = 0; n <= p; ++n)
    for (int m = -n; m <= n; ++m) {
      const int am = m < 0 ? -m : m;
      normc[coef_index(n, m)] = std::sqrt((2.0 * n + 1.0) / (4.0 * kPi) * kfact(n, am)) * (m ? std::sqrt(2.0) : 1.0);
    }
  if ((rc = upload(g, &d.normc, normc.data(), normc.size(), "normalisation"))) return rc;
  // near pairs and far skip lists (own particle + near particles, ascending)
  if ((rc = upload(g, &d.pair_t, h.pair_t.data(), h.pair_t.size(), "near pairs"))) return rc;
  if ((rc = upload(g, &d.pair_s, h.pair_s.data(), h.pair_s.size(), "near pairs"))) return rc;
  // (the far skip lists were written on the device by the near-set kernels)
  if ((rc = upload(g, &d.tiles, h.tiles.data(), h.tiles.size(), "far tiles"))) return rc;
  // 1/k table of the near kernels' Miller sweeps, long enough for the most
  // elongated particle: targets lie on or outside every surface, so u >= u0
  // and the sweep needs at most ceil(19 / mu(u0)) + 2 steps above the top
  // order (mu = atanh(minor / major semi-axis) at u0)
  int inv_len = kInvTable;
  for (const PartGeom& P : h.parts) {
    const int need = miller_extra(P.u0, P.sgn) + 2 * kMaxP + 40;
    inv_len = std::max(inv_len, need);
  }
  std::vector<double> inv(inv_len, 0.0);
  for (int k = 1; k < inv_len; ++k) inv[k] = 1.0 / k;
  inv[0] = (double)inv_len;
  if ((rc = upload(g, &d.inv, inv.data(), inv.size(), "inverse table"))) return rc;
  // FP32 hi/lo target positions and centres for the mixed far field
  std::vector<float4> tgt(N * 2), cen(M * 2);
  for (int64_t t = 0; t < N; ++t) {
    float hi[3], lo[3];
    for (int c = 0; c < 3; ++c) split_f32(h.xyz[t * 3 + c], hi[c], lo[c]);
    tgt[t * 2 + 0] = make_float4(hi[0], hi[1], hi[2], 0.f);
    tgt[t * 2 + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
  }
  for (int i = 0; i < M; ++i) {
    float hi[3], lo[3];
    for (int c = 0; c < 3; ++c) split_f32(h.parts[i].c[c], hi[c], lo[c]);
    cen[i * 2 + 0] = make_float4(hi[0], hi[1], hi[2], 0.f);
    cen[i * 2 + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
  }
  if ((rc = upload(g, &d.tgt32, tgt.data(), tgt.size(), "fp32 targets"))) return rc;
  if ((rc = upload(g, &d.cen32, cen.data(), cen.size(), "fp32 centres"))) return rc;
  // Stokes tables: exterior factor and normalisation to order p+1, the y.f
  // transform grid ((p+2) GL x (2p+4) trapezoid: exact for degree 2p+2)
  {
    const int p1 = p + 1, nm1 = nm_count(p1), nc1 = (p1 + 1) * (p1 + 1);
    std::vector<double> ext((size_t)M * nm1), Pq(nm_count(p1 + 1));
    for (int i = 0; i < M; ++i) {
      const PartGeom& P = h.parts[i];
      radial_P(P.u0, P.sgn, p1, Pq.data());
      for (int n = 0; n <= p1; ++n)
        for (int m = 0; m <= n; ++m)
          ext[(size_t)i * nm1 + nm_index(n, m)] =
              P.a * kfact(n, m) * ((m & 1) ? -1.0 : 1.0) * (P.A / P.a) * Pq[nm_index(n, m)];
    }
    if ((rc = upload(g, &d.st_ext, ext.data(), ext.size(), "Stokes multipliers"))) return rc;
    std::vector<double> nc1v(nc1);
    for (int n = 0; n <= p1; ++n)
      for (int m = -n; m <= n; ++m) {
        const int am = m < 0 ? -m : m;
        nc1v[coef_index(n, m)] = std::sqrt((2.0 * n + 1.0) / (4.0 * kPi) * kfact(n, am)) * (m ? std::sqrt(2.0) : 1.0);
      }
    if ((rc = upload(g, &d.st_normc, nc1v.data(), nc1v.size(), "Stokes normalisation"))) return rc;
    h.n_q = p + 2;
    h.n_f = 2 * p + 4;
    std::vector<double> qv, qw;
    gauss_legendre(h.n_q, qv, qw);
    std::vector<double> qpt((size_t)h.n_q * nm1), ft(nm_count(p1 + 1));
    for (int j = 0; j < h.n_q; ++j) {
      ferrers(qv[j], p1, ft.data());
      for (int n = 0; n <= p1; ++n)
        for (int m = 0; m <= n; ++m)
          qpt[(size_t)j * nm1 + nm_index(n, m)] = std::sqrt((2.0 * n + 1.0) / (4.0 * kPi) * kfact(n, m)) * ft[nm_index(n, m)];
    }
    std::vector<double> qtr((size_t)h.n_f * (p1 + 1) * 2);
    for (int l = 0; l < h.n_f; ++l)
      for (int m = 0; m <= p1; ++m) {
        const double ph = 2.0 * kPi * l / h.n_f;
        qtr[((size_t)l * (p1 + 1) + m) * 2 + 0] = std::cos(m * ph);
        qtr[((size_t)l * (p1 + 1) + m) * 2 + 1] = std::sin(m * ph);
      }
    if ((rc = upload(g, &d.st_qv, qv.data(), qv.size(), "Stokes grid"))) return rc;
    if ((rc = upload(g, &d.st_qw, qw.data(), qw.size(), "Stokes grid"))) return rc;
    if ((rc = upload(g, &d.st_qptab, qpt.data(), qpt.size(), "Stokes grid"))) return rc;
    if ((rc = upload(g, &d.st_qtrig, qtr.data(), qtr.size(), "Stokes grid"))) return rc;
    // self term at u = u0: radial values and derivatives per particle, Ferrers
    // tables at the GL nodes (unnormalised), trig up to order p+1
    std::vector<double> qu((size_t)M * nm1), dqu((size_t)M * nm1), Qr1(nm_count(p1 + 1));
    for (int i = 0; i < M; ++i) {
      const PartGeom& P = h.parts[i];
      radial_Q(P.u0, P.sgn, p1 + 1, Qr1.data());
      const double den = P.u0 * P.u0 + P.sgn;
      for (int n = 0; n <= p1; ++n)
        for (int m = 0; m <= n; ++m) {
          qu[(size_t)i * nm1 + nm_index(n, m)] = Qr1[nm_index(n, m)];
          dqu[(size_t)i * nm1 + nm_index(n, m)] =
              (-P.sgn * (n - m + 1.0) * Qr1[nm_index(n + 1, m)] - (n + 1.0) * P.u0 * Qr1[nm_index(n, m)]) / den;
        }
    }
    std::vector<double> fP((size_t)h.n_v * nm1), fV((size_t)h.n_v * nm1), fF((size_t)h.n_v * nm1);
    std::vector<double> fr(nm_count(p1 + 2));
    for (int j = 0; j < h.n_v; ++j) {
      const double v = gv[j], sv = std::sqrt((1.0 - v) * (1.0 + v));
      ferrers(v, p1 + 1, fr.data());
      for (int n = 0; n <= p1; ++n)
        for (int m = 0; m <= n; ++m) {
          const double Pn = fr[nm_index(n, m)], Pn1 = fr[nm_index(n + 1, m)];
          fP[(size_t)j * nm1 + nm_index(n, m)] = Pn;
          // sqrt(1-v^2) dP/dv from eq. (derivative) on the cut; GL nodes have sv > 0
          fV[(size_t)j * nm1 + nm_index(n, m)] = ((n + 1.0) * v * Pn - (n - m + 1.0) * Pn1) / sv;
          fF[(size_t)j * nm1 + nm_index(n, m)] = m * Pn / sv;
        }
    }
    std::vector<double> tr1((size_t)h.n_phi * (p1 + 1) * 2);
    for (int k = 0; k < h.n_phi; ++k)
      for (int m = 0; m <= p1; ++m) {
        const double ph = 2.0 * kPi * k / h.n_phi;
        tr1[((size_t)k * (p1 + 1) + m) * 2 + 0] = std::cos(m * ph);
        tr1[((size_t)k * (p1 + 1) + m) * 2 + 1] = std::sin(m * ph);
      }
    if ((rc = upload(g, &d.st_qu0, qu.data(), qu.size(), "Stokes self radial"))) return rc;
    if ((rc = upload(g, &d.st_dqu0, dqu.data(), dqu.size(), "Stokes self radial"))) return rc;
    if ((rc = upload(g, &d.st_fP, fP.data(), fP.size(), "Stokes self Ferrers"))) return rc;
    if ((rc = upload(g, &d.st_fV, fV.data(), fV.size(), "Stokes self Ferrers"))) return rc;
    if ((rc = upload(g, &d.st_fF, fF.data(), fF.size(), "Stokes self Ferrers"))) return rc;
    if ((rc = upload(g, &d.st_trig1, tr1.data(), tr1.size(), "Stokes self trig"))) return rc;
    if ((rc = upload(g, &d.st_glv, gv.data(), gv.size(), "GL nodes"))) return rc;
    if ((rc = dev_alloc(g, (void**)&d.st_coef, (size_t)M * 4 * nc1 * sizeof(double), "Stokes coefficients"))) return rc;
    if ((rc = dev_alloc(g, (void**)&d.st_src64, (size_t)N * 8 * sizeof(double), "Stokes fp64 sources"))) return rc;
    if ((rc = dev_alloc(g, (void**)&d.st_src32, (size_t)N * 2 * sizeof(float4), "Stokes fp32 sources"))) return rc;
    // Stokes double layer: exterior D factor to order p+1, FP32 normals, 13
    // folded expansions per particle
    std::vector<double> extd((size_t)M * nm1), Pr2(nm_count(p1 + 1));
    for (int i = 0; i < M; ++i) {
      const PartGeom& P = h.parts[i];
      radial_P(P.u0, P.sgn, p1 + 1, Pr2.data());
      const double s0 = P.A / P.a, den = P.u0 * P.u0 + P.sgn;
      for (int n = 0; n <= p1; ++n)
        for (int m = 0; m <= n; ++m) {
          const double dp = ((n - m + 1.0) * Pr2[nm_index(n + 1, m)] - (n + 1.0) * P.u0 * Pr2[nm_index(n, m)]) / den;
          extd[(size_t)i * nm1 + nm_index(n, m)] = kfact(n, m) * ((m & 1) ? -1.0 : 1.0) * s0 * s0 * dp;
        }
    }
    if ((rc = upload(g, &d.sdl_ext, extd.data(), extd.size(), "Stokes DL multipliers"))) return rc;
    std::vector<float4> n32(N);
    for (int64_t t = 0; t < N; ++t)
      n32[t] = make_float4((float)h.nrm[t * 3 + 0], (float)h.nrm[t * 3 + 1], (float)h.nrm[t * 3 + 2], 0.f);
    if ((rc = upload(g, &d.nrm32, n32.data(), n32.size(), "fp32 normals"))) return rc;
    if ((rc = dev_alloc(g, (void**)&d.sdl_coef, (size_t)M * 13 * nc1 * sizeof(double), "Stokes DL coefficients")))
      return rc;
  }
  // workspaces
  if ((rc = dev_alloc(g, (void**)&d.src64, (size_t)N * 8 * sizeof(double), "fp64 sources"))) return rc;
  if ((rc = dev_alloc(g, (void**)&d.src32, (size_t)N * 2 * sizeof(float4), "fp32 sources"))) return rc;
  if ((rc = dev_alloc(g, (void**)&d.alpha, (size_t)M * nc * sizeof(double), "near S coefficients"))) return rc;
  if ((rc = dev_alloc(g, (void**)&d.beta, (size_t)M * nc * sizeof(double), "near D coefficients"))) return rc;
  if ((rc = dev_alloc(g, (void**)&d.alpha32, (size_t)M * nc * sizeof(float), "near S coefficients (FP32)"))) return rc;
  if ((rc = dev_alloc(g, (void**)&d.beta32, (size_t)M * nc * sizeof(float), "near D coefficients (FP32)"))) return rc;
  if ((rc = dev_alloc(g, (void**)&d.host_in, (size_t)3 * M * nc * sizeof(double), "host staging"))) return rc;
  if ((rc = dev_alloc(g, (void**)&d.host_out, (size_t)3 * N * sizeof(double), "host staging"))) return rc;
  SBIO_CUDA_TRY(cudaStreamSynchronize(g->setup_stream));
  return SBIO_OK;
}

static void free_geom(sbio_geom* g) {
  if (!g) return;
  tree_free(g->tree);   // host tables only; its device arrays are in g->allocs
  g->tree = nullptr;
  if (g->near_stream) {
    cudaStreamSynchronize(g->near_stream);
    cudaStreamDestroy(g->near_stream);
    g->near_stream = nullptr;
  }
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  g->ev_fork = g->ev_join = nullptr;
  if (g->async_alloc) {
    for (void* p : g->allocs) cudaFreeAsync(p, g->setup_stream);
    g->allocs.clear();
  }
  for (int k = 0; k < 4; ++k)
    if (g->ev[k]) {
      cudaEventDestroy(g->ev[k]);
      g->ev[k] = nullptr;
    }
  for (void* p : g->allocs) cudaFree(p);
  if (g->ctx) g->ctx->used.fetch_sub(g->bytes);
  g->allocs.clear();
  g->bytes = 0;
}

static int geom_create_impl(sbio_ctx* ctx, const sbio_spheroid* sph, int32_t M, const sbio_options* opts,
                            cudaStream_t stream, bool async_alloc, sbio_geom** out) {
  clear_error();
  if (!ctx || !out) return set_error(SBIO_EINVAL, "null context or output pointer");
  *out = nullptr;
  int rc = validate(sph, M, opts);
  if (rc) return rc;
  SBIO_CUDA_TRY(cudaSetDevice(ctx->device));
  sbio_geom* g = new sbio_geom();
  g->ctx = ctx;
  g->setup_stream = stream;
  g->async_alloc = async_alloc;
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  rc = build_host(g->h, sph, M, opts);
  const auto t1 = clk::now();
  if (!rc) rc = build_near(g);
  const auto t2 = clk::now();
  if (!rc) rc = build_device(g);
  const auto t3 = clk::now();
  g->setup_ms[0] = std::chrono::duration<double, std::milli>(t1 - t0).count();
  g->setup_ms[1] = std::chrono::duration<double, std::milli>(t2 - t1).count();
  g->setup_ms[2] = std::chrono::duration<double, std::milli>(t3 - t2).count();
  if (rc) {
    free_geom(g);
    delete g;
    return rc;
  }
  if (!async_alloc) {
    // near/far overlap resources (the serving engine's geometries run in order)
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&g->near_stream, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      g->overlap = false;
    }
  } else {
    g->overlap = false;
  }
  ctx->n_geoms.fetch_add(1);
  *out = g;
  return SBIO_OK;
}

int geom_create_async(sbio_ctx* ctx, const sbio_spheroid* sph, int32_t M, const sbio_options* opts,
                      cudaStream_t st, sbio_geom** out) {
  return geom_create_impl(ctx, sph, M, opts, st, true, out);
}

void geom_destroy_async(sbio_geom* g, cudaStream_t st) {
  if (!g) return;
  g->setup_stream = st;
  free_geom(g);
  g->ctx->n_geoms.fetch_sub(1);
  delete g;
}

}  // namespace sbio

using namespace sbio;

extern "C" {

const char* sbio_version(void) { return "sbio 0.1 (sm_103a)"; }

const char* sbio_last_error(const sbio_ctx*) { return t_err.c_str(); }

int64_t sbio_launch_count(void) { return g_launches.load(); }

int sbio_ctx_create(int device, size_t mem_budget_bytes, sbio_ctx** out) {
  clear_error();
  if (!out) return set_error(SBIO_EINVAL, "null output pointer");
  *out = nullptr;
  int n = 0;
  SBIO_CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return set_error(SBIO_EINVAL, "device %d of %d", device, n);
  SBIO_CUDA_TRY(cudaSetDevice(device));
  sbio_ctx* c = new sbio_ctx();
  c->device = device;
  c->budget = mem_budget_bytes;
  *out = c;
  return SBIO_OK;
}

int sbio_ctx_destroy(sbio_ctx* ctx) {
  if (!ctx) return SBIO_OK;
  if (ctx->n_geoms.load() != 0) return set_error(SBIO_EINVAL, "context still owns %d geometries", ctx->n_geoms.load());
  delete ctx;
  return SBIO_OK;
}

int sbio_ctx_mem_used(const sbio_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return set_error(SBIO_EINVAL, "null argument");
  *bytes = ctx->used.load();
  return SBIO_OK;
}

int sbio_geom_create(sbio_ctx* ctx, const sbio_spheroid* sph, int32_t M, const sbio_options* opts, void* stream,
                     sbio_geom** out) {
  return geom_create_impl(ctx, sph, M, opts, (cudaStream_t)stream, false, out);
}

int sbio_geom_destroy(sbio_geom* g) {
  clear_error();
  if (!g) return SBIO_OK;
  if (g->n_target_sets.load() > 0)
    return set_error(SBIO_EINVAL, "geometry still has %d target set(s); destroy them first", g->n_target_sets.load());
  cudaSetDevice(g->ctx->device);
  cudaDeviceSynchronize();
  free_geom(g);
  g->ctx->n_geoms.fetch_sub(1);
  delete g;
  return SBIO_OK;
}

int sbio_geom_info(const sbio_geom* g, int64_t* n_targets, int64_t* n_near_pairs, int64_t* n_far_pairs,
                   size_t* device_bytes) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (n_targets) *n_targets = g->h.N;
  if (n_near_pairs) *n_near_pairs = (int64_t)g->h.pair_t.size();
  if (n_far_pairs) *n_far_pairs = g->h.far_pairs;
  if (device_bytes) *device_bytes = g->bytes;
  return SBIO_OK;
}

int sbio_geom_nodes(const sbio_geom* g, double* xyz, double* normal, double* weight) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (xyz) std::memcpy(xyz, g->h.xyz.data(), g->h.xyz.size() * sizeof(double));
  if (normal) std::memcpy(normal, g->h.nrm.data(), g->h.nrm.size() * sizeof(double));
  if (weight) std::memcpy(weight, g->h.w.data(), g->h.w.size() * sizeof(double));
  return SBIO_OK;
}

int sbio_geom_near_pairs(const sbio_geom* g, int32_t* target, int32_t* source) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (target) std::memcpy(target, g->h.pair_t.data(), g->h.pair_t.size() * sizeof(int32_t));
  if (source) std::memcpy(source, g->h.pair_s.data(), g->h.pair_s.size() * sizeof(int32_t));
  return SBIO_OK;
}

int sbio_geom_enable_timing(sbio_geom* g, int32_t on) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  if (on && !g->ev[0])
    for (int k = 0; k < 4; ++k) SBIO_CUDA_TRY(cudaEventCreate(&g->ev[k]));
  g->timing = on != 0;
  return SBIO_OK;
}

int sbio_geom_phase_times(sbio_geom* g, double* ms_synth, double* ms_near, double* ms_far) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (!g->timing) return set_error(SBIO_EINVAL, "timing not enabled");
  float t[3] = {0.f, 0.f, 0.f};
  SBIO_CUDA_TRY(cudaEventSynchronize(g->ev[3]));
  for (int k = 0; k < 3; ++k) SBIO_CUDA_TRY(cudaEventElapsedTime(&t[k], g->ev[k], g->ev[k + 1]));
  if (ms_synth) *ms_synth = t[0];
  if (ms_near) *ms_near = t[1];
  if (ms_far) *ms_far = t[2];
  return SBIO_OK;
}

int sbio_geom_setup_times(const sbio_geom* g, double* host_ms, double* near_ms, double* device_ms) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (host_ms) *host_ms = g->setup_ms[0];
  if (near_ms) *near_ms = g->setup_ms[1];
  if (device_ms) *device_ms = g->setup_ms[2];
  return SBIO_OK;
}

int sbio_geom_set_overlap(sbio_geom* g, int32_t on) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (on && !g->near_stream) return set_error(SBIO_ENOTSUP, "this geometry has no overlap stream");
  g->overlap = on != 0;
  return SBIO_OK;
}

int sbio_geom_set_precision(sbio_geom* g, int32_t precision) {
  if (!g) return set_error(SBIO_EINVAL, "null geometry");
  if (precision != SBIO_FP64 && precision != SBIO_MIXED) return set_error(SBIO_EINVAL, "precision %d", precision);
  g->h.precision = precision;
  return SBIO_OK;
}

}  // extern "C"
