// Allocation-free entry point: on-surface self interaction of a set of
// spheroids (the block-diagonal part of the Laplace S and D apply) for callers
// that must not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not an option -- a solver
// embedded in a framework whose caching allocator (or a pre-reservation of most
// of the device, as some runtimes do at start-up) owns the GPU memory, so a
// private cudaMalloc can fail or fragment the pool; or a loop that has been
// told never to allocate after initialisation.  Such a caller hands over its
// own input and output buffers, and every other byte the kernel touches comes
// from one fixed array that the library reserves in device memory when it is
// loaded.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes (8 MiB).
// Every GPU on which the library's module is loaded holds these 8 MiB until the
// process exits.  Host code never dereferences the array's symbol: its device
// address is looked up once per device with cudaGetSymbolAddress (on the first
// call made with that device current) and cached.
#include <cstring>
#include <mutex>
#include <vector>

#include "sbio_internal.cuh"

namespace sbio {

__global__ void synth_kernel(int p, int n_v, int n_phi, const PartGeom* __restrict__ parts,
                             const double* __restrict__ xyz, const double* __restrict__ nrm,
                             const double* __restrict__ w, const double* __restrict__ ptab,
                             const double* __restrict__ trig, const double* __restrict__ sqrtw,
                             const double* __restrict__ mult, const double* __restrict__ normc,
                             const double* __restrict__ sigma, const double* __restrict__ mu, int write_self,
                             int side, double* __restrict__ S_out, double* __restrict__ D_out,
                             double* __restrict__ src64,
                             float4* __restrict__ src32, double* __restrict__ alpha, double* __restrict__ beta,
                             float* __restrict__ alpha32, float* __restrict__ beta32);

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).  Nothing in the array has to start at zero: every
// call first overwrites the table region and the kernel only writes the
// workspace region, so stale contents from an earlier call are never read.
static int scratch_address(void** out) {
  int dev = 0;
  SBIO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(SBIO_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return set_error(SBIO_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SBIO_OK;
}

// Bump layout of the scratch array (offsets 256-byte aligned).
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

}  // namespace sbio

using namespace sbio;

extern "C" int sbio_apply_self_noalloc(const sbio_spheroid* sph, int32_t M, int32_t p, int32_t n_phi,
                                       const double* sigma_tilde, const double* mu_hat, double* S_out,
                                       double* D_out, void* stream) {
  clear_error();
  if ((sigma_tilde == nullptr) != (S_out == nullptr) || (mu_hat == nullptr) != (D_out == nullptr))
    return set_error(SBIO_EINVAL, "each output must be given exactly when its input is");
  if (!sigma_tilde && !mu_hat) return set_error(SBIO_EINVAL, "nothing to apply");
  sbio_options o;
  o.p = p;
  o.n_phi = n_phi;
  o.near_factor = 1.0;
  o.far_upsample = 1;
  o.precision = SBIO_FP64;
  int rc = validate(sph, M, &o);
  if (rc) return rc;
  GeomHost h;
  rc = build_host(h, sph, M, &o);
  if (rc) return rc;
  const int nm = nm_count(p), nc = (p + 1) * (p + 1);
  const int64_t N = h.N;

  // layout of everything the kernel reads or writes besides the caller's buffers
  Layout L;
  const size_t o_parts = L.take(sizeof(PartGeom) * M);
  const size_t o_xyz = L.take(sizeof(double) * N * 3);
  const size_t o_nrm = L.take(sizeof(double) * N * 3);
  const size_t o_w = L.take(sizeof(double) * N);
  const size_t o_ptab = L.take(sizeof(double) * h.n_v * nm);
  const size_t o_trig = L.take(sizeof(double) * h.n_phi * (p + 1) * 2);
  const size_t o_sqrtw = L.take(sizeof(double) * M * h.n_v);
  const size_t o_mult = L.take(sizeof(double) * M * 4 * nm);
  const size_t o_normc = L.take(sizeof(double) * nc);
  const size_t tables_end = L.off;
  const size_t o_src64 = L.take(sizeof(double) * N * 8);
  const size_t o_src32 = L.take(sizeof(float4) * N * 2);
  const size_t o_alpha = L.take(sizeof(double) * M * nc);
  const size_t o_beta = L.take(sizeof(double) * M * nc);
  if (L.off > kNoAllocScratchBytes)
    return set_error(SBIO_EINVAL,
                     "sbio_apply_self_noalloc: %d spheroids at p = %d need %zu bytes of scratch, more than the "
                     "fixed %zu-byte array; use sbio_geom_create + sbio_apply_laplace_parts instead",
                     M, p, L.off, kNoAllocScratchBytes);

  // host image of the tables (the node data comes from the shared set-up)
  std::vector<unsigned char> img(tables_end, 0);
  std::memcpy(img.data() + o_parts, h.parts.data(), sizeof(PartGeom) * M);
  std::memcpy(img.data() + o_xyz, h.xyz.data(), sizeof(double) * N * 3);
  std::memcpy(img.data() + o_nrm, h.nrm.data(), sizeof(double) * N * 3);
  std::memcpy(img.data() + o_w, h.w.data(), sizeof(double) * N);
  std::vector<double> gv, gw;
  gauss_legendre(h.n_v, gv, gw);
  double* ptab = reinterpret_cast<double*>(img.data() + o_ptab);
  std::vector<double> tmp(nm_count(p + 2));
  for (int j = 0; j < h.n_v; ++j) {
    ferrers(gv[j], p, tmp.data());
    for (int n = 0; n <= p; ++n)
      for (int m = 0; m <= n; ++m)
        ptab[(size_t)j * nm + nm_index(n, m)] = std::sqrt((2.0 * n + 1.0) / (4.0 * kPi) * kfact(n, m)) * tmp[nm_index(n, m)];
  }
  double* trig = reinterpret_cast<double*>(img.data() + o_trig);
  for (int k = 0; k < h.n_phi; ++k)
    for (int m = 0; m <= p; ++m) {
      const double ph = 2.0 * kPi * k / h.n_phi;
      trig[((size_t)k * (p + 1) + m) * 2 + 0] = std::cos(m * ph);
      trig[((size_t)k * (p + 1) + m) * 2 + 1] = std::sin(m * ph);
    }
  double* sqrtw = reinterpret_cast<double*>(img.data() + o_sqrtw);
  double* mult = reinterpret_cast<double*>(img.data() + o_mult);
  std::vector<double> Pr(nm_count(p + 1)), Qr(nm_count(p + 1));
  for (int i = 0; i < M; ++i) {
    const PartGeom& P = h.parts[i];
    for (int j = 0; j < h.n_v; ++j) {
      const double v = gv[j];
      const double c2 = (P.kind == SBIO_PROLATE) ? P.C * P.C * (1.0 - v * v) + P.A * P.A * v * v
                                                 : P.C * P.C + P.a * P.a * v * v;
      sqrtw[(size_t)i * h.n_v + j] = std::sqrt(c2) / P.a;
    }
    const double u0 = P.u0, sgn = P.sgn, s0 = P.A / P.a, den = u0 * u0 + sgn;
    radial_P(u0, sgn, p + 1, Pr.data());
    radial_Q(u0, sgn, p + 1, Qr.data());
    double* mm = mult + (size_t)i * 4 * nm;
    for (int n = 0; n <= p; ++n)
      for (int m = 0; m <= n; ++m) {
        const double K = kfact(n, m) * ((m & 1) ? -1.0 : 1.0);
        const double pn = Pr[nm_index(n, m)], qn = Qr[nm_index(n, m)];
        const double pn1 = Pr[nm_index(n + 1, m)], qn1 = Qr[nm_index(n + 1, m)];
        const double dp = ((n - m + 1.0) * pn1 - (n + 1.0) * u0 * pn) / den;
        const double dq = (-sgn * (n - m + 1.0) * qn1 - (n + 1.0) * u0 * qn) / den;
        const double extS = P.a * K * s0 * pn, extD = K * s0 * s0 * dp;
        mm[0 * nm + nm_index(n, m)] = extS;
        mm[1 * nm + nm_index(n, m)] = extD;
        mm[2 * nm + nm_index(n, m)] = extS * qn;
        mm[3 * nm + nm_index(n, m)] = 0.5 * (extD * qn + K * s0 * s0 * dq * pn);
      }
  }
  double* normc = reinterpret_cast<double*>(img.data() + o_normc);
  for (int n = 0; n <= p; ++n)
    for (int m = -n; m <= n; ++m) {
      const int am = m < 0 ? -m : m;
      normc[coef_index(n, m)] = std::sqrt((2.0 * n + 1.0) / (4.0 * kPi) * kfact(n, am)) * (m ? std::sqrt(2.0) : 1.0);
    }

  // The tables are staged from `img`, which is freed when this call returns.
  // Outside stream capture the pageable copy has read it before the call
  // returns; a captured copy would instead keep the host address and read it
  // at every replay, so calls on a capturing stream are refused (before any
  // other CUDA call).
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SBIO_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(SBIO_EINVAL,
                     "sbio_apply_self_noalloc stages its tables from host memory freed on return; it cannot be "
                     "called on a stream that is being captured");
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  unsigned char* b = static_cast<unsigned char*>(base);
  // pageable source: the copy is staged before the call returns, so `img` may go
  SBIO_CUDA_TRY(cudaMemcpyAsync(b, img.data(), tables_end, cudaMemcpyHostToDevice, st));
  const int nmw = 2 * p + 1;
  const size_t smem = (size_t)(2 * nc + 4 * h.n_v * nmw) * sizeof(double);
  if (smem > 48 * 1024)
    SBIO_CUDA_TRY(cudaFuncSetAttribute(synth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  synth_kernel<<<M, 256, smem, st>>>(
      p, h.n_v, h.n_phi, reinterpret_cast<const PartGeom*>(b + o_parts), reinterpret_cast<const double*>(b + o_xyz),
      reinterpret_cast<const double*>(b + o_nrm), reinterpret_cast<const double*>(b + o_w),
      reinterpret_cast<const double*>(b + o_ptab), reinterpret_cast<const double*>(b + o_trig),
      reinterpret_cast<const double*>(b + o_sqrtw), reinterpret_cast<const double*>(b + o_mult),
      reinterpret_cast<const double*>(b + o_normc), sigma_tilde, mu_hat, 1, 0, S_out, D_out,
      reinterpret_cast<double*>(b + o_src64), reinterpret_cast<float4*>(b + o_src32),
      reinterpret_cast<double*>(b + o_alpha), reinterpret_cast<double*>(b + o_beta), nullptr, nullptr);
  count_launch();
  SBIO_CUDA_TRY(cudaGetLastError());
  return SBIO_OK;
}
