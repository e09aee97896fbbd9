// Stokes single layer at arbitrary points (Sec. 4.3 with the Sec. 4.1
// particle-to-target algorithm): velocity by eq. (stokes) for near pairs and
// the Stokeslet quadrature for far pairs (the kernels of the on-surface
// apply, through a view of the geometry's tables whose targets are the
// points), and the pressure p = int P(x, y) . f dS with the printed kernel
// P = r / (4 pi |r|^3): the divergence of the Laplace expansions for near
// pairs (sbio_stokes_points.cuh), the smooth quadrature for far pairs (in
// mixed precision summed by the Stokeslet far kernel in the same pass, in
// FP64 by the kernel here).
#include "sbio_internal.cuh"
#include "sbio_stokes_near.cuh"
#include "sbio_stokes_points.cuh"

struct sbio_targets;

namespace sbio {

stokes_near_launcher stokes_near_lookup_a(int p);
stokes_near_launcher stokes_near_lookup_b(int p);
stokes_near_launcher stokes_near_lookup_c(int p);
stokes_point_near_launcher stokes_point_near_lookup_a(int p);
stokes_point_near_launcher stokes_point_near_lookup_b(int p);
stokes_point_near_launcher stokes_point_near_lookup_c(int p);


namespace {

constexpr double kInv4PiP = 0.07957747154594767;   // 1/(4 pi)

struct alignas(32) pd4 {
  double x, y, z, w;
};

// FP64: one target per thread; sources (y - c, w f_1), (w f_2, w f_3, 0, 0).
__global__ void __launch_bounds__(kFarTile) pressure_far_fp64_kernel(const int4* __restrict__ tiles, int n_tiles,
                                                                     const double* __restrict__ src64,
                                                                     const double* __restrict__ xyz,
                                                                     const PartGeom* __restrict__ parts,
                                                                     const int32_t* __restrict__ skip_ptr,
                                                                     const int32_t* __restrict__ skip_idx, int64_t N,
                                                                     double* __restrict__ p_out) {
  __shared__ pd4 sh[kFarTile * 2];
  const int64_t t = (int64_t)blockIdx.x * kFarTile + threadIdx.x;
  const bool valid = t < N;
  double x = 0, y = 0, z = 0;
  int sp = 0, nxt = INT32_MAX;
  if (valid) {
    x = xyz[t * 3 + 0];
    y = xyz[t * 3 + 1];
    z = xyz[t * 3 + 2];
    sp = skip_ptr[t];
    nxt = skip_idx[sp];
  }
  double acc = 0.0;
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
      const pd4* s = reinterpret_cast<const pd4*>(src64 + (int64_t)(tile.y + threadIdx.x) * 8);
      sh[threadIdx.x * 2 + 0] = s[0];
      sh[threadIdx.x * 2 + 1] = s[1];
    }
    __syncthreads();
    if (!skip) {
      for (int j = 0; j < tile.z; ++j) {
        const pd4 a = sh[j * 2], b = sh[j * 2 + 1];
        const double dx = X - a.x, dy = Y - a.y, dz = Z - a.z;
        const double ri = rsqrt(dx * dx + dy * dy + dz * dz);
        acc = fma(a.w * dx + b.x * dy + b.y * dz, ri * ri * ri, acc);
      }
    }
    __syncthreads();
  }
  if (valid) atomicAdd(p_out + t, acc * kInv4PiP);
}

// FP64 pressure quadrature (the mixed form is summed by the Stokeslet far
// kernel in the same pass as the velocity).
void launch_pressure_far_fp64(const DevGeom& d, const GeomHost& h, int64_t NT, double* pr, cudaStream_t st) {
  if (NT <= 0) return;
  const int nt = (int)h.tiles.size();
  const int64_t tb = (NT + kFarTile - 1) / kFarTile;
  const dim3 grid((unsigned)tb, (unsigned)far_split_count(tb, nt, 0));
  pressure_far_fp64_kernel<<<grid, kFarTile, 0, st>>>(d.tiles, nt, d.st_src64, d.xyz, d.parts, d.skip_ptr,
                                                      d.skip_idx, NT, pr);
  count_launch();
}

}  // namespace
}  // namespace sbio

using namespace sbio;

extern "C" {

int sbio_eval_targets_stokes(sbio_targets* ts, const double* f_tilde, double* u_out, double* p_out, void* stream) {
  clear_error();
  if (!ts || !f_tilde || !u_out) return set_error(SBIO_EINVAL, "null argument");
  sbio_geom* g = nullptr;
  const DevGeom* view = nullptr;
  int64_t T = 0, n_pro = 0, n_pairs = 0;
  int rc = targets_view(ts, &g, &view, &T, &n_pro, &n_pairs);
  if (rc) return rc;
  const GeomHost& h = g->h;
  if (h.p > 20) return set_error(SBIO_ENOTSUP, "Stokes single layer is built for p <= 20 (p = %d)", h.p);
  SBIO_CUDA_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (T == 0) return SBIO_OK;
  SBIO_CUDA_TRY(cudaMemsetAsync(u_out, 0, T * 3 * sizeof(double), st));
  if (p_out) SBIO_CUDA_TRY(cudaMemsetAsync(p_out, 0, T * sizeof(double), st));
  if ((rc = launch_stokes_prep(g, f_tilde, st))) return rc;
  DevGeom v = *view;   // a copy: the near grid cap is per launch
  const bool fork = g->overlap && !g->timing && g->near_stream && n_pairs > 0;
  cudaStream_t ns = fork ? g->near_stream : st;
  SideFork sf;
  if (fork) {
    SBIO_CUDA_TRY(sf.fork(g, st));
    // with the pressure a near pair costs about twice the velocity-only pair
    // the cap was tuned on (four derivative sums per expansion instead of one
    // combined gradient), against a similar far pair: twice the CTAs
    const int cap = h.st_near_ctas_per_sm * (p_out ? 2 : 1);
    v.near_grid_cap = cap > 0 ? cap * sm_count() : 0;
  }
  if (n_pairs > 0) {
    if (p_out) {
      stokes_point_near_launcher nl = stokes_point_near_lookup_a(h.p);
      if (!nl) nl = stokes_point_near_lookup_b(h.p);
      if (!nl) nl = stokes_point_near_lookup_c(h.p);
      if (!nl) return set_error(SBIO_ENOTSUP, "no Stokes point kernel for p = %d", h.p);
      nl(v, n_pro, n_pairs, u_out, p_out, ns);
    } else {
      stokes_near_launcher nl = stokes_near_lookup_a(h.p);
      if (!nl) nl = stokes_near_lookup_b(h.p);
      if (!nl) nl = stokes_near_lookup_c(h.p);
      if (!nl) return set_error(SBIO_ENOTSUP, "no Stokes near-field kernel for p = %d", h.p);
      nl(v, n_pro, n_pairs, v.inv, u_out, ns);
    }
    SBIO_CUDA_TRY(cudaGetLastError());
  }
  const bool fp64 = h.precision == SBIO_FP64;
  if ((rc = launch_stokes_far_on(v, h, T, u_out, fp64 ? nullptr : p_out, st))) return rc;
  if (p_out && fp64) launch_pressure_far_fp64(v, h, T, p_out, st);
  SBIO_CUDA_TRY(cudaGetLastError());
  SBIO_CUDA_TRY(sf.join());
  return SBIO_OK;
}

}  // extern "C"
