// Measured issue rates of the pipes the hot path is bound by: FP32 FMA
// (scalar and packed f32x2), the MUFU reciprocal square root, FP64 FMA, and
// the far-field pair's instruction mix with no memory traffic.  These are the
// roofline denominators for kernels that no copy or GEMM benchmark measures:
// the far-field sums are bound by the FP32 and MUFU pipes, the near field by
// the FP64 pipe.
//
// Every kernel runs independent dependency chains (enough per thread to cover
// the pipe latency) over a full-occupancy grid of 8 CTAs x 256 threads per SM,
// with operands the compiler cannot fold (kernel arguments), and stores its
// result only under a data-dependent condition that never holds, so no work
// is removed.  Each kernel is launched once to warm up and then timed with
// CUDA events on a private stream; block 0 also reads %clock64 and
// %globaltimer around its loop to give the SM clock during the run.
#include <cuda_runtime.h>

#include "sbio_internal.cuh"

namespace sbio {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 8;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct ClockProbe {
  unsigned long long c0, t0;
  __device__ void start() {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      t0 = global_ns();
      c0 = clock64();
    }
  }
  __device__ void stop(double* mhz) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const unsigned long long c1 = clock64(), t1 = global_ns();
      if (t1 > t0) *mhz = (double)(c1 - c0) * 1e3 / (double)(t1 - t0);
    }
  }
};

// scalar FP32 FMA: kChains chains of fma(a, b, c) per thread, `iters` rounds
__global__ void __launch_bounds__(kPeakThreads) ffma_kernel(int iters, float b, float c, float* sink, double* mhz) {
  ClockProbe cp;
  cp.start();
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
  }
  cp.stop(mhz);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.2345f) sink[0] = s;
}

// packed f32x2 FMA (two FP32 FMAs per lane per instruction)
__global__ void __launch_bounds__(kPeakThreads) ffma2_kernel(int iters, float b, float c, float* sink, double* mhz) {
  ClockProbe cp;
  cp.start();
  float2 a[kChains];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    }
  }
  cp.stop(mhz);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  if (s == -1.2345f) sink[0] = s;
}

// MUFU reciprocal square root (the far kernels' one special-function op)
__global__ void __launch_bounds__(kPeakThreads) rsqrt_kernel(int iters, float b, float c, float* sink, double* mhz) {
  ClockProbe cp;
  cp.start();
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = b + (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = rsqrt_f32(a[k]);
    }
  }
  cp.stop(mhz);
  float s = c;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.2345f) sink[0] = s;
}

// FP64 FMA
__global__ void __launch_bounds__(kPeakThreads) dfma_kernel(int iters, double b, double c, float* sink, double* mhz) {
  ClockProbe cp;
  cp.start();
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  cp.stop(mhz);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.2345) sink[0] = (float)s;
}

// The packed far pair's arithmetic with the operands in registers: per round
// 11 packed FP32 instructions and 2 MUFU rsqrt, the mix of two S + D pairs
// (targets paired in f32x2), on independent chains so that only the pipes
// bound it.  Counted as 2 pairs per round.
__global__ void __launch_bounds__(kPeakThreads) pairmix_kernel(int iters, float b, float c, float* sink,
                                                                double* mhz) {
  ClockProbe cp;
  cp.start();
  constexpr int kF = 11;
  float2 a[kF];
  float r0 = b + (float)threadIdx.x, r1 = b + 1.f + (float)threadIdx.x;
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kF; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int k = 0; k < kF; ++k) {
        a[k] = __ffma2_rn(a[k], b2, c2);
        if (k == 3) r0 = rsqrt_f32(r0);
        if (k == 8) r1 = rsqrt_f32(r1);
      }
    }
  }
  cp.stop(mhz);
  float s = r0 + r1;
#pragma unroll
  for (int k = 0; k < kF; ++k) s += a[k].x + a[k].y;
  if (s == -1.2345f) sink[0] = s;
}

// The same pair fed from shared memory as the far kernel feeds it: 128
// sources staged once per CTA with every operand duplicated into an f32x2
// pair (five 16-byte loads per source), 8 targets per thread, no tiles, skip
// lists or barriers inside the loop.  Counted as 8 pairs per source per thread.
__global__ void __launch_bounds__(128) pairsmem_kernel(int reps, float b, float c, float* sink, double* mhz) {
  ClockProbe cp;
  cp.start();
  __shared__ float4 sh[5 * 128];
  const int tid = threadIdx.x;
  {
    const float y0 = b * (float)(tid % 7), y1 = c * (float)(tid % 5), y2 = -b * (float)(tid % 3);
    const float yy = y0 * y0 + y1 * y1 + y2 * y2;
    sh[tid * 5 + 0] = make_float4(-2.f * y0, -2.f * y0, -2.f * y1, -2.f * y1);
    sh[tid * 5 + 1] = make_float4(-2.f * y2, -2.f * y2, yy, yy);
    sh[tid * 5 + 2] = make_float4(c, c, -b, -b);
    sh[tid * 5 + 3] = make_float4(b, b, c, c);
    sh[tid * 5 + 4] = make_float4(b, b, 0.f, 0.f);
  }
  __syncthreads();
  constexpr int TP = 4;
  float2 Xp[TP], Yp[TP], Zp[TP], XXp[TP], sS[TP], sD[TP];
#pragma unroll
  for (int k = 0; k < TP; ++k) {
    const float x0 = 3.f + 0.01f * tid + k, x1 = 2.f - 0.01f * k, x2 = 4.f + 0.001f * tid;
    Xp[k] = make_float2(x0, x0 + 0.1f);
    Yp[k] = make_float2(x1, x1 - 0.1f);
    Zp[k] = make_float2(x2, x2 + 0.2f);
    XXp[k] = make_float2(x0 * x0 + x1 * x1 + x2 * x2,
                         (x0 + .1f) * (x0 + .1f) + (x1 - .1f) * (x1 - .1f) + (x2 + .2f) * (x2 + .2f));
    sS[k] = sD[k] = make_float2(0.f, 0.f);
  }
  for (int r = 0; r < reps; ++r) {
#pragma unroll 1
    for (int j = 0; j < 128; ++j) {
      const float4 A = sh[j * 5 + 0], B = sh[j * 5 + 1], Cc = sh[j * 5 + 2], Dd = sh[j * 5 + 3], Ee = sh[j * 5 + 4];
      const float2 mx = make_float2(A.x, A.y), my = make_float2(A.z, A.w), mz = make_float2(B.x, B.y);
      const float2 yy = make_float2(B.z, B.w), q2 = make_float2(Cc.x, Cc.y), ndy = make_float2(Cc.z, Cc.w);
      const float2 dwx = make_float2(Dd.x, Dd.y), dwy = make_float2(Dd.z, Dd.w), dwz = make_float2(Ee.x, Ee.y);
#pragma unroll
      for (int k = 0; k < TP; ++k) {
        const float2 r2 = __ffma2_rn(Xp[k], mx, __ffma2_rn(Yp[k], my, __ffma2_rn(Zp[k], mz, __fadd2_rn(XXp[k], yy))));
        const float2 ri = make_float2(rsqrt_f32(r2.x), rsqrt_f32(r2.y));
        sS[k] = __ffma2_rn(q2, ri, sS[k]);
        const float2 dn = __ffma2_rn(dwx, Xp[k], __ffma2_rn(dwy, Yp[k], __ffma2_rn(dwz, Zp[k], ndy)));
        sD[k] = __ffma2_rn(__fmul2_rn(dn, ri), __fmul2_rn(ri, ri), sD[k]);
      }
    }
  }
  cp.stop(mhz);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < TP; ++k) s += sS[k].x + sS[k].y + sD[k].x + sD[k].y;
  if (s == -1.2345f) sink[0] = s;
}

}  // namespace

}  // namespace sbio

using namespace sbio;

extern "C" int sbio_measure_peaks(int32_t device, sbio_peaks* out) {
  clear_error();
  if (!out) return set_error(SBIO_EINVAL, "null output");
  int n_dev = 0;
  SBIO_CUDA_TRY(cudaGetDeviceCount(&n_dev));
  if (device < 0 || device >= n_dev) return set_error(SBIO_EINVAL, "device %d of %d", device, n_dev);
  SBIO_CUDA_TRY(cudaSetDevice(device));
  int sms = 0;
  SBIO_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  cudaStream_t st = nullptr;
  SBIO_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float* sink = nullptr;
  double* mhz = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) err = cudaMalloc(&sink, sizeof(float));
  if (err == cudaSuccess) err = cudaMalloc(&mhz, 6 * sizeof(double));
  if (err == cudaSuccess) err = cudaMemsetAsync(mhz, 0, 6 * sizeof(double), st);
  const dim3 grid((unsigned)(sms * kPeakCtasPerSm)), block(kPeakThreads);
  const double threads = (double)grid.x * block.x;
  double ms[6] = {0, 0, 0, 0, 0, 0};
  // rounds per thread: each kernel runs for a few milliseconds at full rate
  const int it_f32 = 4096, it_mufu = 512, it_f64 = 512, it_mix = 2048;
  auto timed = [&](int k, auto launch) {
    if (err != cudaSuccess) return;
    launch();   // warm-up
    err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) launch();
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    ms[k] = t;
  };
  timed(0, [&] { ffma_kernel<<<grid, block, 0, st>>>(it_f32, 0.999f, 1e-3f, sink, mhz + 0); });
  timed(1, [&] { ffma2_kernel<<<grid, block, 0, st>>>(it_f32, 0.999f, 1e-3f, sink, mhz + 1); });
  timed(2, [&] { rsqrt_kernel<<<grid, block, 0, st>>>(it_mufu, 1.5f, 0.f, sink, mhz + 2); });
  timed(3, [&] { dfma_kernel<<<grid, block, 0, st>>>(it_f64, 0.999, 1e-3, sink, mhz + 3); });
  timed(4, [&] { pairmix_kernel<<<grid, block, 0, st>>>(it_mix, 0.999f, 1e-3f, sink, mhz + 4); });
  const int reps_smem = 32;
  const dim3 grid_smem((unsigned)(sms * 16));
  timed(5, [&] { pairsmem_kernel<<<grid_smem, 128, 0, st>>>(reps_smem, 0.1f, 0.2f, sink, mhz + 5); });
  count_launch(12);
  double clk[6] = {0, 0, 0, 0, 0, 0};
  if (err == cudaSuccess) err = cudaMemcpy(clk, mhz, sizeof(clk), cudaMemcpyDeviceToHost);
  if (sink) cudaFree(sink);
  if (mhz) cudaFree(mhz);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (err != cudaSuccess) return set_error(SBIO_ECUDA, "peak measurement failed: %s", cudaGetErrorString(err));
  const double s = 1e-3;
  out->sms = sms;
  out->fp32_ffma_tflops = threads * it_f32 * 4 * kChains * 2.0 / (ms[0] * s) / 1e12;
  out->fp32_ffma2_tflops = threads * it_f32 * 4 * kChains * 4.0 / (ms[1] * s) / 1e12;
  out->rsqrt_per_s = threads * it_mufu * 4 * kChains / (ms[2] * s);
  out->fp64_dfma_tflops = threads * it_f64 * kChains * 2.0 / (ms[3] * s) / 1e12;
  out->pairmix_pairs_per_s = threads * it_mix * 4 * 2.0 / (ms[4] * s);
  out->pairsmem_pairs_per_s = (double)grid_smem.x * 128 * reps_smem * 128 * 8.0 / (ms[5] * s);
  double c = 0.0;
  int nc = 0;
  for (double v : clk)
    if (v > 0) {
      c += v;
      ++nc;
    }
  out->sm_clock_mhz = nc ? c / nc : 0.0;
  return SBIO_OK;
}
