// FP64 throughput microbenchmarks: the denominators of the FP64 form's fraction of peak.
//
// GB300's FP64 rate is far below its 16-bit tensor rate, and whether the FP64 tensor
// instruction (DMMA, mma.sync m8n8k4 f64) or the plain FP64 FMA pipe (DFMA) is faster on
// this part decides which one the FP64 updates should use.  Both kernels keep every SM
// busy with independent dependency chains so that the pipe, not latency, is the limit:
//   dfma_kernel : each thread carries kChains independent FMA chains (2 flops per FMA).
//   dmma_kernel : each warp carries kChains independent m8n8k4 accumulators (2*8*8*4 =
//                 512 flops per instruction).
// The results feed only the measurement; no factorization uses these kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tqr.h"
#include "tqr_internal.h"

namespace tqr {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) dfma_kernel(int iters, double seed, double *sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 0.001 * (threadIdx.x + c);
  const double x = 1.0 - 1e-9, y = 1e-9;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) sink[threadIdx.x] = s;  // never true: keeps the chains alive
}

__global__ void __launch_bounds__(kPeakThreads) dmma_kernel(int iters, double seed, double *sink) {
  double acc[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c][0] = acc[c][1] = 0.0;
  const double a = seed + 1e-3 * (threadIdx.x & 31), b = 1e-6;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(acc[c][0]), "+d"(acc[c][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c][0] + acc[c][1];
  if (s == 12345.678) sink[threadIdx.x] = s;
}

// Times one launch (after one warm-up launch) with CUDA events; returns TFLOP/s or < 0.
template <typename K>
double time_kernel(K kern, int grid, int iters, double flops_per_iter_thread, double *sink, cudaStream_t st) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
  kern<<<grid, kPeakThreads, 0, st>>>(iters / 8, 1.0, sink);
  count_launch();
  cudaEventRecord(e0, st);
  kern<<<grid, kPeakThreads, 0, st>>>(iters, 1.0, sink);
  count_launch();
  cudaEventRecord(e1, st);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                  cudaGetLastError() == cudaSuccess && ms > 0.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return -1.0;
  const double flops = flops_per_iter_thread * iters * static_cast<double>(grid) * kPeakThreads;
  return flops / (ms * 1e-3) / 1e12;
}

}  // namespace
}  // namespace tqr

extern "C" int tqr_fp64_peak(double *dfma_tflops, double *dmma_tflops, void *stream) {
  using namespace tqr;
  if (!dfma_tflops) return -1;
  if (!dmma_tflops) return -2;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    set_error("tqr_fp64_peak: no device");
    return TQR_ECUDA;
  }
  double *sink = nullptr;
  if (cudaMalloc(&sink, kPeakThreads * sizeof(double)) != cudaSuccess) return TQR_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = nsm * 4;  // 4 CTAs of 8 warps per SM
  // DFMA: 2 flops per FMA, kChains FMAs per iteration and thread
  *dfma_tflops = time_kernel(dfma_kernel, grid, 8192, 2.0 * kChains, sink, st);  // 2.0e10 flops
  // DMMA: 512 flops per warp-wide instruction = 16 per thread, kChains per iteration
  *dmma_tflops = time_kernel(dmma_kernel, grid, 2048, 16.0 * kChains, sink, st);  // 4.1e10 flops
  cudaFree(sink);
  if (*dfma_tflops < 0 || *dmma_tflops < 0) {
    set_error("tqr_fp64_peak: kernel launch or timing failed");
    return TQR_ECUDA;
  }
  return TQR_OK;
}
