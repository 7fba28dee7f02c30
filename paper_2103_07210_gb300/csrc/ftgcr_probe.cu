// Measurement probe of libftgcr: the device's FP64 fused multiply-add rate,
// the ceiling of the FP64 path's arithmetic (its row-solve chains and its
// compensated dot products run on the FP64 pipe).  Off every solve path; a
// benchmark calls it beside the memory-copy peak.
#include <cuda_runtime.h>

#include "../../include/ftgcr.h"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread (covers the pipe latency)
constexpr int kThreads = 256;

// Each thread runs kChains independent chains x <- fma(x, a, b) for `iters`
// iterations.  a and b come from the caller so the compiler cannot fold the
// chains; |a| < 1 keeps every value finite.  One value per thread is written
// out so that the work is not removed.
__global__ void __launch_bounds__(kThreads) k_fma_rate(int iters, double a, double b, double* out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int ftgcr_fp64_fma_rate(int32_t iters, double* tflops, void* stream) {
  if (!tflops || iters < 1 || iters > (1 << 24)) return FTGCR_ERR_ARG;
  *tflops = 0.0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return FTGCR_ERR_CUDA;
  }
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  cudaStream_t st = (cudaStream_t)stream;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FTGCR_OK;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * kThreads) != cudaSuccess) {
    cudaGetLastError();
    return FTGCR_ERR_OOM;
  }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = FTGCR_ERR_CUDA;
  if (!rc) {
    k_fma_rate<<<blocks, kThreads, 0, st>>>(iters < 64 ? iters : 64, 0.5, 0.25, out);  // warm
    cudaEventRecord(e0, st);
    k_fma_rate<<<blocks, kThreads, 0, st>>>(iters, 0.5, 0.25, out);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
      rc = FTGCR_ERR_CUDA;
  }
  if (!rc) *tflops = 2.0 * kChains * (double)iters * blocks * kThreads / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc) cudaGetLastError();
  return rc;
}
