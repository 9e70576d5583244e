// FP32 fused multiply-add rate of the device, measured: the denominator the fused solver's
// roofline is reported against is SMs x 128 FP32 lanes x 2 flop x clock, and this confirms it
// on the part at hand, both for the scalar FFMA and for the paired f32x2 form the solver's
// butterflies use.  Every thread runs 16 independent multiply-add chains (enough to cover the
// pipe latency at full occupancy); the values stay bounded (x <- 0.999 x + 1e-3).
#include <cuda_runtime.h>

#include "bccb.h"
#include "common.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ int g_fma_sink;  // written only if a result is impossible, so the work cannot be dropped

template <bool PAIRED>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
  if constexpr (PAIRED) {
    // the chains stay packed in 64-bit registers for the whole loop
    unsigned long long av, bv, v[kChains / 2];
    asm("mov.b64 %0, {%1,%2};" : "=l"(av) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1,%2};" : "=l"(bv) : "f"(b), "f"(b));
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) asm("mov.b64 %0, {%1,%2};" : "=l"(v[k]) : "f"(x[2 * k]), "f"(x[2 * k + 1]));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kChains / 2; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[k]) : "l"(av), "l"(bv));
    }
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) asm("mov.b64 {%0,%1}, %2;" : "=f"(x[2 * k]), "=f"(x[2 * k + 1]) : "l"(v[k]));
  } else {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) atomicAdd(&g_fma_sink, 1);  // the chains converge to 1: never taken
}

}  // namespace

extern "C" int bccb_fp32_fma_rate(int paired, int iters, void* cuda_stream, double* tflops_out) {
  if (!tflops_out || iters < 1) return BCCB_ERR_INVALID_ARG;
  *tflops_out = 0.0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BCCB_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return BCCB_ERR_CUDA;
  const dim3 grid(sms * kBlocksPerSm);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return BCCB_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BCCB_ERR_CUDA;
  }
  auto launch = [&]() {
    if (paired)
      fma_rate_kernel<true><<<grid, kThreads, 0, st>>>(iters, 0.999f, 1e-3f);
    else
      fma_rate_kernel<false><<<grid, kThreads, 0, st>>>(iters, 0.999f, 1e-3f);
  };
  int status = BCCB_OK;
  double best = 0.0;
  launch();  // warm-up (clocks, code load)
  for (int rep = 0; rep < 3 && status == BCCB_OK; ++rep) {
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      status = BCCB_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kChains * (double)iters * (double)grid.x * kThreads;
    if (ms > 0.f && flops / (ms * 1e-3) * 1e-12 > best) best = flops / (ms * 1e-3) * 1e-12;
  }
  if (status == BCCB_OK && cudaGetLastError() != cudaSuccess) status = BCCB_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops_out = best;
  return status;
}
