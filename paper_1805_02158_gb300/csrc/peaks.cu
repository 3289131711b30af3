// Throughput microbenchmarks of the arithmetic units the hot path is bound by: FP32 FMA,
// scalar and packed f32x2 (the NLM's distance and accumulation arithmetic), the EX2
// special-function unit (its weights) and FP64 FMA (the SVD-MPE solve). Each thread runs independent
// dependency chains long enough that issue, not latency, limits them (the iteration loop
// is unrolled so that loop overhead is a few percent of the issue slots); the grid fills
// every SM. Used by the benchmark to put the derived peaks beside measured ones.
#include <cuda_runtime.h>

#include "red.h"
#include "runtime.h"

namespace red {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_fp32_fma(float *out, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-7f + c;
  const float m = 0.999999f, b = 1e-7f;
#pragma unroll 8
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.f) out[threadIdx.x] = s;   // keeps the chains alive
}

// Packed FP32 (fma.rn.f32x2, sm_100 and later): each instruction does two lane FMAs on a
// 64-bit register pair; counted as two lane operations.
__global__ void __launch_bounds__(256) k_fp32x2_fma(float *out, float seed) {
  unsigned long long a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    const float lo = seed + threadIdx.x * 1e-7f + c, hi = lo + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[c]) : "f"(lo), "f"(hi));
  }
  unsigned long long m, b;
  asm("mov.b64 %0, {%1, %2};" : "=l"(m) : "f"(0.999999f), "f"(0.999998f));
  asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(1e-7f), "f"(2e-7f));
#pragma unroll 8
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[c]) : "l"(m), "l"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[c]));
    s += lo + hi;
  }
  if (s == 12345.f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ex2(float *out, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed * 1e-3f + c * 1e-4f;
#pragma unroll 8
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
      a[c] = y * -0.25f;   // stays in a small range
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_fp64_fma(double *out, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-9 + c;
  const double m = 0.999999999, b = 1e-9;
#pragma unroll 8
  for (int i = 0; i < kIters / 16; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.0) out[threadIdx.x] = s;
}

template <class Launch>
double time_launch(Launch &&launch, cudaStream_t s) {
  cudaEvent_t e0, e1;
  CUDA_OK(cudaEventCreate(&e0));
  CUDA_OK(cudaEventCreate(&e1));
  launch();   // warm-up
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaEventRecord(e0, s));
  for (int r = 0; r < 5; ++r) launch();
  CUDA_OK(cudaEventRecord(e1, s));
  CUDA_OK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / 5.0;
}

}  // namespace
}  // namespace red

using namespace red;

extern "C" red_status red_measure_peaks(double *fp32_fma_lane_ops, double *ex2_lane_ops,
                                        double *fp64_fma_lane_ops,
                                        double *fp32x2_fma_lane_ops, void *stream) {
  return guarded([&] {
    CHECK_ARG(fp32_fma_lane_ops && ex2_lane_ops && fp64_fma_lane_ops && fp32x2_fma_lane_ops,
              "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    CUDA_OK(cudaGetDevice(&dev));
    CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    void *buf = nullptr;
    CUDA_OK(cudaMalloc(&buf, 4096));
    const double lanes = (double)blocks * threads * kChains;
    double ms = time_launch([&] { k_fp32_fma<<<blocks, threads, 0, s>>>((float *)buf, 1.f); }, s);
    *fp32_fma_lane_ops = lanes * kIters / (ms * 1e-3);
    ms = time_launch([&] { k_fp32x2_fma<<<blocks, threads, 0, s>>>((float *)buf, 1.f); }, s);
    *fp32x2_fma_lane_ops = 2.0 * lanes * kIters / (ms * 1e-3);
    ms = time_launch([&] { k_ex2<<<blocks, threads, 0, s>>>((float *)buf, 1.f); }, s);
    *ex2_lane_ops = lanes * kIters / (ms * 1e-3);
    ms = time_launch([&] { k_fp64_fma<<<blocks, threads, 0, s>>>((double *)buf, 1.0); }, s);
    *fp64_fma_lane_ops = lanes * (kIters / 16) / (ms * 1e-3);
    count_launches(24);
    CUDA_OK(cudaFree(buf));
    return RED_OK;
  });
}
