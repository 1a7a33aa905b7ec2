// Measured arithmetic rates of the context's GPU, the denominators of the ALU rooflines of the
// pair kernels: FP32 FMA (fma.rn.f32), packed FP32 FMA (fma.rn.f32x2, two lanes per instruction)
// and FP64 FMA.  Each thread runs eight independent chains x <- x*b + c (b = 0.999, c = 0.001, whose
// fixed point 1 keeps every value normal), unrolled so that loop overhead stays below 2% of the
// issue slots.  The grid is eight 256-thread blocks per SM (full occupancy).  Nothing here changes
// a setting of the GPU: the rate is whatever the clocks give while the kernel runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.cuh"

namespace bie {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreadsPk = 256;

__device__ inline unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ inline float2 unpack2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

template <int KIND>
__global__ void __launch_bounds__(kThreadsPk) k_alu_peak(float* __restrict__ sink, int iters, float seed) {
  const float s0 = seed + 1e-6f * (float)(threadIdx.x & 63);
  if (KIND == 0) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = s0 + 0.01f * i;
    const float b = 0.999f, c = 0.001f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], b, c);
    }
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += x[i];
    if (acc == 12345.678f) sink[0] = acc;
  } else if (KIND == 1) {
    unsigned long long x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = pack2(s0 + 0.01f * i, s0 - 0.01f * i);
    const unsigned long long b = pack2(0.999f, 0.999f), c = pack2(0.001f, 0.001f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int i = 0; i < kChains; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(b), "l"(c));
    }
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      const float2 v = unpack2(x[i]);
      acc += v.x + v.y;
    }
    if (acc == 12345.678f) sink[0] = acc;
  } else {
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (double)s0 + 0.01 * i;
    const double b = 0.999, c = 0.001;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], b, c);
    }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += x[i];
    if (acc == 12345.678) sink[0] = (float)acc;
  }
}

}  // namespace
}  // namespace bie

using namespace bie;

extern "C" int bie_alu_peak(bie_ctx* ctx, int which, double* tflops) {
  if (!ctx || !tflops || which < BIE_PEAK_FP32 || which > BIE_PEAK_FP64) {
    set_error("bie_alu_peak: null argument or unknown rate");
    return BIE_EINVAL;
  }
  const int device = ctx_device(ctx);
  BIE_CUDA_TRY(cudaSetDevice(device));
  int sms = 0;
  BIE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int blocks = sms * 8;
  // inner iterations sized for about 10 ms per launch at each unit's nominal rate
  const int iters = which == BIE_PEAK_FP32 ? 8192 : (which == BIE_PEAK_FP32X2 ? 4096 : 128);
  const double fma_per_launch =
      (double)blocks * kThreadsPk * iters * kUnroll * kChains * (which == BIE_PEAK_FP32X2 ? 2.0 : 1.0);
  float* sink = nullptr;
  BIE_CUDA_TRY(cudaMalloc(&sink, sizeof(float)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = BIE_OK;
  double best_ms = 1e30;
  auto launch = [&]() {
    if (which == BIE_PEAK_FP32)
      k_alu_peak<0><<<blocks, kThreadsPk>>>(sink, iters, 0.5f);
    else if (which == BIE_PEAK_FP32X2)
      k_alu_peak<1><<<blocks, kThreadsPk>>>(sink, iters, 0.5f);
    else
      k_alu_peak<2><<<blocks, kThreadsPk>>>(sink, iters, 0.5f);
    count_launch();
    return cudaGetLastError();
  };
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch();  // warm-up
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) best_ms = std::min(best_ms, (double)ms);
  }
  if (e != cudaSuccess) {
    set_error(std::string("bie_alu_peak: ") + cudaGetErrorString(e));
    st = BIE_ECUDA;
  } else {
    *tflops = 2.0 * fma_per_launch / (best_ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}
