// Double-float numbers for the FP64-grade kernels that run on the FP32 pipes.
//
// A value is the unevaluated sum h + l of two FP32 numbers (about 44 significant bits).  Sums use
// Knuth's TwoSum and products the FMA-based TwoProduct (error-free transformations); results are
// left unnormalised (|l| may exceed ulp(h)/2 by a few units), which costs no accuracy over the short
// chains of one output; the conversion to double adds the two parts exactly.
#pragma once
#include <cuda_runtime.h>

namespace bie {

struct dff {
  float h, l;
  dff() = default;
  __host__ __device__ constexpr dff(float a, float b) : h(a), l(b) {}
  __host__ __device__ dff(int a) : h((float)a), l(0.0f) {}
  __host__ __device__ dff(double a) : h((float)a), l((float)(a - (double)(float)a)) {}
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ inline dff operator+(dff a, dff b) {
  const float s = a.h + b.h;
  const float v = s - a.h;
  return dff(s, (a.h - (s - v)) + (b.h - v) + a.l + b.l);
}
__device__ inline dff operator-(dff a) { return dff(-a.h, -a.l); }
__device__ inline dff operator-(dff a, dff b) { return a + (-b); }
__device__ inline dff operator*(dff a, dff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return dff(p, e);
}
__device__ inline dff& operator+=(dff& a, dff b) { return a = a + b; }

// a * b + c and a warp shuffle for every arithmetic type of the templated kernels
__device__ inline float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ inline double fmad(double a, double b, double c) { return ::fma(a, b, c); }
__device__ inline dff fmad(dff a, dff b, dff c) { return a * b + c; }
__device__ inline float shfl_down(float v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
__device__ inline double shfl_down(double v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
__device__ inline dff shfl_down(dff v, int off) {
  return dff(__shfl_down_sync(0xffffffffu, v.h, off), __shfl_down_sync(0xffffffffu, v.l, off));
}

}  // namespace bie
