// Small device helpers shared by the kernels of the library.
#pragma once
#include <cuda_runtime.h>

namespace bie {

template <typename R>
__device__ inline R rsqrt_(R v);
// 1/sqrt(v) in FP64 from the FP32 hardware estimate y and one third-order correction: with
// e = 1 - v y^2 (about 2^-22), 1/sqrt(v) = y (1 - e)^(-1/2) = y (1 + e/2 + 3e^2/8 + O(e^3)), so the
// truncated series leaves a relative error of order e^3 (2^-66), below FP64 rounding; e is formed
// with one fused multiply-add from y^2, so its rounding error is 2^-53 absolute and enters the
// result as 2^-54 relative.  Five FP64 operations against seven for two Newton steps.  Outside the
// FP32 exponent range the estimate is unusable and the quotient of the IEEE square root is
// returned instead.
template <>
__device__ inline double rsqrt_<double>(double v) {
  if (!(v > 1e-30 && v < 1e30)) return 1.0 / sqrt(v);
  const double y = (double)rsqrtf((float)v);
  const double e = fma(-v, y * y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}
template <>
__device__ inline float rsqrt_<float>(float v) {
  return rsqrtf(v);
}

// Block-wide sum of three values; the result is valid in thread 0.  sh holds 3 * 32 entries.
template <typename R>
__device__ inline void block_sum3(R& a, R& b, R& c, R* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[w * 3] = a;
    sh[w * 3 + 1] = b;
    sh[w * 3 + 2] = c;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    a = l < nw ? sh[l * 3] : (R)0;
    b = l < nw ? sh[l * 3 + 1] : (R)0;
    c = l < nw ? sh[l * 3 + 2] : (R)0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
  }
}

// Degree n of the packed index r = n(n+1)+m (0 <= r < (p+1)^2).
__device__ inline int degree_of(int r) {
  int n = (int)sqrtf((float)r);
  while (n * n > r) --n;
  while ((n + 1) * (n + 1) <= r) ++n;
  return n;
}

}  // namespace bie
