// Surface geometry, rotated-grid cache and pair-sum kernels (Table 2, Thm 1, Sec. 2.1-2.3).
#include <cuda_runtime.h>

#include "internal.cuh"

namespace bie {

namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(long long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

__device__ inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// rec[d][0..2] = x, [3..5] = outward normal x_theta x x_phi / W, [6] = wsin[j] * W
__global__ void k_surface(const double* __restrict__ X, const double* __restrict__ Xt,
                          const double* __restrict__ Xp, long long ndrop, int P, const double* __restrict__ wsin,
                          double* __restrict__ rec) {
  const int nk = 2 * P + 2;
  const long long N = (long long)(P + 1) * nk;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ndrop * N) return;
  long long d = idx / N;
  long long q = idx - d * N;
  int j = (int)(q / nk);
  double x[3], xt[3], xp[3], c[3];
  for (int i = 0; i < 3; ++i) {
    x[i] = X[(d * 3 + i) * N + q];
    xt[i] = Xt[(d * 3 + i) * N + q];
    xp[i] = Xp[(d * 3 + i) * N + q];
  }
  cross3(xt, xp, c);
  double W = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  double* r = rec + d * 7 * N;
  for (int i = 0; i < 3; ++i) {
    r[i * N + q] = x[i];
    r[(3 + i) * N + q] = c[i] / W;
  }
  r[6 * N + q] = wsin[j] * W;
}

// cache[t][0..2] = x0 - x', [3..5] = n', [6] = w^s_j W'/sin(theta_j), on the degree-pq grid.
template <typename R>
__global__ void k_rotgeo(const double* __restrict__ X, const double* __restrict__ Xt, const double* __restrict__ Xp,
                         long long ndrop, int ng, int pq, const double* __restrict__ rec_std,
                         const double* __restrict__ wsq, R* __restrict__ cache) {
  const int nk = 2 * pq + 2;
  const long long nq = (long long)(pq + 1) * nk;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = ndrop * ng * nq;
  if (idx >= total) return;
  long long t = idx / nq;
  long long q = idx - t * nq;
  long long ld = t / ng, tl = t - ld * ng;
  int j = (int)(q / nk);
  double x[3], xt[3], xp[3], c[3];
  for (int i = 0; i < 3; ++i) {
    x[i] = X[(t * 3 + i) * nq + q];
    xt[i] = Xt[(t * 3 + i) * nq + q];
    xp[i] = Xp[(t * 3 + i) * nq + q];
  }
  cross3(xt, xp, c);
  double W = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  R* o = cache + t * 7 * nq;
  for (int i = 0; i < 3; ++i) {
    double x0 = rec_std[(ld * 7 + i) * ng + tl];
    o[i * nq + q] = (R)(x0 - x[i]);
    o[(3 + i) * nq + q] = (R)(c[i] / W);
  }
  o[6 * nq + q] = (R)(wsq[j] * W);
}

template <typename R>
__device__ inline R rsqrt_(R v);
template <>
__device__ inline double rsqrt_<double>(double v) {
  return 1.0 / sqrt(v);
}
template <>
__device__ inline float rsqrt_<float>(float v) {
  return rsqrtf(v);
}

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

// One block per target: sum over the nq points of its rotated grid (Thm 1).
template <typename R, int KIND>
__global__ void k_self_pairs(const R* __restrict__ cache, const R* __restrict__ rho, int ng, long long nq,
                             const double* __restrict__ wts, const long long* __restrict__ val_off,
                             double* __restrict__ vals) {
  __shared__ R sh[3 * 32];
  const long long t = blockIdx.x;
  const R* g = cache + t * 7 * nq;
  const R* rh = rho + t * 3 * nq;
  R s0 = 0, s1 = 0, s2 = 0;
  for (long long q = threadIdx.x; q < nq; q += blockDim.x) {
    R x0 = g[q], x1 = g[nq + q], x2 = g[2 * nq + q];
    R w = g[6 * nq + q];
    R r0 = rh[q], r1 = rh[nq + q], r2 = rh[2 * nq + q];
    R rr = x0 * x0 + x1 * x1 + x2 * x2;
    R ri = rsqrt_<R>(rr);
    R xr = x0 * r0 + x1 * r1 + x2 * r2;
    if (KIND == 0) {  // Stokeslet: rho/r + xh (xh.rho)/r^3
      R wi = w * ri;
      R c = wi * xr * ri * ri;
      s0 += wi * r0 + c * x0;
      s1 += wi * r1 + c * x1;
      s2 += wi * r2 + c * x2;
    } else {  // stresslet: -6 (rho.xh)(xh.n) xh / r^5
      R xn = x0 * g[3 * nq + q] + x1 * g[4 * nq + q] + x2 * g[5 * nq + q];
      R ri2 = ri * ri;
      R c = (R)(-6) * w * xr * xn * ri2 * ri2 * ri;
      s0 += c * x0;
      s1 += c * x1;
      s2 += c * x2;
    }
  }
  block_sum3<R>(s0, s1, s2, sh);
  if (threadIdx.x == 0) {
    long long ld = t / ng, tl = t - ld * ng;
    double wt = wts[ld];
    double* v = vals + val_off[ld] + tl;
    v[0] = wt * (double)s0;
    v[ng] = wt * (double)s1;
    v[2 * (long long)ng] = wt * (double)s2;
  }
}

}  // namespace

int launch_surface(const double* X, const double* Xt, const double* Xp, long long ndrop, int P,
                   const double* wsin, double* rec, cudaStream_t s) {
  long long n = ndrop * (long long)(P + 1) * (2 * P + 2);
  if (n == 0) return BIE_OK;
  k_surface<<<blocks_for(n), kThreads, 0, s>>>(X, Xt, Xp, ndrop, P, wsin, rec);
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R>
int launch_rotgeo(const double* X, const double* Xt, const double* Xp, long long ndrop, int ng, int pq,
                  const double* rec_std, const double* wsq, R* cache, cudaStream_t s) {
  long long n = ndrop * ng * (long long)(pq + 1) * (2 * pq + 2);
  if (n == 0) return BIE_OK;
  k_rotgeo<R><<<blocks_for(n), kThreads, 0, s>>>(X, Xt, Xp, ndrop, ng, pq, rec_std, wsq, cache);
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R>
int launch_self_pairs(int kind, const R* cache, const R* rho, long long ndrop, int ng, long long nq,
                      const double* wts, const long long* val_off, double* vals, cudaStream_t s) {
  long long nt = ndrop * ng;
  if (nt == 0) return BIE_OK;
  if (nt > 0x7fffffffLL) return BIE_EINVAL;
  if (kind == 0)
    k_self_pairs<R, 0><<<(unsigned)nt, kThreads, 0, s>>>(cache, rho, ng, nq, wts, val_off, vals);
  else
    k_self_pairs<R, 1><<<(unsigned)nt, kThreads, 0, s>>>(cache, rho, ng, nq, wts, val_off, vals);
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template int launch_rotgeo<double>(const double*, const double*, const double*, long long, int, int, const double*,
                                   const double*, double*, cudaStream_t);
template int launch_rotgeo<float>(const double*, const double*, const double*, long long, int, int, const double*,
                                  const double*, float*, cudaStream_t);
template int launch_self_pairs<double>(int, const double*, const double*, long long, int, long long,
                                       const double*, const long long*, double*, cudaStream_t);
template int launch_self_pairs<float>(int, const float*, const float*, long long, int, long long, const double*,
                                      const long long*, double*, cudaStream_t);

}  // namespace bie
