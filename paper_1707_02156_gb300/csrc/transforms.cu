// SH transforms and Wigner rotation kernels (Sec. 1.1, Sec. 2.1, App. A, App. B).
//
// Synthesis is split into a Legendre step (per order m, a contraction over the degree n with the
// normalised Legendre table of the target grid) and a phi step (per latitude, a real inverse DFT of
// length 2P+2 that uses phi_{k+P+1} = phi_k + pi to evaluate even and odd orders once for two
// longitudes).  Analysis runs the same two steps in the opposite order with the weighted table.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace bie {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(long long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

template <typename CT, typename R>
__global__ void k_leg_synth(const CT* __restrict__ coef, const long long* __restrict__ field_off,
                            long long coef_stride, long long nfield, int p, const R* __restrict__ T, int nj,
                            R* __restrict__ H, int dphi) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long per_field = (long long)(p + 1) * nj;
  if (idx >= nfield * per_field) return;
  long long f = idx / per_field;
  int r = (int)(idx - f * per_field);
  int m = r / nj;
  int j = r - m * nj;
  const CT* c = coef + (field_off ? field_off[f] : f * coef_stride);
  R re = 0, im = 0;
  const R* Tm = T + leg_row(p, m, m, nj) + j;
  for (int n = m; n <= p; ++n) {
    R t = Tm[(long long)(n - m) * nj];
    int base = n * (n + 1);
    re += (R)c[base + m] * t;
    if (m > 0) im += (R)c[base - m] * t;
  }
  if (dphi == 1) {  // multiply by i m
    R t = re;
    re = -(R)m * im;
    im = (R)m * t;
  } else if (dphi == 2) {  // multiply by -m^2
    re *= -(R)(m * m);
    im *= -(R)(m * m);
  }
  R* h = H + ((f * (p + 1) + m) * (long long)nj + j) * 2;
  h[0] = re;
  h[1] = im;
}

template <typename R, typename OT>
__global__ void k_phi_synth(const R* __restrict__ H, long long nfield, int p, int P, const R* __restrict__ cs,
                            OT* __restrict__ out, const long long* __restrict__ out_off, long long out_stride) {
  const int nj = P + 1, nk = 2 * P + 2, half = P + 1;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long per_field = (long long)nj * half;
  if (idx >= nfield * per_field) return;
  long long f = idx / per_field;
  int r = (int)(idx - f * per_field);
  int j = r / half;
  int k = r - j * half;
  const R* h = H + (f * (p + 1) * (long long)nj + j) * 2;
  R ev = h[0], od = 0;  // m = 0 term (cos 0 = 1, imaginary part of h_0 is zero for real fields)
  for (int m = 1; m <= p; ++m) {
    R hr = h[(long long)m * nj * 2], hi = h[(long long)m * nj * 2 + 1];
    R c = cs[((long long)m * nk + k) * 2], s = cs[((long long)m * nk + k) * 2 + 1];
    R v = 2 * (hr * c - hi * s);
    if (m & 1)
      od += v;
    else
      ev += v;
  }
  OT* o = out + (out_off ? out_off[f] : f * out_stride) + (long long)j * nk;
  o[k] = (OT)(ev + od);
  o[k + half] = (OT)(ev - od);
}

// F[f][m][j] = sum_k g[j][k] e^{-i m phi_k}
__global__ void k_phi_analyze(const double* __restrict__ grid, const long long* __restrict__ grid_off,
                              long long grid_stride, long long nfield, int P, int p_out,
                              const double* __restrict__ cs, double* __restrict__ F) {
  const int nj = P + 1, nk = 2 * P + 2;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long per_field = (long long)(p_out + 1) * nj;
  if (idx >= nfield * per_field) return;
  long long f = idx / per_field;
  int r = (int)(idx - f * per_field);
  int m = r / nj;
  int j = r - m * nj;
  const double* g = grid + (grid_off ? grid_off[f] : f * grid_stride) + (long long)j * nk;
  double re = 0, im = 0;
  for (int k = 0; k < nk; ++k) {
    double v = g[k];
    re += v * cs[((long long)m * nk + k) * 2];
    im -= v * cs[((long long)m * nk + k) * 2 + 1];
  }
  double* o = F + ((f * (p_out + 1) + m) * (long long)nj + j) * 2;
  o[0] = re;
  o[1] = im;
}

// coef(n, m) = sum_j A[m][n][j] F[m][j]
__global__ void k_leg_analyze(const double* __restrict__ F, long long nfield, int P, int p_out,
                              const double* __restrict__ A, double* __restrict__ coef,
                              const long long* __restrict__ coef_off, long long coef_stride) {
  const int nj = P + 1;
  const int nc = (p_out + 1) * (p_out + 2) / 2;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nfield * nc) return;
  long long f = idx / nc;
  int r = (int)(idx - f * nc);
  // r enumerates (m, n) with m <= n in the table's row order
  int m = 0;
  while (r >= p_out + 1 - m) {
    r -= p_out + 1 - m;
    ++m;
  }
  int n = m + r;
  const double* a = A + leg_row(p_out, m, n, nj);
  const double* Fm = F + (f * (p_out + 1) + m) * (long long)nj * 2;
  double re = 0, im = 0;
  for (int j = 0; j < nj; ++j) {
    re += a[j] * Fm[2 * j];
    im += a[j] * Fm[2 * j + 1];
  }
  double* c = coef + (coef_off ? coef_off[f] : f * coef_stride);
  c[n * (n + 1) + m] = re;
  if (m > 0) c[n * (n + 1) - m] = im;
}

// Analysis on the field's own grid (degree p), one block per (field, order m): the phi transform
// F_m(theta_j) of the block's order, one warp per latitude with the lanes across the longitudes
// (coalesced loads, shuffle reduction), then the contraction with the weighted Legendre table for
// n = m..p, one warp per degree with the lanes across the latitudes.
constexpr int kAnaThreads = 512;  // 16 warps: about two latitudes, then two degrees, per warp at p = 32

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Several degree groups in one launch: block ranges per group, arguments by value.
__global__ void __launch_bounds__(kAnaThreads) k_analyze_fused(AnaGroups G, const double* __restrict__ grid,
                                                               double* __restrict__ coef) {
  __shared__ double F[2 * (BIE_MAX_P + 1)];
  AnaGroup Gr = G.g[0];
#pragma unroll
  for (int i = 1; i < kMaxAnaGroups; ++i)
    if (i < G.n && (long long)blockIdx.x >= G.g[i].begin) Gr = G.g[i];
  const int p = Gr.p;
  const long long* __restrict__ grid_off = Gr.grid_off;
  const long long* __restrict__ coef_off = Gr.coef_off;
  const double* __restrict__ cs = Gr.cs;
  const double* __restrict__ A = Gr.A;
  const int nj = p + 1, nk = 2 * p + 2;
  const long long bl = (long long)blockIdx.x - Gr.begin;
  const long long f = bl / (p + 1);
  const int m = (int)(bl - f * (p + 1));
  const double* src = grid + grid_off[f];
  const double* c = cs + (long long)m * nk * 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < nj; j += nw) {
    const double* row = src + (long long)j * nk;
    double re = 0, im = 0;
    for (int k = lane; k < nk; k += 32) {
      const double v = row[k];
      re += v * c[2 * k];
      im -= v * c[2 * k + 1];
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) {
      F[2 * j] = re;
      F[2 * j + 1] = im;
    }
  }
  __syncthreads();
  double* out = coef + coef_off[f];
  for (int n = m + warp; n <= p; n += nw) {
    const double* a = A + leg_row(p, m, n, nj);
    double re = 0, im = 0;
    for (int j = lane; j < nj; j += 32) {
      re += a[j] * F[2 * j];
      im += a[j] * F[2 * j + 1];
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) {
      out[n * (n + 1) + m] = re;
      if (m > 0) out[n * (n + 1) - m] = im;
    }
  }
}

constexpr int kRotB = 16;  // targets (longitudes) per rotation block

// One block per (drop, latitude a, degree n, chunk of kRotB longitudes b).
// Stage: real blocks C (n+1)^2 and S n^2 of the latitude, and g = e^{i m alpha_b} f_n^m for the
// chunk; then Re g'_{m'} = sum_m C[m'][m] Re g_m,  Im g'_{m'} = sum_m S[m'-1][m-1] Im g_m.
template <typename CT, typename R>
__global__ void k_rotate(const CT* __restrict__ coef, const long long* __restrict__ field_off, int ncomp,
                         int p, const R* __restrict__ blocks, long long blk_stride, int na, int nb,
                         const R* __restrict__ ph, R* __restrict__ out, long long out_drop_stride) {
  extern __shared__ unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  const int nbch = (nb + kRotB - 1) / kRotB;
  long long item = blockIdx.x;
  const int bc = (int)(item % nbch);
  item /= nbch;
  const int n = (int)(item % (p + 1));
  item /= (p + 1);
  const int a = (int)(item % na);
  const long long ld = item / na;
  const int b0 = bc * kRotB;
  const int nbh = min(kRotB, nb - b0);
  const int w = 2 * n + 1;
  const int nC = (n + 1) * (n + 1), nS = n * n;
  R* sC = sm;
  R* sS = sC + nC;
  R* sG = sS + nS;  // [bb][c][w]: entries 0..n = Re g_m, n+1..2n = Im g_m (m = 1..n)
  const R* blk = blocks + (long long)a * blk_stride;
  long long boff = 0;
  for (int k = 0; k < n; ++k) boff += (long long)(k + 1) * (k + 1) + (long long)k * k;
  for (int i = threadIdx.x; i < nC + nS; i += blockDim.x) sC[i] = blk[boff + i];
  const int ng = nbh * ncomp;
  for (int i = threadIdx.x; i < ng * (n + 1); i += blockDim.x) {
    int m = i % (n + 1);
    int g = i / (n + 1);
    int c = g % ncomp;
    int bb = g / ncomp;
    const CT* cf = coef + field_off[ld * ncomp + c];
    R fr = (R)cf[n * (n + 1) + m];
    R fi = m > 0 ? (R)cf[n * (n + 1) - m] : (R)0;
    R cr = 1, ci = 0;
    if (ph) {
      cr = ph[((long long)m * nb + (b0 + bb)) * 2];
      ci = ph[((long long)m * nb + (b0 + bb)) * 2 + 1];
    }
    sG[g * w + m] = fr * cr - fi * ci;
    if (m > 0) sG[g * w + n + m] = fr * ci + fi * cr;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ng * w; i += blockDim.x) {
    int o = i % w;
    int g = i / w;
    int c = g % ncomp;
    int bb = g / ncomp;
    const R* G = sG + g * w;
    R acc = 0;
    int dst;
    if (o <= n) {  // Re g'_{o}
      for (int m = 0; m <= n; ++m) acc += sC[m * (n + 1) + o] * G[m];
      dst = n * (n + 1) + o;
    } else {  // Im g'_{mp}, mp = o - n
      int mp = o - n;
      for (int m = 1; m <= n; ++m) acc += sS[(m - 1) * n + (mp - 1)] * G[n + m];
      dst = n * (n + 1) - mp;
    }
    long long t = (long long)a * nb + b0 + bb;
    out[ld * out_drop_stride + (t * ncomp + c) * (long long)((p + 1) * (p + 1)) + dst] = acc;
  }
}

__global__ void k_phase(double* __restrict__ coef, long long nfield, int p, double gamma) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long per = (long long)(p + 1) * (p + 1);
  if (idx >= nfield * per) return;
  long long f = idx / per;
  int r = (int)(idx - f * per);
  int n = 0;
  while ((n + 1) * (n + 1) <= r) ++n;
  int m = r - n * (n + 1);
  if (m <= 0) return;  // the thread owning Re f_n^m (m > 0) rotates the pair
  double* c = coef + f * per;
  double re = c[n * (n + 1) + m], im = c[n * (n + 1) - m];
  double s, co;
  sincos(m * gamma, &s, &co);
  c[n * (n + 1) + m] = re * co - im * s;
  c[n * (n + 1) - m] = re * s + im * co;
}

}  // namespace

template <typename CT, typename R>
int launch_leg_synth(const CT* coef, const long long* field_off, long long coef_stride, long long nfield, int p,
                     const R* T, int nj, R* H, int dphi, cudaStream_t s) {
  long long n = nfield * (long long)(p + 1) * nj;
  if (n == 0) return BIE_OK;
  k_leg_synth<CT, R><<<blocks_for(n), kThreads, 0, s>>>(coef, field_off, coef_stride, nfield, p, T, nj, H, dphi);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R, typename OT>
int launch_phi_synth(const R* H, long long nfield, int p, int P, const R* cs, OT* out, const long long* out_off,
                     long long out_stride, cudaStream_t s) {
  long long n = nfield * (long long)(P + 1) * (P + 1);
  if (n == 0) return BIE_OK;
  k_phi_synth<R, OT><<<blocks_for(n), kThreads, 0, s>>>(H, nfield, p, P, cs, out, out_off, out_stride);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_analyze(const double* grid, const long long* grid_off, long long grid_stride, long long nfield, int P,
                   int p_out, const double* cs, const double* A, double* F, double* coef,
                   const long long* coef_off, long long coef_stride, cudaStream_t s) {
  long long n1 = nfield * (long long)(p_out + 1) * (P + 1);
  if (n1 == 0) return BIE_OK;
  k_phi_analyze<<<blocks_for(n1), kThreads, 0, s>>>(grid, grid_off, grid_stride, nfield, P, p_out, cs, F);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  long long n2 = nfield * (long long)(p_out + 1) * (p_out + 2) / 2;
  k_leg_analyze<<<blocks_for(n2), kThreads, 0, s>>>(F, nfield, P, p_out, A, coef, coef_off, coef_stride);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_analyze_fused(const std::vector<AnaGroup>& groups, const double* grid, double* coef, cudaStream_t s) {
  for (size_t g0 = 0; g0 < groups.size(); g0 += kMaxAnaGroups) {
    AnaGroups G{};
    G.n = (int)std::min<size_t>(kMaxAnaGroups, groups.size() - g0);
    long long nblk = 0;
    for (int i = 0; i < G.n; ++i) {
      G.g[i] = groups[g0 + i];
      if (G.g[i].p > BIE_MAX_P) return BIE_EINVAL;
      G.g[i].begin = nblk;
      nblk += G.g[i].nfield * (G.g[i].p + 1);
    }
    if (nblk == 0) continue;
    if (nblk > 0x7fffffffLL) return BIE_EINVAL;
    k_analyze_fused<<<(unsigned)nblk, kAnaThreads, 0, s>>>(G, grid, coef);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
  }
  return BIE_OK;
}

template <typename CT, typename R>
int launch_rotate(const CT* coef, const long long* field_off, int ncomp, long long ndrop, int p, const R* blocks,
                  long long blk_stride, int na, int nb, const R* ph, R* out, long long out_drop_stride,
                  cudaStream_t s) {
  const int nbch = (nb + kRotB - 1) / kRotB;
  long long nblk = ndrop * na * (long long)(p + 1) * nbch;
  if (nblk == 0) return BIE_OK;
  size_t smem = sizeof(R) * ((size_t)(p + 1) * (p + 1) + (size_t)p * p + (size_t)kRotB * ncomp * (2 * p + 1));
  static thread_local bool attr_set[2] = {false, false};
  if (smem > 48 * 1024 && !attr_set[sizeof(R) == 8]) {
    BIE_CUDA_TRY(cudaFuncSetAttribute(k_rotate<CT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set[sizeof(R) == 8] = true;
  }
  if (nblk > 0x7fffffffLL) return BIE_EINVAL;
  k_rotate<CT, R><<<(unsigned)nblk, 128, smem, s>>>(coef, field_off, ncomp, p, blocks, blk_stride, na, nb, ph, out,
                                                    out_drop_stride);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_phase(double* coef, long long nfield, int p, double gamma, cudaStream_t s) {
  long long n = nfield * (long long)(p + 1) * (p + 1);
  if (n == 0 || gamma == 0.0) return BIE_OK;
  k_phase<<<blocks_for(n), kThreads, 0, s>>>(coef, nfield, p, gamma);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

// explicit instantiations
template int launch_leg_synth<double, double>(const double*, const long long*, long long, long long, int,
                                              const double*, int, double*, int, cudaStream_t);
template int launch_leg_synth<double, float>(const double*, const long long*, long long, long long, int,
                                             const float*, int, float*, int, cudaStream_t);
template int launch_leg_synth<float, float>(const float*, const long long*, long long, long long, int,
                                            const float*, int, float*, int, cudaStream_t);
template int launch_phi_synth<double, double>(const double*, long long, int, int, const double*, double*,
                                              const long long*, long long, cudaStream_t);
template int launch_phi_synth<float, float>(const float*, long long, int, int, const float*, float*,
                                            const long long*, long long, cudaStream_t);
template int launch_phi_synth<float, double>(const float*, long long, int, int, const float*, double*,
                                             const long long*, long long, cudaStream_t);
template int launch_rotate<double, double>(const double*, const long long*, int, long long, int, const double*,
                                           long long, int, int, const double*, double*, long long, cudaStream_t);
template int launch_rotate<double, float>(const double*, const long long*, int, long long, int, const float*,
                                          long long, int, int, const float*, float*, long long, cudaStream_t);

}  // namespace bie
