// Surface geometry, rotated-grid cache and pair-sum kernels (Table 2, Thm 1, Sec. 2.1-2.3).
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
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
                         const long long* __restrict__ rec_off, const double* __restrict__ wsq,
                         R* __restrict__ cache) {
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
    double x0 = rec_std[rec_off[ld] + (long long)i * ng + tl];
    o[i * nq + q] = (R)(x0 - x[i]);
    o[(3 + i) * nq + q] = (R)(c[i] / W);
  }
  o[6 * nq + q] = (R)(wsq[j] * W);
}

// Interfacial force f = -2 sigma K n - grad_gamma sigma at grid points (Sec. 1, Table 2), from the
// six derivative fields of x ([3][N] each, order: f, t, p, tt, tp, pp) and of Gamma (f, t, p).
// K = (E N - 2 F M + G L) / (2 W^2) with E = x_p.x_p, F = x_p.x_t, G = x_t.x_t, L = x_pp.n,
// M = x_tp.n, N = x_tt.n, outward n = x_t x x_p / W; sigma = 1 + E_s ln(1 - x_s Gamma) (x_s > 0)
// or 1 - E_s Gamma; grad sigma = [(G s_p - F s_t) x_p + (E s_t - F s_p) x_t] / W^2.
__global__ void k_force(const double* __restrict__ X, const double* __restrict__ Gm, long long N, double es,
                        double xs, double* __restrict__ f) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  double xt[3], xp[3], xtt[3], xtp[3], xpp[3], n[3];
  for (int c = 0; c < 3; ++c) {
    xt[c] = X[(1 * 3 + c) * N + q];
    xp[c] = X[(2 * 3 + c) * N + q];
    xtt[c] = X[(3 * 3 + c) * N + q];
    xtp[c] = X[(4 * 3 + c) * N + q];
    xpp[c] = X[(5 * 3 + c) * N + q];
  }
  cross3(xt, xp, n);
  const double W = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int c = 0; c < 3; ++c) n[c] /= W;
  const double E = xp[0] * xp[0] + xp[1] * xp[1] + xp[2] * xp[2];
  const double F = xp[0] * xt[0] + xp[1] * xt[1] + xp[2] * xt[2];
  const double G = xt[0] * xt[0] + xt[1] * xt[1] + xt[2] * xt[2];
  const double L = xpp[0] * n[0] + xpp[1] * n[1] + xpp[2] * n[2];
  const double M = xtp[0] * n[0] + xtp[1] * n[1] + xtp[2] * n[2];
  const double Nn = xtt[0] * n[0] + xtt[1] * n[1] + xtt[2] * n[2];
  const double W2 = W * W;
  const double K = (E * Nn - 2.0 * F * M + G * L) / (2.0 * W2);
  const double gam = Gm[q], gt = Gm[N + q], gp = Gm[2 * N + q];
  double sigma, ds;
  if (xs > 0.0) {
    sigma = 1.0 + es * log(1.0 - xs * gam);
    ds = -es * xs / (1.0 - xs * gam);
  } else {
    sigma = 1.0 - es * gam;
    ds = -es;
  }
  const double st = ds * gt, sp = ds * gp;
  const double a = (G * sp - F * st) / W2, b = (E * st - F * sp) / W2;
  for (int c = 0; c < 3; ++c) f[c * N + q] = -2.0 * sigma * K * n[c] - (a * xp[c] + b * xt[c]);
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

}  // namespace

int launch_to_float(const double* in, float* out, long long n, cudaStream_t s) {
  if (n == 0) return BIE_OK;
  k_to_float<<<blocks_for(n), kThreads, 0, s>>>(in, out, n);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_force(const double* X, const double* Gm, long long N, double es, double xs, double* f, cudaStream_t s) {
  if (N == 0) return BIE_OK;
  k_force<<<blocks_for(N), kThreads, 0, s>>>(X, Gm, N, es, xs, f);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_surface(const double* X, const double* Xt, const double* Xp, long long ndrop, int P,
                   const double* wsin, double* rec, cudaStream_t s) {
  long long n = ndrop * (long long)(P + 1) * (2 * P + 2);
  if (n == 0) return BIE_OK;
  k_surface<<<blocks_for(n), kThreads, 0, s>>>(X, Xt, Xp, ndrop, P, wsin, rec);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R>
int launch_rotgeo(const double* X, const double* Xt, const double* Xp, long long ndrop, int ng, int pq,
                  const double* rec_std, const long long* rec_off, const double* wsq, R* cache, cudaStream_t s) {
  long long n = ndrop * ng * (long long)(pq + 1) * (2 * pq + 2);
  if (n == 0) return BIE_OK;
  k_rotgeo<R><<<blocks_for(n), kThreads, 0, s>>>(X, Xt, Xp, ndrop, ng, pq, rec_std, rec_off, wsq, cache);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template int launch_rotgeo<double>(const double*, const double*, const double*, long long, int, int, const double*,
                                   const long long*, const double*, double*, cudaStream_t);
template int launch_rotgeo<float>(const double*, const double*, const double*, long long, int, int, const double*,
                                  const long long*, const double*, float*, cudaStream_t);
}  // namespace bie

