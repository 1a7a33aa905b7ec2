// Surfactant transport on the drop surfaces (Eq. surfactant0, Sec. 1.2, Sec. 3): the explicit
// (convection and stretching) and implicit (diffusion) right-hand sides at the grid points, the
// coefficients of the surface Laplacian for the implicit solve, and per-drop surface integrals and
// maxima for the error estimates of Alg. 1.
//
// Surface calculus in the parameters (theta, phi): metric g = [[G, F], [F, E]] with G = x_t.x_t,
// F = x_t.x_p, E = x_p.x_p, W^2 = E G - F^2 and inverse [[E, -F], [-F, G]] / W^2;
//   grad s = g^ij s_j x_i,  div v = g^ij x_i . v_j,  lap s = g^ij (s_ij - x_ij . grad s).
// Points of the surface move with the full velocity u (dx/dt = u), so the rate of Gamma at fixed
// parameters is
//   f_E = -div(Gamma u_tan) + u_tan . grad Gamma + 2 K Gamma (u.n),  f_I = (1/Pe) lap Gamma,
// with the outward normal n and the mean curvature K = (E N - 2 F M + G L) / (2 W^2) (-1/R on a
// sphere), L = x_pp.n, M = x_tp.n, N = x_tt.n.
//
// Field layouts, for a group of nd drops of one degree on the grid of degree P (N points each):
//   X  [6][nd*3][N]  x and its derivatives, order f, t, p, tt, tp, pp
//   U  [3][nd*3][N]  u and its first derivatives, order f, t, p
//   Gm [6][nd][N]    Gamma and its derivatives, order f, t, p, tt, tp, pp
#include <cuda_runtime.h>

#include "internal.cuh"

namespace bie {

namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(long long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

struct V3 {
  double x, y, z;
};
__device__ inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

// component c of vector field block k of a group with nvec vectors per block
__device__ inline V3 load3(const double* F, int k, long long nvec, long long v, long long N, long long q) {
  const double* b = F + ((long long)k * nvec * 3 + v * 3) * N + q;
  return {b[0], b[N], b[2 * N]};
}

struct Metric {
  V3 xt, xp;
  double gtt, gtp, gpp, W;
};

__device__ inline Metric metric(V3 xt, V3 xp) {
  Metric m;
  m.xt = xt;
  m.xp = xp;
  const double G = dot(xt, xt), F = dot(xt, xp), E = dot(xp, xp);
  const double W2 = E * G - F * F;
  m.gtt = E / W2;
  m.gtp = -F / W2;
  m.gpp = G / W2;
  m.W = sqrt(W2);
  return m;
}

__device__ inline V3 grad(const Metric& m, double st, double sp) {
  return (m.gtt * st + m.gtp * sp) * m.xt + (m.gtp * st + m.gpp * sp) * m.xp;
}

__device__ inline double div(const Metric& m, V3 vt, V3 vp) {
  return m.gtt * dot(m.xt, vt) + m.gtp * (dot(m.xt, vp) + dot(m.xp, vt)) + m.gpp * dot(m.xp, vp);
}

// f_E and lap Gamma at every grid point of a group
__global__ void k_surf_rates(const double* __restrict__ X, const double* __restrict__ U,
                             const double* __restrict__ Gm, long long nd, long long N, double inv_pe,
                             double* __restrict__ fe, double* __restrict__ fi) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * N) return;
  const long long d = idx / N, q = idx - d * N;
  const V3 xt = load3(X, 1, nd, d, N, q), xp = load3(X, 2, nd, d, N, q);
  const V3 xtt = load3(X, 3, nd, d, N, q), xtp = load3(X, 4, nd, d, N, q), xpp = load3(X, 5, nd, d, N, q);
  const Metric m = metric(xt, xp);
  const V3 c = cross(xt, xp);
  const V3 ct = cross(xtt, xp) + cross(xt, xtp);
  const V3 cp = cross(xtp, xp) + cross(xt, xpp);
  const double W = m.W, W3 = W * W * W;
  const V3 n = (1.0 / W) * c;
  const V3 nt = (1.0 / W) * ct - (dot(c, ct) / W3) * c;
  const V3 np = (1.0 / W) * cp - (dot(c, cp) / W3) * c;
  const double E = dot(xp, xp), F = dot(xt, xp), G = dot(xt, xt);
  const double K = (E * dot(xtt, n) - 2.0 * F * dot(xtp, n) + G * dot(xpp, n)) / (2.0 * W * W);

  const V3 u = load3(U, 0, nd, d, N, q), ut = load3(U, 1, nd, d, N, q), up = load3(U, 2, nd, d, N, q);
  const double un = dot(u, n);
  const V3 utan = u - un * n;
  const V3 utan_t = ut - (dot(ut, n) + dot(u, nt)) * n - un * nt;
  const V3 utan_p = up - (dot(up, n) + dot(u, np)) * n - un * np;

  const double* g = Gm + d * N + q;
  const long long gs = nd * N;
  const double gam = g[0], gt = g[gs], gp = g[2 * gs], gtt = g[3 * gs], gtp = g[4 * gs], gpp = g[5 * gs];
  const V3 flux_t = gt * utan + gam * utan_t;
  const V3 flux_p = gp * utan + gam * utan_p;
  const V3 gg = grad(m, gt, gp);
  const double conv = div(m, flux_t, flux_p);
  const double frame = dot(utan, gg);
  const double stretch = 2.0 * K * gam * un;
  fe[idx] = -conv + frame + stretch;
  if (fi) {
    const double lap = m.gtt * (gtt - dot(xtt, gg)) + 2.0 * m.gtp * (gtp - dot(xtp, gg)) + m.gpp * (gpp - dot(xpp, gg));
    fi[idx] = inv_pe * lap;
  }
}

// Coefficients of lap s = a_tt s_tt + a_tp s_tp + a_pp s_pp + b_t s_t + b_p s_p, L[5][nd][N].
// With C_t = g^ij x_ij . x_t and C_p = g^ij x_ij . x_p (sum over i, j): b_t = -(g^tt C_t + g^tp C_p),
// b_p = -(g^tp C_t + g^pp C_p).
__global__ void k_lap_coef(const double* __restrict__ X, long long nd, long long N, double* __restrict__ L) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * N) return;
  const long long d = idx / N, q = idx - d * N;
  const V3 xt = load3(X, 1, nd, d, N, q), xp = load3(X, 2, nd, d, N, q);
  const V3 xtt = load3(X, 3, nd, d, N, q), xtp = load3(X, 4, nd, d, N, q), xpp = load3(X, 5, nd, d, N, q);
  const Metric m = metric(xt, xp);
  const double Ct = m.gtt * dot(xtt, xt) + 2.0 * m.gtp * dot(xtp, xt) + m.gpp * dot(xpp, xt);
  const double Cp = m.gtt * dot(xtt, xp) + 2.0 * m.gtp * dot(xtp, xp) + m.gpp * dot(xpp, xp);
  const long long s = nd * N;
  L[idx] = m.gtt;
  L[s + idx] = 2.0 * m.gtp;
  L[2 * s + idx] = m.gpp;
  L[3 * s + idx] = -(m.gtt * Ct + m.gtp * Cp);
  L[4 * s + idx] = -(m.gtp * Ct + m.gpp * Cp);
}

// out = lap s from the coefficients L[5][nd][N] and the fields S[6][nd][N] of s (f, t, p, tt, tp, pp)
__global__ void k_lap_apply(const double* __restrict__ L, const double* __restrict__ S, long long nd, long long N,
                            double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long s = nd * N;
  if (idx >= s) return;
  out[idx] = L[idx] * S[3 * s + idx] + L[s + idx] * S[4 * s + idx] + L[2 * s + idx] * S[5 * s + idx] +
             L[3 * s + idx] * S[s + idx] + L[4 * s + idx] * S[2 * s + idx];
}

// One block per drop: out[d] = sum over the drop's grid of wsin[j] W (x.n / 3) (the volume, mode 0)
// or of wsin[j] W Gamma (the surfactant mass, mode 1), summed in a fixed order.
__global__ void k_drop_integral(const double* __restrict__ X, const double* __restrict__ Gm, long long nd,
                                int P, const double* __restrict__ wsin, int mode, double* __restrict__ out) {
  __shared__ double sh[kThreads];
  const long long d = blockIdx.x;
  const int nk = 2 * P + 2;
  const long long N = (long long)(P + 1) * nk;
  double acc = 0;
  for (long long q = threadIdx.x; q < N; q += blockDim.x) {
    const V3 xt = load3(X, 1, nd, d, N, q), xp = load3(X, 2, nd, d, N, q);
    const V3 c = cross(xt, xp);
    const double W = sqrt(dot(c, c));
    const double w = wsin[q / nk] * W;
    if (mode == 0) {
      const V3 x = load3(X, 0, nd, d, N, q);
      acc += w * dot(x, c) / (3.0 * W);
    } else {
      acc += w * Gm[d * N + q];
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[d] = sh[0];
}

// One block per drop: out[d] = max |F| over the drop's nper fields of N points (F[d*nper + f][N])
__global__ void k_drop_absmax(const double* __restrict__ F, long long nd, int nper, long long N,
                              double* __restrict__ out) {
  __shared__ double sh[kThreads];
  const long long d = blockIdx.x;
  const double* f = F + d * nper * N;
  double mx = 0;
  for (long long i = threadIdx.x; i < nper * N; i += blockDim.x) mx = fmax(mx, fabs(f[i]));
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[d] = sh[0];
}

// w = (y - a c) * inv_diag (the preconditioned implicit operator in coefficient space)
__global__ void k_implicit_combine(const double* __restrict__ y, const double* __restrict__ c, double a,
                                   const double* __restrict__ inv_diag, long long n, double* __restrict__ w) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = (y[i] - a * c[i]) * inv_diag[i];
}

// y = x * s (elementwise)
__global__ void k_mul(const double* __restrict__ x, const double* __restrict__ s, long long n,
                      double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] * s[i];
}

}  // namespace

int launch_surf_rates(const double* X, const double* U, const double* Gm, long long nd, long long N, double inv_pe,
                      double* fe, double* fi, cudaStream_t s) {
  if (nd * N == 0) return BIE_OK;
  k_surf_rates<<<blocks_for(nd * N), kThreads, 0, s>>>(X, U, Gm, nd, N, inv_pe, fe, fi);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_lap_coef(const double* X, long long nd, long long N, double* L, cudaStream_t s) {
  if (nd * N == 0) return BIE_OK;
  k_lap_coef<<<blocks_for(nd * N), kThreads, 0, s>>>(X, nd, N, L);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_lap_apply(const double* L, const double* S, long long nd, long long N, double* out, cudaStream_t s) {
  if (nd * N == 0) return BIE_OK;
  k_lap_apply<<<blocks_for(nd * N), kThreads, 0, s>>>(L, S, nd, N, out);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_drop_integral(const double* X, const double* Gm, long long nd, int P, const double* wsin, int mode,
                         double* out, cudaStream_t s) {
  if (nd == 0) return BIE_OK;
  k_drop_integral<<<(unsigned)nd, kThreads, 0, s>>>(X, Gm, nd, P, wsin, mode, out);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_drop_absmax(const double* F, long long nd, int nper, long long N, double* out, cudaStream_t s) {
  if (nd == 0) return BIE_OK;
  k_drop_absmax<<<(unsigned)nd, kThreads, 0, s>>>(F, nd, nper, N, out);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_implicit_combine(const double* y, const double* c, double a, const double* inv_diag, long long n,
                            double* w, cudaStream_t s) {
  if (n == 0) return BIE_OK;
  k_implicit_combine<<<blocks_for(n), kThreads, 0, s>>>(y, c, a, inv_diag, n, w);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_mul(const double* x, const double* sc, long long n, double* y, cudaStream_t s) {
  if (n == 0) return BIE_OK;
  k_mul<<<blocks_for(n), kThreads, 0, s>>>(x, sc, n, y);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
