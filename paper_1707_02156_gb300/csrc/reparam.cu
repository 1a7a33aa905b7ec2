// Angle reparametrisation of the drop surfaces and their surfactant (Sec. 4, Alg. 2): the kernels.
//
// Every drop of a degree group carries the parameter points (theta*, phi*) of the working grid of
// degree P (one per grid point), which start at the grid's (theta_j, phi_k) and move with the angle
// velocity of Eq. system_rep_sol in pseudo-time.  The kernels here
//   * evaluate SH expansions of degree P and their first parameter derivatives at those scattered
//     points (the original surface and surfactant, Eqs. rep_trasf1, rep_trasf2),
//   * sum the mode norms |x_n^m| per degree (Eqs. energy_rep, ncutoff_adaptive),
//   * scale coefficients by the per-drop attenuation a_n (the gradient of Eq. energy_rep),
//   * project the energy gradient on the tangent plane (Eq. pseudo_rep), reduce its largest norm per
//     drop (the stopping test of Alg. 2), and take the forward Euler step of the angles.
// All in FP64.  The host loop that strings them together is bie_reparametrize (bie.cu).
#include <cuda_runtime.h>

#include "internal.cuh"

namespace bie {
namespace {

constexpr int kThreads = 128;
inline unsigned blocks_for(long long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// Values, theta and phi derivatives at the points (th, ph) of drop d of nf scalar expansions of
// degree P, coef[d][f][(P+1)^2].  out[d][f][3][N]: value, d/dtheta, d/dphi (derivs = 0: value only,
// out[d][f][1][N]).  The normalised associated Legendre functions (Condon-Shortley phase) and their
// theta derivatives come from the recursions in the degree, differentiated term by term, so no
// division by sin(theta) occurs:
//   P_m^m = -c_m s P_{m-1}^{m-1},             d P_m^m = -c_m (x P_{m-1}^{m-1} + s d P_{m-1}^{m-1}),
//   P_{m+1}^m = e_m x P_m^m,                  d P_{m+1}^m = e_m (-s P_m^m + x d P_m^m),
//   P_n^m = a (x P_{n-1}^m + b P_{n-2}^m),     d P_n^m = a (-s P_{n-1}^m + x d P_{n-1}^m + b d P_{n-2}^m),
// x = cos(theta), s = sin(theta), c_m = sqrt(1 + 1/(2m)), e_m = sqrt(2m + 3),
// a = sqrt((4n^2 - 1)/(n^2 - m^2)), b = -sqrt(((n-1)^2 - m^2)/(4(n-1)^2 - 1)); ab holds (a, b) per (m, n).
template <int NF>
__global__ void __launch_bounds__(kThreads) k_eval_points(const double* __restrict__ coef, int P, long long N,
                                                          const double* __restrict__ th, const double* __restrict__ ph,
                                                          const double* __restrict__ ab, int derivs,
                                                          double* __restrict__ out) {
  const long long d = blockIdx.y;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const long long nc = (long long)(P + 1) * (P + 1);
  const double* c = coef + d * NF * nc;
  const double t = th[d * N + q], phi = ph[d * N + q];
  double x, s;
  sincos(t, &s, &x);
  double f[NF], ft[NF], fp[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) f[k] = ft[k] = fp[k] = 0.0;
  double pmm = 0.28209479177387814347;  // sqrt(1/(4 pi))
  double dpmm = 0.0;
  for (int m = 0; m <= P; ++m) {
    if (m > 0) {
      const double cm = -sqrt(1.0 + 0.5 / m);
      const double np = cm * s * pmm, nd = cm * (x * pmm + s * dpmm);
      pmm = np;
      dpmm = nd;
    }
    double hr[NF], hi[NF], dr[NF], di[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) hr[k] = hi[k] = dr[k] = di[k] = 0.0;
    double p2 = 0, dp2 = 0, p1 = pmm, dp1 = dpmm;
    const double* abm = ab + 2 * ((long long)m * (P + 1) - (long long)m * (m - 1) / 2);  // row of order m
    for (int n = m; n <= P; ++n) {
      double pn, dpn;
      if (n == m) {
        pn = p1;
        dpn = dp1;
      } else if (n == m + 1) {
        const double e = sqrt(2.0 * m + 3.0);
        pn = e * x * pmm;
        dpn = e * (-s * pmm + x * dpmm);
        p2 = p1;
        dp2 = dp1;
        p1 = pn;
        dp1 = dpn;
      } else {
        const double a = abm[2 * (n - m)], b = abm[2 * (n - m) + 1];
        pn = a * (x * p1 + b * p2);
        dpn = a * (-s * p1 + x * dp1 + b * dp2);
        p2 = p1;
        dp2 = dp1;
        p1 = pn;
        dp1 = dpn;
      }
      const long long ir = (long long)n * (n + 1) + m, ii = (long long)n * (n + 1) - m;
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const double cr = c[k * nc + ir], ci = m > 0 ? c[k * nc + ii] : 0.0;
        hr[k] = fma(cr, pn, hr[k]);
        hi[k] = fma(ci, pn, hi[k]);
        dr[k] = fma(cr, dpn, dr[k]);
        di[k] = fma(ci, dpn, di[k]);
      }
    }
    double sm, cmv;
    sincos((double)m * phi, &sm, &cmv);
    const double fac = m == 0 ? 1.0 : 2.0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      f[k] += fac * (hr[k] * cmv - hi[k] * sm);
      ft[k] += fac * (dr[k] * cmv - di[k] * sm);
      fp[k] += fac * m * (-hr[k] * sm - hi[k] * cmv);
    }
  }
  const int kinds = derivs ? 3 : 1;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    double* o = out + ((d * NF + k) * kinds) * N + q;
    o[0] = f[k];
    if (derivs) {
      o[N] = ft[k];
      o[2 * N] = fp[k];
    }
  }
}

// norms[d][n][0] = sum_{m=-n..n} |x_n^m|, norms[d][n][1] = sum_{m=-n..n} |x_n^m|^2, with |x_n^m| the
// Euclidean norm of the three complex coefficients of x (|x_n^{-m}| = |x_n^m| for a real surface).
__global__ void k_mode_norms(const double* __restrict__ coef, int P, long long nd, double* __restrict__ norms) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * (P + 1)) return;
  const long long d = idx / (P + 1);
  const int n = (int)(idx - d * (P + 1));
  const long long nc = (long long)(P + 1) * (P + 1);
  const double* c = coef + d * 3 * nc;
  double s1 = 0, s2 = 0;
  for (int m = 0; m <= n; ++m) {
    double a2 = 0;
    for (int k = 0; k < 3; ++k) {
      const double re = c[k * nc + n * (n + 1) + m], im = m > 0 ? c[k * nc + n * (n + 1) - m] : 0.0;
      a2 += re * re + im * im;
    }
    const double w = m == 0 ? 1.0 : 2.0;
    s1 += w * sqrt(a2);
    s2 += w * a2;
  }
  norms[2 * idx] = s1;
  norms[2 * idx + 1] = s2;
}

// out[d][c][(n, m)] = scale * a[d][n] * in[d][c][(n, m)]
__global__ void k_scale_degrees(const double* __restrict__ in, const double* __restrict__ a, int P, long long nd,
                                int ncomp, double scale, double* __restrict__ out) {
  const long long nc = (long long)(P + 1) * (P + 1);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * ncomp * nc) return;
  const long long d = idx / (ncomp * nc);
  const int r = (int)(idx % nc);
  int n = (int)sqrt((double)r);
  while (n * n > r) --n;
  while ((n + 1) * (n + 1) <= r) ++n;
  out[idx] = scale * a[d * (P + 1) + n] * in[idx];
}

// Order-preserving bit pattern of a non-negative double, for atomicMax on unsigned long long.
__device__ inline void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// g = (I - n n) gradE at every point, n the unit normal x_t x x_p / |x_t x x_p| of the original
// surface there (E: [d][3][3][N] value, t, p of x0 at the points; gradE [d][3][N]); gmax[d] = max |g|.
__global__ void k_rep_gradient(const double* __restrict__ E, const double* __restrict__ gradE, long long N,
                               long long nd, double* __restrict__ g, double* __restrict__ gmax) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double gn = 0.0;
  long long d = idx / N;
  if (idx < nd * N) {
    const long long q = idx - d * N;
    const double* e = E + d * 9 * N + q;  // [comp][kind][N]
    const double tx = e[1 * N], ty = e[4 * N], tz = e[7 * N];
    const double px = e[2 * N], py = e[5 * N], pz = e[8 * N];
    double nx = ty * pz - tz * py, ny = tz * px - tx * pz, nz = tx * py - ty * px;
    const double inv = 1.0 / sqrt(nx * nx + ny * ny + nz * nz);
    nx *= inv;
    ny *= inv;
    nz *= inv;
    const double* ge = gradE + d * 3 * N + q;
    const double gx = ge[0], gy = ge[N], gz = ge[2 * N];
    const double gd = gx * nx + gy * ny + gz * nz;
    const double ox = gx - gd * nx, oy = gy - gd * ny, oz = gz - gd * nz;
    double* go = g + d * 3 * N + q;
    go[0] = ox;
    go[N] = oy;
    go[2 * N] = oz;
    gn = sqrt(ox * ox + oy * oy + oz * oz);
  }
  // warp reduction of the maximum, then one atomic per warp and drop
  const unsigned full = 0xffffffffu;
  long long d0 = __shfl_sync(full, d, 0);
  const bool same = __all_sync(full, d == d0);
  if (same) {
    for (int o = 16; o > 0; o >>= 1) gn = fmax(gn, __shfl_xor_sync(full, gn, o));
    if ((threadIdx.x & 31) == 0 && idx < nd * N) atomic_max_nonneg(gmax + d, gn);
  } else if (idx < nd * N) {
    atomic_max_nonneg(gmax + d, gn);
  }
}

// One forward Euler step of the angles of the drops with active[d] != 0 (Eq. system_rep_sol with
// the pseudo-velocity w = -g): alpha = A^-1 (w.x_t, w.x_p), A the metric of the original surface at
// the point; a step across a pole is mapped back to theta in [0, pi] with phi + pi.
__global__ void k_rep_step(const double* __restrict__ E, const double* __restrict__ g, long long N, long long nd,
                           const int* __restrict__ active, double dtau, double* __restrict__ th,
                           double* __restrict__ ph) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * N) return;
  const long long d = idx / N, q = idx - d * N;
  if (!active[d]) return;
  const double* e = E + d * 9 * N + q;
  const double tx = e[1 * N], ty = e[4 * N], tz = e[7 * N];
  const double px = e[2 * N], py = e[5 * N], pz = e[8 * N];
  const double* gg = g + d * 3 * N + q;
  const double wx = -gg[0], wy = -gg[N], wz = -gg[2 * N];
  const double A11 = tx * tx + ty * ty + tz * tz, A12 = tx * px + ty * py + tz * pz, A22 = px * px + py * py + pz * pz;
  const double b1 = wx * tx + wy * ty + wz * tz, b2 = wx * px + wy * py + wz * pz;
  const double det = A11 * A22 - A12 * A12;
  const double at = (A22 * b1 - A12 * b2) / det, ap = (-A12 * b1 + A11 * b2) / det;
  const double kTwoPi = 6.283185307179586476925286766559, kPiD = 3.141592653589793238462643383279;
  double t = th[idx] + dtau * at, f = ph[idx] + dtau * ap;
  t = fmod(t, kTwoPi);
  if (t < 0) t += kTwoPi;
  if (t > kPiD) {
    t = kTwoPi - t;
    f += kPiD;
  }
  th[idx] = t;
  ph[idx] = f;
}

// The grid's parameter points: th[d][j][k] = theta_j (from the nodes t_j, ascending), ph = pi k/(P+1).
__global__ void k_grid_points(const double* __restrict__ nodes, int P, long long nd, double* __restrict__ th,
                              double* __restrict__ ph) {
  const long long N = (long long)(P + 1) * (2 * P + 2);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * N) return;
  const long long q = idx % N;
  const int j = (int)(q / (2 * P + 2)), k = (int)(q % (2 * P + 2));
  th[idx] = acos(nodes[j]);
  ph[idx] = 3.141592653589793238462643383279 * k / (P + 1);
}

// dst[d][c][(P+1)^2] = src coefficients of degree p of drop d (at src + off[d] + c (p+1)^2), zero-padded
__global__ void k_pad_coef(const double* __restrict__ src, const long long* __restrict__ off, int p, int P,
                           long long nd, int ncomp, double* __restrict__ dst) {
  const long long nC = (long long)(P + 1) * (P + 1), nc = (long long)(p + 1) * (p + 1);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * ncomp * nC) return;
  const long long d = idx / (ncomp * nC);
  const long long r = idx - d * ncomp * nC;
  const int c = (int)(r / nC);
  const long long i = r - c * nC;
  dst[idx] = i < nc ? src[off[d] + c * nc + i] : 0.0;
}

}  // namespace

int launch_pad_coef(const double* src, const long long* off, int p, int P, long long nd, int ncomp, double* dst,
                    cudaStream_t s) {
  const long long n = nd * ncomp * (long long)(P + 1) * (P + 1);
  if (n == 0) return BIE_OK;
  k_pad_coef<<<blocks_for(n), kThreads, 0, s>>>(src, off, p, P, nd, ncomp, dst);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_eval_points(const double* coef, int nf, int P, long long nd, long long N, const double* th,
                       const double* ph, const double* ab, int derivs, double* out, cudaStream_t s) {
  if (nd == 0 || N == 0) return BIE_OK;
  if (nd > 65535) return BIE_EINVAL;
  dim3 grid(blocks_for(N), (unsigned)nd);
  switch (nf) {
    case 1: k_eval_points<1><<<grid, kThreads, 0, s>>>(coef, P, N, th, ph, ab, derivs, out); break;
    case 3: k_eval_points<3><<<grid, kThreads, 0, s>>>(coef, P, N, th, ph, ab, derivs, out); break;
    default: return BIE_EINVAL;
  }
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_mode_norms(const double* coef, int P, long long nd, double* norms, cudaStream_t s) {
  if (nd == 0) return BIE_OK;
  k_mode_norms<<<blocks_for(nd * (P + 1)), kThreads, 0, s>>>(coef, P, nd, norms);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_scale_degrees(const double* in, const double* a, int P, long long nd, int ncomp, double scale, double* out,
                         cudaStream_t s) {
  const long long n = nd * ncomp * (long long)(P + 1) * (P + 1);
  if (n == 0) return BIE_OK;
  k_scale_degrees<<<blocks_for(n), kThreads, 0, s>>>(in, a, P, nd, ncomp, scale, out);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_rep_gradient(const double* E, const double* gradE, long long N, long long nd, double* g, double* gmax,
                        cudaStream_t s) {
  if (nd * N == 0) return BIE_OK;
  BIE_CUDA_TRY(cudaMemsetAsync(gmax, 0, nd * sizeof(double), s));
  k_rep_gradient<<<blocks_for(nd * N), kThreads, 0, s>>>(E, gradE, N, nd, g, gmax);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_rep_step(const double* E, const double* g, long long N, long long nd, const int* active, double dtau,
                    double* th, double* ph, cudaStream_t s) {
  if (nd * N == 0) return BIE_OK;
  k_rep_step<<<blocks_for(nd * N), kThreads, 0, s>>>(E, g, N, nd, active, dtau, th, ph);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_grid_points(const double* nodes, int P, long long nd, double* th, double* ph, cudaStream_t s) {
  const long long n = nd * (long long)(P + 1) * (2 * P + 2);
  if (n == 0) return BIE_OK;
  k_grid_points<<<blocks_for(n), kThreads, 0, s>>>(nodes, P, nd, th, ph);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
