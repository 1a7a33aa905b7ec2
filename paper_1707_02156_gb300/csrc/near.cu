// Near-singular (Omega_2) step of Sec. 2.3: closest point on the source surface by damped Newton
// (Eqs. f_phi, f_theta, newton_ite and the Levenberg-Marquardt footnote), check points along the
// line through the closest point and the target, their regular-rule values, the on-surface value
// from the SH expansion of the source drop's self-interaction values, and 1-D Lagrange interpolation
// in the distance.
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.cuh"
#include "near.h"

namespace bie {
namespace {

constexpr double kPiD = 3.14159265358979323846;

// Coefficients of the normalised Legendre recursion of App. A at (n, m):
// P_n^m = rec_a (cos(theta) P_{n-1}^m - rec_b P_{n-2}^m) for n >= m + 2, and the factor rec_c of the
// derivative identity dP_n^m = rec_c P_n^{m+1} + m cot(theta) P_n^m.
__device__ __forceinline__ double rec_a(int n, int m) {
  return sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
}
__device__ __forceinline__ double rec_b(int n, int m) {
  return sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
}
__device__ __forceinline__ double rec_c(int n, int m) { return sqrt((double)(n - m) * (n + m + 1.0)); }
__device__ __forceinline__ long long tri(int n, int m) { return (long long)n * (n + 1) / 2 + m; }

// tab[3 tri(n, m) + k] = rec_a, rec_b (0 for n < m + 2), rec_c, for 0 <= m <= n <= P
__global__ void k_rec_table(int P, double* __restrict__ tab) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tri(P + 1, 0)) return;
  int n = (int)((sqrt(8.0 * t + 1.0) - 1.0) / 2.0);
  while (tri(n + 1, 0) <= t) ++n;
  while (tri(n, 0) > t) --n;
  const int m = (int)(t - tri(n, 0));
  tab[3 * t] = n >= m + 2 ? rec_a(n, m) : 0.0;
  tab[3 * t + 1] = n >= m + 2 ? rec_b(n, m) : 0.0;
  tab[3 * t + 2] = rec_c(n, m);
}

// Value and first/second parameter derivatives of three real SH series (coefficients c[3][(p+1)^2])
// at (theta, phi), with the Legendre recursion of App. A and the derivative identities
// dP = alpha P^{m+1} + m cot(theta) P^m and the Legendre equation (theta away from the poles).
// out[k][c], k: 0 f, 1 f_t, 2 f_p, 3 f_tt, 4 f_tp, 5 f_pp.
__device__ void sh_eval_d2(const double* __restrict__ c, long long cstride, int p, double th, double ph,
                           const double* __restrict__ tab, double out[6][3]) {
  for (int k = 0; k < 6; ++k)
    for (int q = 0; q < 3; ++q) out[k][q] = 0;
  double st, ct;
  sincos(th, &st, &ct);
  const double cot = ct / st, s2 = st * st;
  double dm = sqrt(1.0 / (4.0 * kPiD));  // P~_m^m
  for (int m = 0; m <= p; ++m) {
    const double dm1 = m + 1 <= p ? -sqrt(1.0 + 1.0 / (2.0 * (m + 1))) * st * dm : 0.0;
    double pm2 = 0, pm1 = 0, qm2 = 0, qm1 = 0;
    double h0r[3] = {0, 0, 0}, h0i[3] = {0, 0, 0}, h1r[3] = {0, 0, 0}, h1i[3] = {0, 0, 0}, h2r[3] = {0, 0, 0},
           h2i[3] = {0, 0, 0};
    for (int n = m; n <= p; ++n) {
      double P;
      if (n == m)
        P = dm;
      else if (n == m + 1)
        P = sqrt(2.0 * m + 3.0) * ct * dm;
      else
        P = tab[3 * tri(n, m)] * (ct * pm1 - tab[3 * tri(n, m) + 1] * pm2);
      double Q = 0;  // P~_n^{m+1}
      const int m1 = m + 1;
      if (n == m1)
        Q = dm1;
      else if (n == m1 + 1)
        Q = sqrt(2.0 * m1 + 3.0) * ct * dm1;
      else if (n > m1 + 1)
        Q = tab[3 * tri(n, m1)] * (ct * qm1 - tab[3 * tri(n, m1) + 1] * qm2);
      pm2 = pm1;
      pm1 = P;
      if (n >= m1) {
        qm2 = qm1;
        qm1 = Q;
      }
      const double dP = tab[3 * tri(n, m) + 2] * Q + m * cot * P;
      const double d2P = -cot * dP + ((double)m * m / s2 - n * (n + 1.0)) * P;
      for (int q = 0; q < 3; ++q) {
        const double re = c[q * cstride + n * (n + 1) + m];
        const double im = m > 0 ? c[q * cstride + n * (n + 1) - m] : 0.0;
        h0r[q] += re * P;
        h0i[q] += im * P;
        h1r[q] += re * dP;
        h1i[q] += im * dP;
        h2r[q] += re * d2P;
        h2i[q] += im * d2P;
      }
    }
    double sm, cm;
    sincos(m * ph, &sm, &cm);
    const double fac = m == 0 ? 1.0 : 2.0;
    for (int q = 0; q < 3; ++q) {
      const double v0 = h0r[q] * cm - h0i[q] * sm, w0 = h0r[q] * sm + h0i[q] * cm;  // Re, Im of h0 e^{i m phi}
      const double v1 = h1r[q] * cm - h1i[q] * sm, w1 = h1r[q] * sm + h1i[q] * cm;
      const double v2 = h2r[q] * cm - h2i[q] * sm;
      out[0][q] += fac * v0;
      out[1][q] += fac * v1;
      out[3][q] += fac * v2;
      out[2][q] += fac * (-m * w0);  // Re(i m h e^{i m phi})
      out[4][q] += fac * (-m * w1);
      out[5][q] += fac * (-(double)m * m * v0);
    }
    dm = dm1;
  }
}

// Value of three real SH series at (theta, phi) (any theta, poles included).
__device__ void sh_eval3(const double* __restrict__ c, long long cstride, int p, double th, double ph, double* out) {
  out[0] = out[1] = out[2] = 0;
  double st, ct;
  sincos(th, &st, &ct);
  double dm = sqrt(1.0 / (4.0 * kPiD));
  for (int m = 0; m <= p; ++m) {
    double pm2 = 0, pm1 = 0;
    double hr[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int n = m; n <= p; ++n) {
      double P;
      if (n == m)
        P = dm;
      else if (n == m + 1)
        P = sqrt(2.0 * m + 3.0) * ct * dm;
      else
        P = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m)) *
            (ct * pm1 - sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0)) * pm2);
      pm2 = pm1;
      pm1 = P;
      for (int q = 0; q < 3; ++q) {
        hr[q] += c[q * cstride + n * (n + 1) + m] * P;
        if (m > 0) hi[q] += c[q * cstride + n * (n + 1) - m] * P;
      }
    }
    double sm, cm;
    sincos(m * ph, &sm, &cm);
    const double fac = m == 0 ? 1.0 : 2.0;
    for (int q = 0; q < 3; ++q) out[q] += fac * (hr[q] * cm - hi[q] * sm);
    dm = m + 1 <= p ? -sqrt(1.0 + 1.0 / (2.0 * (m + 1))) * st * dm : 0.0;
  }
}

// seed: nearest standard grid point of drop j to the target
__global__ void k_near_seed(const NearPair* __restrict__ pairs, int npair, const double* __restrict__ rec_std,
                            const long long* __restrict__ toff, const int* __restrict__ ngd,
                            const long long* __restrict__ tgt_loc, const int* __restrict__ tdrop,
                            int* __restrict__ seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npair) return;
  const long long t = pairs[i].target;
  const int j = pairs[i].src_drop, di = tdrop[t];
  const long long ngi = ngd[di];
  const double* ri = rec_std + 7 * toff[di];
  const double x0 = ri[tgt_loc[t]], x1 = ri[ngi + tgt_loc[t]], x2 = ri[2 * ngi + tgt_loc[t]];
  const long long N = ngd[j];
  const double* r = rec_std + 7 * toff[j];
  double best = 1e300;
  int bi = 0;
  for (long long s = 0; s < N; ++s) {
    const double d0 = x0 - r[s], d1 = x1 - r[N + s], d2 = x2 - r[2 * N + s];
    const double d = d0 * d0 + d1 * d1 + d2 * d2;
    if (d < best) {
      best = d;
      bi = (int)s;
    }
  }
  seed[i] = bi;
}

// Levenberg-Marquardt Newton on F = |x(theta, phi) - x0|^2 / 2 in the rotated frame (seed at the
// equator).  One thread per pair; rotated coefficients xr[pair][3][(p+1)^2].
__global__ void k_near_newton(const NearPair* __restrict__ pairs, int npair, const double* __restrict__ xr,
                              const int* __restrict__ pdeg, const long long* __restrict__ xr_off,
                              const double* __restrict__ x0all, const double* __restrict__ tab,
                              double* __restrict__ result) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npair) return;
  const int p = pdeg[pairs[i].src_drop];
  const long long cs = (long long)(p + 1) * (p + 1);
  const double* c = xr + xr_off[i];
  const double x0[3] = {x0all[3 * i], x0all[3 * i + 1], x0all[3 * i + 2]};
  double th = 0.5 * kPiD, ph = 0.0;
  double d[6][3];
  sh_eval_d2(c, cs, p, th, ph, tab, d);
  auto half_sq = [&](const double* x) {
    const double a = x[0] - x0[0], b = x[1] - x0[1], e = x[2] - x0[2];
    return 0.5 * (a * a + b * b + e * e);
  };
  double F = half_sq(d[0]);
  double mu = -1.0;
  for (int it = 0; it < 30; ++it) {
    double r[3], xt[3], xp[3];
    for (int q = 0; q < 3; ++q) {
      r[q] = d[0][q] - x0[q];
      xt[q] = d[1][q];
      xp[q] = d[2][q];
    }
    const double g0 = r[0] * xt[0] + r[1] * xt[1] + r[2] * xt[2];
    const double g1 = r[0] * xp[0] + r[1] * xp[1] + r[2] * xp[2];
    const double Haa = xt[0] * xt[0] + xt[1] * xt[1] + xt[2] * xt[2] + r[0] * d[3][0] + r[1] * d[3][1] + r[2] * d[3][2];
    const double Hab = xt[0] * xp[0] + xt[1] * xp[1] + xt[2] * xp[2] + r[0] * d[4][0] + r[1] * d[4][1] + r[2] * d[4][2];
    const double Hbb = xp[0] * xp[0] + xp[1] * xp[1] + xp[2] * xp[2] + r[0] * d[5][0] + r[1] * d[5][1] + r[2] * d[5][2];
    if (mu < 0) mu = 1e-8 * fabs(Haa + Hbb);
    bool accepted = false;
    double s0 = 0, s1 = 0;
    for (int k = 0; k < 40; ++k) {
      const double a = Haa + mu, b = Hab, e = Hbb + mu;
      const double det = a * e - b * b;
      s0 = -(e * g0 - b * g1) / det;
      s1 = -(a * g1 - b * g0) / det;
      double dn[6][3];
      sh_eval_d2(c, cs, p, th + s0, ph + s1, tab, dn);
      if (half_sq(dn[0]) <= F) {
        accepted = true;
        break;
      }
      mu *= 10.0;
    }
    if (!accepted) break;
    th += s0;
    ph += s1;
    sh_eval_d2(c, cs, p, th, ph, tab, d);
    F = half_sq(d[0]);
    if (fmax(fabs(s0), fabs(s1)) < 1e-14) break;
  }
  result[5 * i + 0] = th;
  result[5 * i + 1] = ph;
  result[5 * i + 2] = d[0][0];
  result[5 * i + 3] = d[0][1];
  result[5 * i + 4] = d[0][2];
}

// grid of each check point: 0 standard (Omega_0), 1 upsampled otherwise (same distance rule as the
// region split)
__global__ void k_near_checkgrid(const NearPair* __restrict__ pairs, int npair, int L, const double* __restrict__ pts,
                                 const double* __restrict__ centre, const double* __restrict__ bound,
                                 const double* __restrict__ h, double a_tilde, const double* __restrict__ rec_up,
                                 const long long* __restrict__ up_off, const long long* __restrict__ up_n,
                                 int* __restrict__ grid) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npair * L) return;
  const int i = idx / L;
  const int j = pairs[i].src_drop;
  const double x0 = pts[3 * idx], x1 = pts[3 * idx + 1], x2 = pts[3 * idx + 2];
  const double dc0 = x0 - centre[3 * j], dc1 = x1 - centre[3 * j + 1], dc2 = x2 - centre[3 * j + 2];
  if (sqrt(dc0 * dc0 + dc1 * dc1 + dc2 * dc2) - bound[j] > a_tilde * h[j]) {
    grid[idx] = 0;
    return;
  }
  const long long N = up_n[j];
  const double* r = rec_up + 7 * up_off[j];
  double best = 1e300;
  for (long long s = 0; s < N; ++s) {
    const double d0 = x0 - r[s], d1 = x1 - r[N + s], d2 = x2 - r[2 * N + s];
    best = fmin(best, d0 * d0 + d1 * d1 + d2 * d2);
  }
  grid[idx] = sqrt(best) <= a_tilde * h[j] ? 1 : 0;
}

// Regular-rule value of drop j's layer at check point (pair, l): one block per check point.
template <typename R, int KIND>
__global__ void __launch_bounds__(256) k_near_checks(
    const NearPair* __restrict__ pairs, int L, const double* __restrict__ pts, const int* __restrict__ grid,
    const double* __restrict__ centre, const long long* __restrict__ toff, const int* __restrict__ ngd,
    const long long* __restrict__ up_off, const long long* __restrict__ up_n, const R* __restrict__ Xs,
    const R* __restrict__ Ns, const R* __restrict__ Qs, long long nstd, const R* __restrict__ Xu,
    const R* __restrict__ Nu, const R* __restrict__ Qu, long long nup, const double* __restrict__ wts,
    double* __restrict__ cv) {
  __shared__ R red[3 * 32];
  const int idx = blockIdx.x;
  const int i = idx / L;
  const int j = pairs[i].src_drop;
  const bool up = grid[idx] != 0;
  const R* X = up ? Xu : Xs;
  const R* N = up ? Nu : Ns;
  const R* Q = up ? Qu : Qs;
  const long long ld = up ? nup : nstd;
  const long long s0 = up ? up_off[j] : toff[j];
  const long long s1 = s0 + (up ? up_n[j] : (long long)ngd[j]);
  const R px = (R)(pts[3 * idx] - centre[3 * j]), py = (R)(pts[3 * idx + 1] - centre[3 * j + 1]),
          pz = (R)(pts[3 * idx + 2] - centre[3 * j + 2]);
  R a0 = 0, a1 = 0, a2 = 0;
  for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const R dx = px - X[s], dy = py - X[ld + s], dz = pz - X[2 * ld + s];
    const R ri = rsqrt_<R>(dx * dx + dy * dy + dz * dz);
    const R q0 = Q[s], q1 = Q[ld + s], q2 = Q[2 * ld + s];
    const R xq = dx * q0 + dy * q1 + dz * q2;
    if (KIND == 0) {
      const R c = xq * ri * ri * ri;
      a0 += q0 * ri + c * dx;
      a1 += q1 * ri + c * dy;
      a2 += q2 * ri + c * dz;
    } else {
      const R xn = dx * N[s] + dy * N[ld + s] + dz * N[2 * ld + s];
      const R ri2 = ri * ri;
      const R c = (R)(-6) * xq * xn * ri2 * ri2 * ri;
      a0 += c * dx;
      a1 += c * dy;
      a2 += c * dz;
    }
  }
  block_sum3<R>(a0, a1, a2, red);
  if (threadIdx.x == 0) {
    const double w = wts[j];
    cv[3 * idx] = w * (double)a0;
    cv[3 * idx + 1] = w * (double)a1;
    cv[3 * idx + 2] = w * (double)a2;
  }
}

// One thread per target with near pairs: anchor from the source drop's (weighted) self expansion,
// minus 4 pi w_j u(x*) for the double layer, then Lagrange interpolation at the target's distance.
__global__ void k_near_interp(const NearPair* __restrict__ pairs, const int* __restrict__ tbeg, int ntgt, int L,
                              int kind, const double* __restrict__ selfcoef, const double* __restrict__ dens,
                              const long long* __restrict__ coef_off, const int* __restrict__ pdeg,
                              const double* __restrict__ hdrop, const double* __restrict__ wts,
                              const double* __restrict__ cv, const int* __restrict__ tdrop,
                              const long long* __restrict__ tgt_loc, const long long* __restrict__ val_off,
                              const int* __restrict__ ngd, double* __restrict__ vals) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= ntgt) return;
  double acc[3] = {0, 0, 0};
  const long long t = pairs[tbeg[u]].target;
  for (int i = tbeg[u]; i < tbeg[u + 1]; ++i) {
    const NearPair& P = pairs[i];
    const int j = P.src_drop, p = pdeg[j];
    const long long cs = (long long)(p + 1) * (p + 1);
    double anchor[3];
    sh_eval3(selfcoef + coef_off[j], cs, p, P.theta_v, P.phi_v, anchor);
    if (kind == 1) {
      double us[3];
      sh_eval3(dens + coef_off[j], cs, p, P.theta_v, P.phi_v, us);
      for (int q = 0; q < 3; ++q) anchor[q] -= 4.0 * kPiD * wts[j] * us[q];
    }
    // Lagrange through (0, anchor) and (h sqrt(l), cv_l), l = 1..L, at distance d0
    const double h = hdrop[j], x = P.d0;
    for (int l = 0; l <= L; ++l) {
      const double xl = l == 0 ? 0.0 : h * sqrt((double)l);
      double bas = 1.0;
      for (int k = 0; k <= L; ++k) {
        if (k == l) continue;
        const double xk = k == 0 ? 0.0 : h * sqrt((double)k);
        bas *= (x - xk) / (xl - xk);
      }
      for (int q = 0; q < 3; ++q) acc[q] += bas * (l == 0 ? anchor[q] : cv[3 * ((long long)i * L + (l - 1)) + q]);
    }
  }
  const int d = tdrop[t];
  const long long ng = ngd[d];
  double* v = vals + val_off[d] + tgt_loc[t];
  v[0] += acc[0];
  v[ng] += acc[1];
  v[2 * ng] += acc[2];
}

// The source drop's shape coefficients of pair i with the phases of its seed longitude applied,
// g_n^m = e^{i m alpha_i} x_n^m (real-packed; ph[i][m] = (cos m alpha_i, sin m alpha_i)), written to
// out + dst_off[i] as [3][(p+1)^2]: the first step of the rotation R_z(alpha) R_y(beta), so that the
// pairs of one seed latitude then share one rotation launch.  One block per pair.
__global__ void k_near_phase_shift(const NearPair* __restrict__ pairs, int npair, const double* __restrict__ coef,
                                   const long long* __restrict__ coef_off, const int* __restrict__ pdeg, int pmax,
                                   const double* __restrict__ ph, const long long* __restrict__ dst_off,
                                   double* __restrict__ out) {
  const int i = blockIdx.x;
  if (i >= npair) return;
  const int j = pairs[i].src_drop;
  const int p = pdeg[j];
  const long long nc = (long long)(p + 1) * (p + 1);
  const double* phi = ph + (long long)i * 2 * (pmax + 1);
  for (long long q = threadIdx.x; q < 3 * nc; q += blockDim.x) {
    const int c = (int)(q / nc);
    const long long k = q - c * nc;
    int n = (int)sqrt((double)k);
    while ((long long)n * n > k) --n;
    while ((long long)(n + 1) * (n + 1) <= k) ++n;
    const int mm = (int)(k - (long long)n * (n + 1));
    const int m = mm < 0 ? -mm : mm;
    const double* f = coef + coef_off[j] + c * nc;
    const double fr = f[n * (n + 1) + m];
    const double fi = m > 0 ? f[n * (n + 1) - m] : 0.0;
    const double cr = phi[2 * m], ci = phi[2 * m + 1];
    out[dst_off[i] + c * nc + k] = mm >= 0 ? fr * cr - fi * ci : fr * ci + fi * cr;
  }
}

}  // namespace

int launch_near_phase_shift(const NearPair* pairs, int npair, const double* coef, const long long* coef_off,
                            const int* pdeg, int pmax, const double* ph, const long long* dst_off, double* out,
                            cudaStream_t s) {
  if (!npair) return BIE_OK;
  k_near_phase_shift<<<npair, 128, 0, s>>>(pairs, npair, coef, coef_off, pdeg, pmax, ph, dst_off, out);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_near_seed(const NearPair* pairs, int npair, const double* rec_std, const long long* toff, const int* ngd,
                     const long long* tgt_loc, const int* tdrop, int* seed, cudaStream_t s) {
  if (!npair) return BIE_OK;
  k_near_seed<<<(npair + 127) / 128, 128, 0, s>>>(pairs, npair, rec_std, toff, ngd, tgt_loc, tdrop, seed);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int near_rec_table_doubles(int P) { return 3 * (P + 1) * (P + 2) / 2; }

int launch_near_rec_table(int P, double* tab, cudaStream_t s) {
  const int n = (P + 1) * (P + 2) / 2;
  k_rec_table<<<(n + 127) / 128, 128, 0, s>>>(P, tab);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_near_newton(const NearPair* pairs, int npair, const double* xr, const int* pdeg, const long long* xr_off,
                       const double* x0, const double* tab, double* result, cudaStream_t s) {
  if (!npair) return BIE_OK;
  k_near_newton<<<(npair + 63) / 64, 64, 0, s>>>(pairs, npair, xr, pdeg, xr_off, x0, tab, result);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_near_checkgrid(const NearPair* pairs, int npair, int L, const double* pts, const double* centre,
                          const double* bound, const double* h, double a_tilde, const double* rec_up,
                          const long long* up_off, const long long* up_n, int* grid, cudaStream_t s) {
  if (!npair) return BIE_OK;
  k_near_checkgrid<<<(npair * L + 127) / 128, 128, 0, s>>>(pairs, npair, L, pts, centre, bound, h, a_tilde, rec_up,
                                                           up_off, up_n, grid);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R>
int launch_near_checks(int kind, const NearPair* pairs, int npair, int L, const double* pts, const int* grid,
                       const double* centre, const long long* toff, const int* ngd, const long long* up_off,
                       const long long* up_n, const R* Xs, const R* Ns, const R* Qs, long long nstd, const R* Xu,
                       const R* Nu, const R* Qu, long long nup, const double* wts, double* cv, cudaStream_t s) {
  if (!npair) return BIE_OK;
  if (kind == 0)
    k_near_checks<R, 0><<<npair * L, 256, 0, s>>>(pairs, L, pts, grid, centre, toff, ngd, up_off, up_n, Xs, Ns, Qs,
                                                  nstd, Xu, Nu, Qu, nup, wts, cv);
  else
    k_near_checks<R, 1><<<npair * L, 256, 0, s>>>(pairs, L, pts, grid, centre, toff, ngd, up_off, up_n, Xs, Ns, Qs,
                                                  nstd, Xu, Nu, Qu, nup, wts, cv);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_near_interp(const NearPair* pairs, const int* tbeg, int ntgt, int L, int kind, const double* selfcoef,
                       const double* dens, const long long* coef_off, const int* pdeg, const double* hdrop,
                       const double* wts, const double* cv, const int* tdrop, const long long* tgt_loc,
                       const long long* val_off, const int* ngd, double* vals, cudaStream_t s) {
  if (!ntgt) return BIE_OK;
  k_near_interp<<<(ntgt + 63) / 64, 64, 0, s>>>(pairs, tbeg, ntgt, L, kind, selfcoef, dens, coef_off, pdeg, hdrop,
                                                wts, cv, tdrop, tgt_loc, val_off, ngd, vals);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template int launch_near_checks<double>(int, const NearPair*, int, int, const double*, const int*, const double*,
                                        const long long*, const int*, const long long*, const long long*,
                                        const double*, const double*, const double*, long long, const double*,
                                        const double*, const double*, long long, const double*, double*,
                                        cudaStream_t);
template int launch_near_checks<float>(int, const NearPair*, int, int, const double*, const int*, const double*,
                                       const long long*, const int*, const long long*, const long long*, const float*,
                                       const float*, const float*, long long, const float*, const float*,
                                       const float*, long long, const double*, double*, cudaStream_t);

}  // namespace bie
