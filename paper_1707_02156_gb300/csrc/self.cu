// Singular self interaction of every drop (Thm 1, Sec. 2.2, App. B): one block per target.
//
// Both forms rotate the density so that the target sits at the pole (App. B, real blocks of the
// latitude's Wigner matrices applied to e^{i m phi_b} rho_n^m) and run the Legendre step of the
// synthesis on the degree-pq grid, h_m(theta_j) = sum_n rho'_n^m P~_n^m(cos theta_j), in shared memory.
//
//  * direct form: the phi step rho'(theta_j, phi_k) = h_0 + 2 Re sum_m h_m e^{i m phi_k} is evaluated
//    for the longitude pair (k, k + pq + 1) from the even and odd orders, and the Stokeslet or
//    stresslet pair sum of Thm 1 is accumulated against the cached rotated geometry;
//  * Fourier form: the same double sum reassociated exactly,
//        sum_{j,k} M_jk rho'_jk = sum_j sum_m c_m Re[ Mhat_jm h_m(theta_j) ],   c_0 = 1, c_m = 2,
//    with M_jk the 3x3 kernel weight of the quadrature point (w^s_j K(x0 - x') W'/sin theta_j, geometry
//    only) and Mhat_jm = sum_k M_jk e^{i m phi_k} its phi transform, built once per geometry.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace bie {
namespace {

// Stages 0-1: g = e^{i m phi_b} rho_n^m (three components) then the rotation, rc = rotated
// coefficients (real-packed, [3][(p+1)^2]).  g and rc are shared-memory arrays.
template <typename R>
__device__ void rotate_target(const double* __restrict__ dens, const long long* __restrict__ foff3, long long ld,
                              int p, int a, int b, const R* __restrict__ wblk, long long wstride,
                              const R* __restrict__ ph, R* rc, R* g) {
  const int nc = (p + 1) * (p + 1);
  const int nb = 2 * p + 2;
  for (int i = threadIdx.x; i < 3 * nc; i += blockDim.x) {
    const int c = i / nc, r = i - c * nc;
    const int n = degree_of(r);
    const int m = r - n * (n + 1);
    if (m < 0) continue;  // the owner of Re rho_n^m writes both parts
    const double* f = dens + foff3[ld * 3 + c];
    const R fr = (R)f[n * (n + 1) + m];
    const R fi = m > 0 ? (R)f[n * (n + 1) - m] : (R)0;
    const R co = ph[((long long)m * nb + b) * 2], si = ph[((long long)m * nb + b) * 2 + 1];
    g[c * nc + n * (n + 1) + m] = fr * co - fi * si;
    if (m > 0) g[c * nc + n * (n + 1) - m] = fr * si + fi * co;
  }
  __syncthreads();
  const R* blk = wblk + (long long)a * wstride;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int n = degree_of(i);
    const int o = i - n * n;  // 0..2n
    // blocks of degree n start after sum_{k<n} (k+1)^2 + k^2 entries
    const long long boff = (long long)n * (n + 1) * (2 * n + 1) / 6 + (long long)(n - 1) * n * (2 * n - 1) / 6;
    const R* g0 = g + n * (n + 1);
    R a0 = 0, a1 = 0, a2 = 0;
    int dst;
    if (o <= n) {
      const R* Cc = blk + boff + o;  // column-major: entry (o, m) at m (n+1) + o
      for (int m = 0; m <= n; ++m) {
        const R cv = Cc[(long long)m * (n + 1)];
        a0 += cv * g0[m];
        a1 += cv * g0[nc + m];
        a2 += cv * g0[2 * nc + m];
      }
      dst = n * (n + 1) + o;
    } else {
      const int mp = o - n;
      const R* Sc = blk + boff + (long long)(n + 1) * (n + 1) + (mp - 1);
      for (int m = 1; m <= n; ++m) {
        const R sv = Sc[(long long)(m - 1) * n];
        a0 += sv * g0[-m];
        a1 += sv * g0[nc - m];
        a2 += sv * g0[2 * nc - m];
      }
      dst = n * (n + 1) - mp;
    }
    rc[dst] = a0;
    rc[nc + dst] = a1;
    rc[2 * nc + dst] = a2;
  }
  __syncthreads();
}

// Stage 2: h[c][jj][m] (complex) = sum_n rc[c](n, m) T0[m][n][j0 + jj] for jj < jn.
template <typename R>
__device__ void legendre_chunk(const R* rc, int p, int nq_j, int j0, int jn, const R* __restrict__ T0, R* h) {
  const int nc = (p + 1) * (p + 1);
  const long long cstride = (long long)jn * (p + 1) * 2;
  for (int i = threadIdx.x; i < (p + 1) * jn; i += blockDim.x) {
    const int m = i / jn, jj = i - m * jn;
    const R* Tm = T0 + leg_row(p, m, m, nq_j) + j0 + jj;
    R r0 = 0, r1 = 0, r2 = 0, i0 = 0, i1 = 0, i2 = 0;
    for (int n = m; n <= p; ++n) {
      const R tv = Tm[(long long)(n - m) * nq_j];
      const int re = n * (n + 1) + m;
      r0 += rc[re] * tv;
      r1 += rc[nc + re] * tv;
      r2 += rc[2 * nc + re] * tv;
      if (m > 0) {
        const int im = n * (n + 1) - m;
        i0 += rc[im] * tv;
        i1 += rc[nc + im] * tv;
        i2 += rc[2 * nc + im] * tv;
      }
    }
    R* hh = h + ((long long)jj * (p + 1) + m) * 2;
    hh[0] = r0;
    hh[1] = i0;
    hh[cstride] = r1;
    hh[cstride + 1] = i1;
    hh[2 * cstride] = r2;
    hh[2 * cstride + 1] = i2;
  }
  __syncthreads();
}

template <typename R>
__device__ inline void write_target(R s0, R s1, R s2, const double* __restrict__ wts,
                                    const long long* __restrict__ val_off, double* __restrict__ vals, long long ld,
                                    int tl, int ng) {
  __shared__ R red[3 * 32];
  block_sum3<R>(s0, s1, s2, red);
  if (threadIdx.x == 0) {
    const double wt = wts[ld];
    double* v = vals + val_off[ld] + tl;
    v[0] = wt * (double)s0;
    v[ng] = wt * (double)s1;
    v[2 * (long long)ng] = wt * (double)s2;
  }
}

// ---- direct form ----
template <typename R, int KIND>
__global__ void __launch_bounds__(256) k_self_direct(
    const double* __restrict__ dens, const long long* __restrict__ foff3, int p, int pq, const R* __restrict__ wblk,
    long long wstride, const R* __restrict__ ph, const R* __restrict__ T0, const R* __restrict__ cs,
    const R* __restrict__ cache, int ng, const double* __restrict__ wts, const long long* __restrict__ val_off,
    double* __restrict__ vals, int jc) {
  extern __shared__ unsigned char smem_raw[];
  R* rc = reinterpret_cast<R*>(smem_raw);
  const int nc = (p + 1) * (p + 1);
  R* un = rc + 3 * nc;
  const long long t = blockIdx.x;
  const long long ld = t / ng;
  const int tl = (int)(t - ld * ng);
  const int a = tl / (2 * p + 2), b = tl - a * (2 * p + 2);
  const int nq_j = pq + 1, nk = 2 * pq + 2, half = pq + 1;
  const long long nq = (long long)nq_j * nk;
  rotate_target<R>(dens, foff3, ld, p, a, b, wblk, wstride, ph, rc, un);
  const R* geo = cache + t * 7 * nq;
  R s0 = 0, s1 = 0, s2 = 0;
  for (int j0 = 0; j0 < nq_j; j0 += jc) {
    const int jn = min(jc, nq_j - j0);
    legendre_chunk<R>(rc, p, nq_j, j0, jn, T0, un);
    const long long cstride = (long long)jn * (p + 1) * 2;
    for (int i = threadIdx.x; i < jn * half; i += blockDim.x) {
      const int jj = i / half, k = i - jj * half;
      const R* hh = un + (long long)jj * (p + 1) * 2;
      R e0 = hh[0], e1 = hh[cstride], e2 = hh[2 * cstride];
      R o0 = 0, o1 = 0, o2 = 0;
      for (int m = 1; m <= p; ++m) {
        const R co = cs[((long long)m * nk + k) * 2], si = cs[((long long)m * nk + k) * 2 + 1];
        const R* hm = hh + 2 * m;
        const R v0 = 2 * (hm[0] * co - hm[1] * si);
        const R v1 = 2 * (hm[cstride] * co - hm[cstride + 1] * si);
        const R v2 = 2 * (hm[2 * cstride] * co - hm[2 * cstride + 1] * si);
        if (m & 1) {
          o0 += v0;
          o1 += v1;
          o2 += v2;
        } else {
          e0 += v0;
          e1 += v1;
          e2 += v2;
        }
      }
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const long long q = (long long)(j0 + jj) * nk + k + side * half;
        const R r0 = side ? e0 - o0 : e0 + o0;
        const R r1 = side ? e1 - o1 : e1 + o1;
        const R r2 = side ? e2 - o2 : e2 + o2;
        const R x0 = geo[q], x1 = geo[nq + q], x2 = geo[2 * nq + q];
        const R w = geo[6 * nq + q];
        const R ri = rsqrt_<R>(x0 * x0 + x1 * x1 + x2 * x2);
        const R xr = x0 * r0 + x1 * r1 + x2 * r2;
        if (KIND == 0) {
          const R wi = w * ri;
          const R c = wi * xr * ri * ri;
          s0 += wi * r0 + c * x0;
          s1 += wi * r1 + c * x1;
          s2 += wi * r2 + c * x2;
        } else {
          const R xn = x0 * geo[3 * nq + q] + x1 * geo[4 * nq + q] + x2 * geo[5 * nq + q];
          const R ri2 = ri * ri;
          const R c = (R)(-6) * w * xr * xn * ri2 * ri2 * ri;
          s0 += c * x0;
          s1 += c * x1;
          s2 += c * x2;
        }
      }
    }
    __syncthreads();
  }
  write_target<R>(s0, s1, s2, wts, val_off, vals, ld, tl, ng);
}

// ---- Fourier form: set-up of Mhat (FP64, optional FP32 copy) ----
// Mhat[t][e][ri][m][j], e over (xx, yy, zz, xy, xz, yz), ri = real / imaginary part.
constexpr int kDftJ = 3;

template <int KIND>
__global__ void __launch_bounds__(256) k_kernel_dft(const double* __restrict__ cache, int pq, int p,
                                                    const double* __restrict__ cs, double* __restrict__ M64,
                                                    float* __restrict__ M32) {
  __shared__ double sm[kDftJ * 6 * 2 * 132];  // [jj][e][S/D][k < half] for half <= 132
  const long long t = blockIdx.x;
  const int nq_j = pq + 1, nk = 2 * pq + 2, half = pq + 1;
  const long long nq = (long long)nq_j * nk;
  const double* geo = cache + t * 7 * nq;
  const long long plane = (long long)nq_j * (p + 1);
  double* o64 = M64 + t * 12 * plane;
  float* o32 = M32 ? M32 + t * 12 * plane : nullptr;
  for (int j0 = 0; j0 < nq_j; j0 += kDftJ) {
    const int jn = min(kDftJ, nq_j - j0);
    for (int i = threadIdx.x; i < jn * half; i += blockDim.x) {
      const int jj = i / half, k = i - jj * half;
      double Mv[2][6];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const long long q = (long long)(j0 + jj) * nk + k + side * half;
        const double x0 = geo[q], x1 = geo[nq + q], x2 = geo[2 * nq + q], w = geo[6 * nq + q];
        const double ri = 1.0 / sqrt(x0 * x0 + x1 * x1 + x2 * x2);
        double d, c;
        if (KIND == 0) {
          d = w * ri;
          c = w * ri * ri * ri;
        } else {
          const double xn = x0 * geo[3 * nq + q] + x1 * geo[4 * nq + q] + x2 * geo[5 * nq + q];
          const double ri2 = ri * ri;
          d = 0.0;
          c = -6.0 * w * xn * ri2 * ri2 * ri;
        }
        Mv[side][0] = d + c * x0 * x0;
        Mv[side][1] = d + c * x1 * x1;
        Mv[side][2] = d + c * x2 * x2;
        Mv[side][3] = c * x0 * x1;
        Mv[side][4] = c * x0 * x2;
        Mv[side][5] = c * x1 * x2;
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        sm[((jj * 6 + e) * 2 + 0) * 132 + k] = Mv[0][e] + Mv[1][e];  // even orders
        sm[((jj * 6 + e) * 2 + 1) * 132 + k] = Mv[0][e] - Mv[1][e];  // odd orders
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < jn * 6 * (p + 1); i += blockDim.x) {
      const int m = i % (p + 1);
      const int r = i / (p + 1);
      const int e = r % 6, jj = r / 6;
      const double* src = sm + ((jj * 6 + e) * 2 + (m & 1)) * 132;
      double re = 0, im = 0;
      for (int k = 0; k < half; ++k) {
        re += src[k] * cs[((long long)m * nk + k) * 2];
        im += src[k] * cs[((long long)m * nk + k) * 2 + 1];
      }
      const long long o = (long long)m * nq_j + (j0 + jj);  // layout [plane][m][j]
      o64[(2 * e) * plane + o] = re;
      o64[(2 * e + 1) * plane + o] = im;
      if (o32) {
        o32[(2 * e) * plane + o] = (float)re;
        o32[(2 * e + 1) * plane + o] = (float)im;
      }
    }
    __syncthreads();
  }
}

// ---- Fourier form: apply ----
// Shared memory (R = float or double): rcA, rcB [tri(n,m)][6], the rotated coefficients of the two
// targets of a pair, (Re, Im) x 3 components at (n, m >= 0) with tri(n,m) = n(n+1)/2 + m; g4
// [(p+1)^2][4], the phase-shifted input coefficients with the three components interleaved.
// The Legendre step evaluates each Gauss-node pair (t_i, t_{pq-i} = -t_i) at once:
// P~_n^m(-t) = (-1)^(n+m) P~_n^m(t), so with E (n+m even) and O (n+m odd) partial sums,
// h(t_i) = E + O and h(-t_i) = E - O.
template <typename R>
__device__ inline int tri_(int n, int m) {
  return n * (n + 1) / 2 + m;
}

// 128-bit vector of R for shared-memory loads (float4 / double2).
template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
  typedef float4 T;
  static constexpr int n = 4;
};
template <>
struct Vec4<double> {
  typedef double2 T;
  static constexpr int n = 2;
};

// Contraction of h_m(theta_j) (Re, Im x 3 components) with the Fourier factors at (m, j).
template <typename R>
__device__ inline void contract(const R* __restrict__ M, long long plane, long long o, R cm, const R* h, R& s0,
                                R& s1, R& s2) {
  R Mr[6], Mi[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    Mr[e] = M[(2 * e) * plane + o];
    Mi[e] = M[(2 * e + 1) * plane + o];
  }
  // rows of the symmetric matrix: (xx xy xz), (xy yy yz), (xz yz zz); h = (Re, Im) x 3 components
  s0 += cm * (Mr[0] * h[0] + Mr[3] * h[2] + Mr[4] * h[4] - Mi[0] * h[1] - Mi[3] * h[3] - Mi[4] * h[5]);
  s1 += cm * (Mr[3] * h[0] + Mr[1] * h[2] + Mr[5] * h[4] - Mi[3] * h[1] - Mi[1] * h[3] - Mi[5] * h[5]);
  s2 += cm * (Mr[4] * h[0] + Mr[5] * h[2] + Mr[2] * h[4] - Mi[4] * h[1] - Mi[5] * h[3] - Mi[2] * h[5]);
}

// Target pairs: the targets (theta_a, phi_b) and (theta_a, phi_b + pi) share the latitude's Wigner
// blocks, and e^{i m (phi + pi)} = (-1)^m e^{i m phi}, so even-m and odd-m partial sums E, O of one
// pass over the blocks give the rotated coefficients of both (E + O and E - O).  The pair also
// shares every Legendre table load.  rc is stored with 6 entries per (n, m): (Re, Im) x 3 components.
template <typename R, typename CT>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_self_fourier(
    const CT* __restrict__ dens, const long long* __restrict__ foff3, int p, int pq, const R* __restrict__ wblk,
    long long wstride, const R* __restrict__ ph, const R* __restrict__ T0, const R* __restrict__ Mhat, int ng,
    const double* __restrict__ wts, const long long* __restrict__ val_off, double* __restrict__ vals) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ntri = (p + 1) * (p + 2) / 2;
  const int nc = (p + 1) * (p + 1);
  // rc [tri(n,m)][12]: target A (Re, Im) x 3 components, then target B, 16-byte aligned records
  R* rc = reinterpret_cast<R*>(smem_raw);
  R* g4 = rc + 12 * ntri;                   // [(p+1)^2][4]: three components interleaved, padded
  const int half_b = p + 1;                 // targets per latitude pair group
  const long long tp = blockIdx.x;          // target pair
  const long long ld = tp / (ng / 2);
  const int r = (int)(tp - ld * (ng / 2));
  const int a = r / half_b, b = r - a * half_b;
  const int nb = 2 * p + 2;
  const int tlA = a * nb + b, tlB = tlA + half_b;
  const long long tA = ld * ng + tlA, tB = ld * ng + tlB;
  typedef typename Vec4<R>::T V4;
  // stage 0: g = e^{i m phi_b} rho_n^m
  for (int i = threadIdx.x; i < 3 * nc; i += blockDim.x) {
    const int c = i / nc, rr = i - c * nc;
    const int n = degree_of(rr);
    const int m = rr - n * (n + 1);
    if (m < 0) continue;
    const CT* f = dens + foff3[ld * 3 + c];
    const R fr = (R)f[n * (n + 1) + m];
    const R fi = m > 0 ? (R)f[n * (n + 1) - m] : (R)0;
    const R co = ph[((long long)m * nb + b) * 2], si = ph[((long long)m * nb + b) * 2 + 1];
    g4[(n * (n + 1) + m) * 4 + c] = fr * co - fi * si;
    if (m > 0) g4[(n * (n + 1) - m) * 4 + c] = fr * si + fi * co;
  }
  __syncthreads();
  // stage 1: rotation of both targets in one pass (even / odd orders)
  const R* blk = wblk + (long long)a * wstride;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int n = degree_of(i);
    const int o = i - n * n;
    const long long boff = (long long)n * (n + 1) * (2 * n + 1) / 6 + (long long)(n - 1) * n * (2 * n - 1) / 6;
    const R* g = g4 + n * (n + 1) * 4;
    R e0 = 0, e1 = 0, e2 = 0, d0 = 0, d1 = 0, d2 = 0;
    if (o <= n) {
      const R* Cc = blk + boff + o;
      for (int m = 0; m <= n; m += 2) {
        const R cv = Cc[(long long)m * (n + 1)];
        const R* gm = g + 4 * m;
        e0 += cv * gm[0];
        e1 += cv * gm[1];
        e2 += cv * gm[2];
      }
      for (int m = 1; m <= n; m += 2) {
        const R cv = Cc[(long long)m * (n + 1)];
        const R* gm = g + 4 * m;
        d0 += cv * gm[0];
        d1 += cv * gm[1];
        d2 += cv * gm[2];
      }
      R* q = rc + tri_<R>(n, o) * 12;
      q[0] = e0 + d0, q[2] = e1 + d1, q[4] = e2 + d2;
      q[6] = e0 - d0, q[8] = e1 - d1, q[10] = e2 - d2;
      if (o == 0) q[1] = q[3] = q[5] = q[7] = q[9] = q[11] = 0;
    } else {
      const int mp = o - n;
      const R* Sc = blk + boff + (long long)(n + 1) * (n + 1) + (mp - 1);
      for (int m = 2; m <= n; m += 2) {
        const R sv = Sc[(long long)(m - 1) * n];
        const R* gm = g - 4 * m;
        e0 += sv * gm[0];
        e1 += sv * gm[1];
        e2 += sv * gm[2];
      }
      for (int m = 1; m <= n; m += 2) {
        const R sv = Sc[(long long)(m - 1) * n];
        const R* gm = g - 4 * m;
        d0 += sv * gm[0];
        d1 += sv * gm[1];
        d2 += sv * gm[2];
      }
      R* q = rc + tri_<R>(n, mp) * 12;
      q[1] = e0 + d0, q[3] = e1 + d1, q[5] = e2 + d2;
      q[7] = e0 - d0, q[9] = e1 - d1, q[11] = e2 - d2;
    }
  }
  __syncthreads();
  // stages 2-3: Legendre step per (order m, node pair i) for both targets, contracted at once
  const int nq_j = pq + 1;
  const int npair = (nq_j + 1) / 2;
  const long long plane = (long long)nq_j * (p + 1);
  const R* MA = Mhat + tA * 12 * plane;
  const R* MB = Mhat + tB * 12 * plane;
  R sa0 = 0, sa1 = 0, sa2 = 0, sb0 = 0, sb1 = 0, sb2 = 0;
  const int nitem = (p + 1) * npair;
  constexpr int NV = 12 / Vec4<R>::n;  // vector loads per rc record
  for (int it = threadIdx.x; it < nitem; it += blockDim.x) {
    const int m = it / npair, i = it - m * npair;
    R e[12], o[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) e[k] = o[k] = 0;
    const R* Tm = T0 + leg_row(p, m, m, nq_j) + i;
    for (int n = m; n <= p; n += 2) {  // n + m even
      const V4* q = reinterpret_cast<const V4*>(rc + tri_<R>(n, m) * 12);
      const R tv = Tm[(long long)(n - m) * nq_j];
      R v[12];
#pragma unroll
      for (int u = 0; u < NV; ++u) *reinterpret_cast<V4*>(v + u * Vec4<R>::n) = q[u];
#pragma unroll
      for (int k = 0; k < 12; ++k) e[k] += v[k] * tv;
    }
    for (int n = m + 1; n <= p; n += 2) {  // n + m odd
      const V4* q = reinterpret_cast<const V4*>(rc + tri_<R>(n, m) * 12);
      const R tv = Tm[(long long)(n - m) * nq_j];
      R v[12];
#pragma unroll
      for (int u = 0; u < NV; ++u) *reinterpret_cast<V4*>(v + u * Vec4<R>::n) = q[u];
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] += v[k] * tv;
    }
    const R cm = m == 0 ? (R)1 : (R)2;
    const int jh = pq - i;
    R hv[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) hv[k] = e[k] + o[k];
    contract<R>(MA, plane, (long long)m * nq_j + i, cm, hv, sa0, sa1, sa2);
#pragma unroll
    for (int k = 0; k < 6; ++k) hv[k] = e[6 + k] + o[6 + k];
    contract<R>(MB, plane, (long long)m * nq_j + i, cm, hv, sb0, sb1, sb2);
    if (jh != i) {
#pragma unroll
      for (int k = 0; k < 6; ++k) hv[k] = e[k] - o[k];
      contract<R>(MA, plane, (long long)m * nq_j + jh, cm, hv, sa0, sa1, sa2);
#pragma unroll
      for (int k = 0; k < 6; ++k) hv[k] = e[6 + k] - o[6 + k];
      contract<R>(MB, plane, (long long)m * nq_j + jh, cm, hv, sb0, sb1, sb2);
    }
  }
  write_target<R>(sa0, sa1, sa2, wts, val_off, vals, ld, tlA, ng);
  __syncthreads();
  write_target<R>(sb0, sb1, sb2, wts, val_off, vals, ld, tlB, ng);
}

// Latitudes per chunk of the direct kernel within a shared-memory budget.
template <typename R>
int pick_jc(int p, int pq, size_t budget, size_t* smem) {
  const size_t nc = (size_t)(p + 1) * (p + 1);
  const size_t fixed = sizeof(R) * 3 * nc;
  int jc = (int)((budget > 2 * fixed ? budget - fixed : 0) / (sizeof(R) * 6 * (p + 1)));
  jc = std::max(1, std::min(jc, pq + 1));
  *smem = fixed + sizeof(R) * std::max(3 * nc, (size_t)6 * (p + 1) * jc);
  return jc;
}

}  // namespace

template <typename R>
int launch_self_direct(int kind, const double* dens, const long long* foff3, long long ndrop, int p, int pq,
                       const R* wblk, long long wstride, const R* ph, const R* T0, const R* cs, const R* cache,
                       const double* wts, const long long* val_off, double* vals, size_t smem_budget,
                       cudaStream_t s) {
  const int ng = (p + 1) * (2 * p + 2);
  const long long nt = ndrop * ng;
  if (nt == 0) return BIE_OK;
  if (nt > 0x7fffffffLL) return BIE_EINVAL;
  size_t smem;
  const int jc = pick_jc<R>(p, pq, smem_budget, &smem);
  auto kern = kind == 0 ? k_self_direct<R, 0> : k_self_direct<R, 1>;
  if (smem > 48 * 1024) BIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)nt, 256, smem, s>>>(dens, foff3, p, pq, wblk, wstride, ph, T0, cs, cache, ng, wts, val_off, vals,
                                       jc);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_kernel_dft(int kind, const double* cache, long long ntarget, int p, int pq, const double* cs, double* M64,
                      float* M32, cudaStream_t s) {
  if (ntarget == 0) return BIE_OK;
  if (pq + 1 > 132 || ntarget > 0x7fffffffLL) return BIE_EINVAL;
  if (kind == 0)
    k_kernel_dft<0><<<(unsigned)ntarget, 256, 0, s>>>(cache, pq, p, cs, M64, M32);
  else
    k_kernel_dft<1><<<(unsigned)ntarget, 256, 0, s>>>(cache, pq, p, cs, M64, M32);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R, typename CT>
int launch_self_fourier(const CT* dens, const long long* foff3, long long ndrop, int p, int pq, const R* wblk,
                        long long wstride, const R* ph, const R* T0, const R* Mhat, const double* wts,
                        const long long* val_off, double* vals, cudaStream_t s) {
  const int ng = (p + 1) * (2 * p + 2);
  const long long nt = ndrop * ng;
  if (nt == 0) return BIE_OK;
  if (nt > 0x7fffffffLL) return BIE_EINVAL;
  const size_t smem = sizeof(R) * (12 * (size_t)(p + 1) * (p + 2) / 2 + 4 * (size_t)(p + 1) * (p + 1));
  auto kern = k_self_fourier<R, CT>;
  if (smem > 48 * 1024) BIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)(nt / 2), 256, smem, s>>>(dens, foff3, p, pq, wblk, wstride, ph, T0, Mhat, ng, wts, val_off, vals);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template int launch_self_direct<double>(int, const double*, const long long*, long long, int, int, const double*,
                                        long long, const double*, const double*, const double*, const double*,
                                        const double*, const long long*, double*, size_t, cudaStream_t);
template int launch_self_direct<float>(int, const double*, const long long*, long long, int, int, const float*,
                                       long long, const float*, const float*, const float*, const float*,
                                       const double*, const long long*, double*, size_t, cudaStream_t);
template int launch_self_fourier<double, double>(const double*, const long long*, long long, int, int,
                                                 const double*, long long, const double*, const double*,
                                                 const double*, const double*, const long long*, double*,
                                                 cudaStream_t);
template int launch_self_fourier<float, float>(const float*, const long long*, long long, int, int, const float*,
                                               long long, const float*, const float*, const float*, const double*,
                                               const long long*, double*, cudaStream_t);

}  // namespace bie
