// Singular self interaction of every drop (Thm 1, Sec. 2.2, App. B): one block per target.
//
// Both forms rotate the density so that the target sits at the pole (App. B, real blocks of the
// latitude's Wigner matrices applied to e^{i m phi_b} rho_n^m).
//
//  * direct form: the Legendre step of the synthesis on the degree-pq grid,
//    h_m(theta_j) = sum_n rho'_n^m P~_n^m(cos theta_j), runs in shared memory; the phi step rho'(theta_j, phi_k) = h_0 + 2 Re sum_m h_m e^{i m phi_k} is evaluated
//    for the longitude pair (k, k + pq + 1) from the even and odd orders, and the Stokeslet or
//    stresslet pair sum of Thm 1 is accumulated against the cached rotated geometry;
//  * projected form: the same double sum reassociated exactly,
//        sum_{j,k} M_jk rho'_jk = sum_j sum_m c_m Re[ Mhat_jm h_m(theta_j) ]
//                               = sum_{n, m >= 0} Re[ Q_nm rho'_n^m ],   Q_nm = c_m sum_j Mhat_jm P~_n^m(cos theta_j),
//    with c_0 = 1, c_m = 2, M_jk the 3x3 kernel weight of the quadrature point
//    (w^s_j K(x0 - x') W'/sin theta_j, geometry only) and Mhat_jm = sum_k M_jk e^{i m phi_k} its phi
//    transform.  Q (6 complex entries per (n, m) and target) is built once per geometry; an apply
//    then rotates the density and contracts it with Q, without the Legendre step.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dfloat.cuh"
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

// ---- projected form: set-up of Q (FP64, optional FP32 copy) ----
// For each target, Q[t][e][ri][tri(n,m)] = c_m sum_j Mhat_{e,jm} P~_n^m(cos theta_j), with
// Mhat_{e,jm} = sum_k M_{e,jk} e^{i m phi_k} the phi transform of entry e of the 3x3 kernel weight
// over (xx, yy, zz, xy, xz, yz), ri = real / imaginary part, c_0 = 1 and c_m = 2.  Latitudes are
// processed kDftJ at a time: kernel weights, their phi transform, then the Legendre projection,
// accumulated in shared memory.
constexpr int kDftJ = 3;

__device__ inline int tri_index_degree(int it) {
  int n = (int)((sqrt(8.0 * it + 1.0) - 1.0) * 0.5);
  while ((n + 1) * (n + 2) / 2 <= it) ++n;
  while (n * (n + 1) / 2 > it) --n;
  return n;
}

template <int KIND>
__global__ void __launch_bounds__(256) k_kernel_proj(const double* __restrict__ cache, int pq, int p,
                                                     const double* __restrict__ cs, const double* __restrict__ T0,
                                                     double* __restrict__ Q64, float* __restrict__ Q32) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long t = blockIdx.x;
  const int nq_j = pq + 1, nk = 2 * pq + 2, half = pq + 1;
  const int ntri = (p + 1) * (p + 2) / 2;
  double* sg = reinterpret_cast<double*>(smem_raw);  // [jj][e][even/odd][k < half]
  double* sm = sg + kDftJ * 12 * half;               // [jj][12][m]
  double* sq = sm + kDftJ * 12 * (p + 1);            // [12][tri]
  const long long nq = (long long)nq_j * nk;
  const double* geo = cache + t * 7 * nq;
  for (int i = threadIdx.x; i < 12 * ntri; i += blockDim.x) sq[i] = 0.0;
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
        sg[((jj * 6 + e) * 2 + 0) * half + k] = Mv[0][e] + Mv[1][e];  // even orders
        sg[((jj * 6 + e) * 2 + 1) * half + k] = Mv[0][e] - Mv[1][e];  // odd orders
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < jn * 6 * (p + 1); i += blockDim.x) {
      const int m = i % (p + 1);
      const int r = i / (p + 1);
      const int e = r % 6, jj = r / 6;
      const double* src = sg + ((jj * 6 + e) * 2 + (m & 1)) * half;
      double re = 0, im = 0;
      for (int k = 0; k < half; ++k) {
        re += src[k] * cs[((long long)m * nk + k) * 2];
        im += src[k] * cs[((long long)m * nk + k) * 2 + 1];
      }
      sm[(jj * 12 + 2 * e) * (p + 1) + m] = re;
      sm[(jj * 12 + 2 * e + 1) * (p + 1) + m] = im;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < ntri; it += blockDim.x) {
      const int n = tri_index_degree(it);
      const int m = it - n * (n + 1) / 2;
      const double* Tn = T0 + leg_row(p, m, n, nq_j) + j0;
      double acc[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) acc[e] = sq[e * ntri + it];
      for (int jj = 0; jj < jn; ++jj) {
        const double P = Tn[jj];
#pragma unroll
        for (int e = 0; e < 12; ++e) acc[e] += sm[(jj * 12 + e) * (p + 1) + m] * P;
      }
#pragma unroll
      for (int e = 0; e < 12; ++e) sq[e * ntri + it] = acc[e];
    }
    __syncthreads();
  }
  // The apply adds every product with a plus sign: the imaginary planes of targets on latitudes
  // a <= p/2 are stored negated (imaginary parts enter as -Q_im), and targets on latitudes a > p/2,
  // which the apply reaches as the mirror pi - theta of a lower latitude, carry (-1)^(n+m).
  double* o64 = Q64 + t * 12 * ntri;
  float* o32 = Q32 ? Q32 + t * 12 * ntri : nullptr;
  const int nbl = 2 * p + 2;
  const int lat = (int)((t % ((long long)(p + 1) * nbl)) / nbl);
  const bool mirror = 2 * lat > p;
  for (int i = threadIdx.x; i < 12 * ntri; i += blockDim.x) {
    const int it = i % ntri, plane = i / ntri;
    const int n = tri_index_degree(it);
    const int m = it - n * (n + 1) / 2;
    double v = (m == 0 ? 1.0 : 2.0) * sq[i];  // c_m
    if (mirror) {
      if ((n + m) & 1) v = -v;
    } else if (plane & 1) {
      v = -v;
    }
    o64[i] = v;
    if (o32) o32[i] = (float)v;
  }
}

// ---- projected form: apply ----
// One block per target quadruple: the latitudes theta_a and pi - theta_a (Gauss nodes t and -t) at the
// longitudes phi_b and phi_b + pi.  One pass over latitude a's real Wigner blocks (C for the real
// parts, S for the imaginary parts, column m the input order) gives the even-m and odd-m partial sums
// E and O of every rotated coefficient (n, m'), and the four targets follow exactly:
//   phi_b + pi:     e^{i m (phi + pi)} = (-1)^m e^{i m phi}                    -> E - O
//   pi - theta_a:   d^n_{m m'}(pi - beta) = (-1)^(n + m') d^n_{-m m'}(beta), so
//                   C' = (-1)^(n + m' + m) C and S' = -(-1)^(n + m' + m) S      -> +-(-1)^(n + m') (E -+ O)
// Each rotated coefficient is contracted at once with the targets' projected kernel factors Q
// (real parts with the real planes, imaginary parts with minus the imaginary planes), so rotated
// coefficients never leave registers.  The middle latitude of an odd node count (t = 0) pairs with
// itself and its block has two targets.  Shared memory: g4 [(p+1)^2][4], the phase-shifted input
// coefficients e^{i m phi_b} rho_n^m with the three components interleaved.
constexpr int kSelfThreads = 256;

// acc += S v for the symmetric 3x3 matrix S with entries (xx, yy, zz, xy, xz, yz) at planes q[0..5]
template <typename R>
__device__ inline void sym_mul_add(const R* q, const R* v, R* acc) {
  acc[0] = fmad(q[4], v[2], fmad(q[3], v[1], fmad(q[0], v[0], acc[0])));
  acc[1] = fmad(q[5], v[2], fmad(q[1], v[1], fmad(q[3], v[0], acc[1])));
  acc[2] = fmad(q[2], v[2], fmad(q[5], v[1], fmad(q[4], v[0], acc[2])));
}

// One launch covers every degree group (a persistent batch over drops of uneven degree): the groups'
// arguments travel by value, block ranges in descending degree so that the longest blocks start first.
template <typename R, typename CT>
__global__ void __launch_bounds__(kSelfThreads, sizeof(R) == 4 ? 4 : 2) k_self_proj(
    SelfGroups<R> G, const CT* __restrict__ dens, double* __restrict__ vals) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red[kSelfThreads / 32][12];
  SelfGroup<R> A = G.g[0];
#pragma unroll
  for (int i = 1; i < kMaxSelfGroups; ++i)
    if (i < G.n && (long long)blockIdx.x >= G.g[i].begin) A = G.g[i];
  const int p = A.p;
  const long long* __restrict__ foff3 = A.foff3;
  const R* __restrict__ wblk = A.wblk;
  const long long wstride = A.wstride;
  const R* __restrict__ ph = A.ph;
  const R* __restrict__ Q = A.Q;
  const double* __restrict__ wts = A.wts;
  const long long* __restrict__ val_off = A.val_off;
  const int ntri = (p + 1) * (p + 2) / 2;
  const int nc = (p + 1) * (p + 1);
  const int ng = (p + 1) * (2 * p + 2);
  R* g4 = reinterpret_cast<R*>(smem_raw);  // [(p+1)^2][4]
  const int hb = p + 1, nb = 2 * p + 2, na2 = (p + 2) / 2;
  const long long bid = (long long)blockIdx.x - A.begin;
  const long long ld = bid / ((long long)na2 * hb);
  const int r = (int)(bid - ld * na2 * hb);
  const int a = r / hb, b = r - a * hb;
  const int a2 = p - a;
  const bool quad = a2 != a;
  const int tlA = a * nb + b, tlC = a2 * nb + b;  // targets A, B = A + hb, C, D = C + hb
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
  // stages 1-2: rotation (even / odd input orders) and contraction, per rotated coefficient
  const R* blk = wblk + (long long)a * wstride;
  const long long qstride = 12 * (long long)ntri;
  const R* QA = Q + (ld * ng + tlA) * qstride;
  const R* QC = Q + (ld * ng + tlC) * qstride;
  const R* Qk_[4] = {QA, QA + hb * qstride, QC, QC + hb * qstride};
  R acc[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int n = degree_of(i);
    const int o = i - n * n;
    const long long boff = (long long)n * (n + 1) * (2 * n + 1) / 6 + (long long)(n - 1) * n * (2 * n - 1) / 6;
    const R* g = g4 + n * (n + 1) * 4;
    const bool re = o <= n;
    const int mo = re ? o : o - n;  // output order m'
    const int t = n * (n + 1) / 2 + mo;
    const int ri = re ? 0 : 1;      // real or imaginary planes of Q
    R q[4][6];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k < 2 || quad) {
        const R* Qk = Qk_[k] + t;
#pragma unroll
        for (int e = 0; e < 6; ++e) q[k][e] = Qk[(2 * e + ri) * (long long)ntri];
      }
    }
    R E[3] = {0, 0, 0}, O[3] = {0, 0, 0};
    if (re) {
      const R* Cc = blk + boff + o;
      int m = 0;
#pragma unroll 2
      for (; m + 1 <= n; m += 2) {
        const R cv = Cc[(long long)m * (n + 1)], cw = Cc[(long long)(m + 1) * (n + 1)];
        const R* gm = g + 4 * m;
        E[0] += cv * gm[0];
        E[1] += cv * gm[1];
        E[2] += cv * gm[2];
        O[0] += cw * gm[4];
        O[1] += cw * gm[5];
        O[2] += cw * gm[6];
      }
      if (m <= n) {
        const R cv = Cc[(long long)m * (n + 1)];
        const R* gm = g + 4 * m;
        E[0] += cv * gm[0];
        E[1] += cv * gm[1];
        E[2] += cv * gm[2];
      }
    } else {
      const R* Sc = blk + boff + (long long)(n + 1) * (n + 1) + (mo - 1);
      int m = 1;
#pragma unroll 2
      for (; m + 1 <= n; m += 2) {
        const R sv = Sc[(long long)(m - 1) * n], sw = Sc[(long long)m * n];
        const R* gm = g - 4 * m;
        O[0] += sv * gm[0];
        O[1] += sv * gm[1];
        O[2] += sv * gm[2];
        E[0] += sw * gm[-4];
        E[1] += sw * gm[-3];
        E[2] += sw * gm[-2];
      }
      if (m <= n) {
        const R sv = Sc[(long long)(m - 1) * n];
        const R* gm = g - 4 * m;
        O[0] += sv * gm[0];
        O[1] += sv * gm[1];
        O[2] += sv * gm[2];
      }
    }
    R vp[3], vm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      vp[c] = E[c] + O[c];
      vm[c] = E[c] - O[c];
    }
    // Real parts enter with +Q_re, imaginary parts with -Q_im; latitude pi - theta_a carries
    // (-1)^(n + m') on the real and -(-1)^(n + m') on the imaginary parts.  Both signs are stored in
    // the factors (see k_kernel_proj), so every product is added.
    sym_mul_add<R>(q[0], vp, acc[0]);
    sym_mul_add<R>(q[1], vm, acc[1]);
    if (quad) {
      sym_mul_add<R>(q[2], vm, acc[2]);
      sym_mul_add<R>(q[3], vp, acc[3]);
    }
  }
  // block reduction of the 12 sums
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      for (int off = 16; off > 0; off >>= 1) acc[k][c] += shfl_down(acc[k][c], off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) red[w][k * 3 + c] = acc[k][c];
  __syncthreads();
  const int nt = quad ? 4 : 2;
  if (threadIdx.x < 3 * nt) {
    R v = 0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) v += red[ww][threadIdx.x];
    const int k = threadIdx.x / 3, c = threadIdx.x - 3 * k;
    const int tl = (k < 2 ? tlA : tlC) + (k & 1) * hb;
    vals[val_off[ld] + (long long)c * ng + tl] = wts[ld] * (double)v;
  }
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

// out[i] = the double-float split of in[i]
__global__ void k_split_dff(const double* __restrict__ in, dff* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = dff(in[i]);
}

}  // namespace

int launch_split_dff(const double* in, dff* out, long long n, cudaStream_t s) {
  if (n == 0) return BIE_OK;
  k_split_dff<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

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

size_t kernel_proj_smem(int p, int pq) {
  return sizeof(double) * ((size_t)kDftJ * 12 * (pq + 1) + (size_t)kDftJ * 12 * (p + 1) + 6 * (size_t)(p + 1) * (p + 2));
}

int launch_kernel_proj(int kind, const double* cache, long long ntarget, int p, int pq, const double* cs,
                       const double* T0, double* Q64, float* Q32, cudaStream_t s) {
  if (ntarget == 0) return BIE_OK;
  if (ntarget > 0x7fffffffLL) return BIE_EINVAL;
  const size_t smem = kernel_proj_smem(p, pq);
  if (smem > 227 * 1024) {
    set_error("degree too large for the projected self form (shared memory)");
    return BIE_ENOTSUP;
  }
  auto kern = kind == 0 ? k_kernel_proj<0> : k_kernel_proj<1>;
  if (smem > 48 * 1024) BIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)ntarget, 256, smem, s>>>(cache, pq, p, cs, T0, Q64, Q32);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R, typename CT>
int launch_self_proj(std::vector<SelfGroup<R>> groups, const CT* dens, double* vals, cudaStream_t s) {
  std::sort(groups.begin(), groups.end(), [](const SelfGroup<R>& x, const SelfGroup<R>& y) { return x.p > y.p; });
  for (size_t g0 = 0; g0 < groups.size(); g0 += kMaxSelfGroups) {
    SelfGroups<R> G{};
    G.n = (int)std::min<size_t>(kMaxSelfGroups, groups.size() - g0);
    long long nblk = 0;
    size_t smem = 0;
    for (int i = 0; i < G.n; ++i) {
      G.g[i] = groups[g0 + i];
      const int p = G.g[i].p;
      G.g[i].begin = nblk;
      nblk += G.g[i].ndrop * ((p + 2) / 2) * (p + 1);
      smem = std::max(smem, sizeof(R) * 4 * (size_t)(p + 1) * (p + 1));
      if (G.g[i].ndrop * (long long)(p + 1) * (2 * p + 2) > 0x7fffffffLL) return BIE_EINVAL;
    }
    if (nblk == 0) continue;
    if (nblk > 0x7fffffffLL) return BIE_EINVAL;
    auto kern = k_self_proj<R, CT>;
    if (smem > 48 * 1024) BIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)nblk, kSelfThreads, smem, s>>>(G, dens, vals);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
  }
  return BIE_OK;
}

template int launch_self_direct<double>(int, const double*, const long long*, long long, int, int, const double*,
                                        long long, const double*, const double*, const double*, const double*,
                                        const double*, const long long*, double*, size_t, cudaStream_t);
template int launch_self_direct<float>(int, const double*, const long long*, long long, int, int, const float*,
                                       long long, const float*, const float*, const float*, const float*,
                                       const double*, const long long*, double*, size_t, cudaStream_t);
template int launch_self_proj<double, double>(std::vector<SelfGroup<double>>, const double*, double*, cudaStream_t);
template int launch_self_proj<float, double>(std::vector<SelfGroup<float>>, const double*, double*, cudaStream_t);
template int launch_self_proj<dff, double>(std::vector<SelfGroup<dff>>, const double*, double*, cudaStream_t);

}  // namespace bie
