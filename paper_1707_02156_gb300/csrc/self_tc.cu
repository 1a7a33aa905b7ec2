// Singular self interaction, projected form, FP32 (Thm 1, Sec. 2.2, App. B) with the Wigner
// rotation on the tensor cores.
//
// The rotation of App. B at latitude beta_a, for the density's degree-n coefficients phase-shifted
// to longitude phi_b, g_m = e^{i m phi_b} rho_n^m, is a product with the real blocks of d^n(beta_a):
//     Re rho'_{n m'} = sum_{m=0..n} C[m'][m] Re g_m,   Im rho'_{n m'} = sum_{m=1..n} S[m'-1][m-1] Im g_m.
// Splitting the input orders m by parity gives the even and odd partial sums E, O, from which the
// four targets (theta_a, phi_b), (theta_a, phi_b + pi), (pi - theta_a, phi_b), (pi - theta_a,
// phi_b + pi) follow exactly (the symmetries are those of the CUDA-core kernel k_self_proj).  With
// the block's NB longitudes b, three components and two parities as columns, each degree is the
// matrix product
//     [E | O](m', (b, c, parity)) = W_n(m', m) G_n(m, (b, c, parity)),
// W_n = C (rows m' = 0..n) or S (rows m' = 1..n), G_n(m, (b, c, par)) = g_m(b, c) when m has the
// column's parity and 0 otherwise.  It runs as mma.sync m16n8k8 in TF32 with the 3-pass split
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a = a_hi + a_lo, each part a TF32 number), accumulated in
// FP32, which keeps the products to about FP32 accuracy.  The result goes to shared memory and is
// contracted there with the targets' projected kernel factors Q (CUDA cores, Q streamed from HBM).
//
// One block per (drop, latitude pair a, chunk of NB longitudes); 8 warps share the degree tiles.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace bie {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcWarps = kTcThreads / 32;

__device__ __forceinline__ unsigned tf32_of(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo with hi, lo TF32 (lo carries the next 11 bits of x's significand)
__device__ __forceinline__ void tf32_split(float x, unsigned& hi, unsigned& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}

// d += a b for one m16n8k8 tile (a: 16x8 row-major fragment, b: 8x8 column-major fragment)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void sym_mul_add_f(const float* q, const float* v, float* acc) {
  acc[0] = fmaf(q[4], v[2], fmaf(q[3], v[1], fmaf(q[0], v[0], acc[0])));
  acc[1] = fmaf(q[5], v[2], fmaf(q[1], v[1], fmaf(q[3], v[0], acc[1])));
  acc[2] = fmaf(q[2], v[2], fmaf(q[5], v[1], fmaf(q[4], v[0], acc[2])));
}

// Number of 16-row tiles of the degree-n products: real part n+1 rows, imaginary part n rows.
__device__ __forceinline__ int tiles_of(int n) { return (n + 1 + 15) / 16 + (n + 15) / 16; }

template <int NB>
__global__ void __launch_bounds__(kTcThreads) k_self_tc(SelfGroups<float> G, const double* __restrict__ dens,
                                                        double* __restrict__ vals) {
  constexpr int NCOL = NB * 6;             // columns (b, c, parity)
  constexpr int NTN = (NCOL + 7) / 8;      // 8-column tiles
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float red[kTcWarps][NB * 12];
  SelfGroup<float> A = G.g[0];
#pragma unroll
  for (int i = 1; i < kMaxSelfGroups; ++i)
    if (i < G.n && (long long)blockIdx.x >= G.g[i].begin) A = G.g[i];
  const int p = A.p;
  const int ntri = (p + 1) * (p + 2) / 2;
  const int nc = (p + 1) * (p + 1);
  const int ng = (p + 1) * (2 * p + 2);
  const int hb = p + 1, nb = 2 * p + 2, na2 = (p + 2) / 2;
  const int nbc = (hb + NB - 1) / NB;
  const long long bid = (long long)blockIdx.x - A.begin;
  const long long ld = bid / ((long long)na2 * nbc);
  const int r = (int)(bid - ld * na2 * nbc);
  const int a = r / nbc, b0 = (r - a * nbc) * NB;
  const int nbh = min(NB, hb - b0);
  const int a2 = p - a;
  const bool quad = a2 != a;
  float* gs = reinterpret_cast<float*>(smem_raw);  // [packed (n, m)][NB][3]: Re g (m >= 0), Im g (m < 0)
  float* V = gs + (long long)nc * NB * 3;          // [packed (n, m')][(b, c, parity)]: E, O
  // stage 0: g = e^{i m phi_b} rho_n^m for the block's longitudes (zero past the last one)
  for (int i = threadIdx.x; i < nc * NB * 3; i += blockDim.x) {
    const int c = i % 3, bb = (i / 3) % NB, rr = i / (3 * NB);
    const int n = degree_of(rr);
    const int m = rr - n * (n + 1);
    float v = 0.f;
    if (bb < nbh) {
      const double* f = dens + A.foff3[ld * 3 + c];
      const int mm = m < 0 ? -m : m;
      const float fr = (float)f[n * (n + 1) + mm];
      const float fi = mm > 0 ? (float)f[n * (n + 1) - mm] : 0.f;
      const float co = A.ph[((long long)mm * nb + b0 + bb) * 2], si = A.ph[((long long)mm * nb + b0 + bb) * 2 + 1];
      v = m >= 0 ? fr * co - fi * si : fr * si + fi * co;
    }
    gs[i] = v;
  }
  __syncthreads();
  // stage 1: the rotation products on the tensor cores; the warps take the (degree, part, row tile)
  // units in turn, highest degree first
  const float* blk = A.wblk + (long long)a * A.wstride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  int unit = 0;
  for (int n = p; n >= 0; --n) {
    const int nt_re = (n + 1 + 15) / 16, nt_all = tiles_of(n);
    const long long boff = (long long)n * (n + 1) * (2 * n + 1) / 6 + (long long)(n - 1) * n * (2 * n - 1) / 6;
    for (int u = 0; u < nt_all; ++u, ++unit) {
      if ((unit % kTcWarps) != warp) continue;
      const bool im = u >= nt_re;
      const int mt = im ? u - nt_re : u;
      const int M = im ? n : n + 1;  // rows = output orders; K = input orders (as many)
      float d[NTN][4];
#pragma unroll
      for (int t = 0; t < NTN; ++t) d[t][0] = d[t][1] = d[t][2] = d[t][3] = 0.f;
      const int r0 = mt * 16 + gq, r1 = r0 + 8;
      for (int k0 = 0; k0 < M; k0 += 8) {
        const int c0 = k0 + tq, c1 = c0 + 4;
        // A fragment: W(row, col), W = C column-major (n+1)^2, or S column-major n^2 after C
        float av[4];
        const int rows[4] = {r0, r1, r0, r1}, cols[4] = {c0, c0, c1, c1};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool ok = rows[e] < M && cols[e] < M;
          const long long off = im ? boff + (long long)(n + 1) * (n + 1) + (long long)cols[e] * n + rows[e]
                                   : boff + (long long)cols[e] * (n + 1) + rows[e];
          av[e] = ok ? __ldg(blk + off) : 0.f;
        }
        unsigned ahi[4], alo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) tf32_split(av[e], ahi[e], alo[e]);
#pragma unroll
        for (int t = 0; t < NTN; ++t) {
          // B fragment: rows k (input order index), column j = (b, c, parity)
          const int j = t * 8 + gq;
          const int kk[2] = {k0 + tq, k0 + tq + 4};
          unsigned bhi[2], blo[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            float bv = 0.f;
            const int m = im ? kk[e] + 1 : kk[e];
            if (kk[e] < M && j < NCOL && (m & 1) == (j & 1)) {
              const int bb = j / 6, c = (j >> 1) % 3;
              const int pk = im ? n * (n + 1) - m : n * (n + 1) + m;
              bv = gs[(pk * NB + bb) * 3 + c];
            }
            tf32_split(bv, bhi[e], blo[e]);
          }
          mma_tf32(d[t], alo, bhi);
          mma_tf32(d[t], ahi, blo);
          mma_tf32(d[t], ahi, bhi);
        }
      }
      // D fragment: rows r0 / r1 (output order m' = row, or row + 1 for the imaginary part), columns
      // 2 tq, 2 tq + 1 of each tile
#pragma unroll
      for (int t = 0; t < NTN; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = e < 2 ? r0 : r1, col = t * 8 + 2 * tq + (e & 1);
          if (row < M && col < NCOL) {
            const int pk = im ? n * (n + 1) - (row + 1) : n * (n + 1) + row;
            V[pk * NCOL + col] = d[t][e];
          }
        }
    }
  }
  __syncthreads();
  // stage 2: contraction of every rotated coefficient with the four targets' factors (as k_self_proj:
  // real parts with the real planes, imaginary parts with the imaginary planes, whose signs the
  // factors carry)
  float acc[NB][4][3];
#pragma unroll
  for (int bb = 0; bb < NB; ++bb)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[bb][k][0] = acc[bb][k][1] = acc[bb][k][2] = 0.f;
  const long long qstride = 12 * (long long)ntri;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int n = degree_of(i);
    const int o = i - n * n;
    const bool re = o <= n;
    const int mo = re ? o : o - n;
    const int t = n * (n + 1) / 2 + mo;
    const int ri = re ? 0 : 1;
    const int pk = re ? n * (n + 1) + mo : n * (n + 1) - mo;
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
      if (bb >= nbh) break;
      const int b = b0 + bb;
      const float* v = V + pk * NCOL + bb * 6;
      float vp[3], vm[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vp[c] = v[2 * c] + v[2 * c + 1];
        vm[c] = v[2 * c] - v[2 * c + 1];
      }
      const long long tl[4] = {a * nb + b, a * nb + b + hb, a2 * nb + b, a2 * nb + b + hb};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= 2 && !quad) break;
        const float* Qk = A.Q + (ld * ng + tl[k]) * qstride + t;
        float q[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) q[e] = __ldg(Qk + (2 * e + ri) * (long long)ntri);
        sym_mul_add_f(q, (k == 0 || k == 3) ? vp : vm, acc[bb][k]);
      }
    }
  }
  // block reduction of the NB x 12 sums
#pragma unroll
  for (int bb = 0; bb < NB; ++bb)
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        for (int off = 16; off > 0; off >>= 1) acc[bb][k][c] += __shfl_down_sync(0xffffffffu, acc[bb][k][c], off);
  if (lane == 0)
#pragma unroll
    for (int bb = 0; bb < NB; ++bb)
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) red[warp][(bb * 4 + k) * 3 + c] = acc[bb][k][c];
  __syncthreads();
  for (int i = threadIdx.x; i < NB * 12; i += blockDim.x) {
    const int bb = i / 12, k = (i / 3) % 4, c = i % 3;
    if (bb >= nbh || (k >= 2 && !quad)) continue;
    float v = 0.f;
    for (int w = 0; w < kTcWarps; ++w) v += red[w][i];
    const int b = b0 + bb;
    const int tl = (k < 2 ? a * nb : a2 * nb) + b + (k & 1) * hb;
    vals[A.val_off[ld] + (long long)c * ng + tl] = A.wts[ld] * (double)v;
  }
}

}  // namespace

size_t self_tc_smem(int p, int nbl) { return sizeof(float) * 9 * (size_t)(p + 1) * (p + 1) * nbl; }

int launch_self_tc(std::vector<SelfGroup<float>> groups, const double* dens, double* vals, cudaStream_t s) {
  std::sort(groups.begin(), groups.end(), [](const SelfGroup<float>& x, const SelfGroup<float>& y) { return x.p > y.p; });
  for (size_t g0 = 0; g0 < groups.size(); g0 += kMaxSelfGroups) {
    SelfGroups<float> G{};
    G.n = (int)std::min<size_t>(kMaxSelfGroups, groups.size() - g0);
    long long nblk = 0;
    size_t smem = 0;
    for (int i = 0; i < G.n; ++i) {
      G.g[i] = groups[g0 + i];
      const int p = G.g[i].p;
      G.g[i].begin = nblk;
      nblk += G.g[i].ndrop * ((p + 2) / 2) * (long long)(p + 1);  // NB = 1: one block per longitude
      smem = std::max(smem, self_tc_smem(p, 1));
      if (G.g[i].ndrop * (long long)(p + 1) * (2 * p + 2) > 0x7fffffffLL) return BIE_EINVAL;
    }
    if (nblk == 0) continue;
    if (nblk > 0x7fffffffLL) return BIE_EINVAL;
    if (smem > 227 * 1024) {
      set_error("degree too large for the tensor-core self kernel (shared memory)");
      return BIE_ENOTSUP;
    }
    auto kern = k_self_tc<1>;
    if (smem > 48 * 1024) BIE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)nblk, kTcThreads, smem, s>>>(G, dens, vals);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
  }
  return BIE_OK;
}

}  // namespace bie
