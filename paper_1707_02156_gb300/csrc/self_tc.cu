// Singular self interaction, projected form, FP32 (Thm 1, Sec. 2.2, App. B) with the Wigner
// rotation on the tensor cores.
//
// The rotation of App. B at latitude beta_a, for the density's degree-n coefficients phase-shifted
// to longitude phi_b, g_m = e^{i m phi_b} rho_n^m, is a product with the real blocks of d^n(beta_a):
//     Re rho'_{n m'} = sum_{m=0..n} C[m'][m] Re g_m,   Im rho'_{n m'} = sum_{m=1..n} S[m'-1][m-1] Im g_m.
// Splitting the input orders m by parity gives the even and odd partial sums E, O, from which the
// four targets (theta_a, phi_b), (theta_a, phi_b + pi), (pi - theta_a, phi_b), (pi - theta_a,
// phi_b + pi) follow exactly (the symmetries of the CUDA-core kernel k_self_proj).  With every
// longitude b < p+1 of the latitude, the three components and the two parities as columns, each
// (latitude, degree) is one matrix product
//     [E | O](m', (b, c, parity)) = W(m', m) G(m, (b, c, parity)),
// W = C (rows m' = 0..n) or S (rows m' = 1..n), G(m, (b, c, par)) = g_m(b, c) when m has the
// column's parity, else 0.  k_rot_tc runs these products as mma.sync m16n8k8 in TF32 with the
// 3-pass split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (x = x_hi + x_lo, both TF32), accumulated in
// FP32 (about FP32 accuracy), from the phase-shifted coefficients that k_phase_g forms once per apply
// for every longitude (already split into TF32 hi / lo parts), with K split by the parity of m (no zero
// padding), and writes E and O to a buffer that stays in L2 for one drop's worth
// of latitudes (drops are taken in chunks whose sums fit a fixed buffer); k_contract_eo then streams the projected kernel factors Q from HBM and contracts
// them with E +- O, one block per target quadruple.
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

// The rotated sums of one launch (a chunk of drops of one degree): EO[ld][a][packed (n, m')][b][c][parity],
// so that a tile row of the products (one output order, eight (b, c, parity) columns) is 32
// contiguous bytes.  eo_row = the offset of (ld, a, packed index pk).
__device__ __forceinline__ long long eo_row(long long ld, int a, int pk, int p) {
  const int hb = p + 1, na2 = (p + 2) / 2, nc = (p + 1) * (p + 1);
  return ((ld * na2 + a) * (long long)nc + pk) * (long long)hb * 6;
}

// The phase-shifted coefficients g = e^{i m phi_b} rho_n^m of every longitude b < p+1, shared by all
// latitudes, already split for the 3-pass products: Ghi, Glo[ld][packed (n, mm)][b][c] = the TF32 hi /
// lo parts of Re g (mm >= 0) or Im g (mm < 0) of |mm|.
__global__ void k_phase_g(SelfGroup<float> A, const double* __restrict__ dens, unsigned* __restrict__ Ghi,
                          unsigned* __restrict__ Glo) {
  const int p = A.p;
  const int hb = p + 1, nb = 2 * p + 2, nc = (p + 1) * (p + 1);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= A.ndrop * (long long)nc * hb * 3) return;
  const int c = (int)(idx % 3), b = (int)((idx / 3) % hb);
  const long long r = idx / (3LL * hb);
  const int pk = (int)(r % nc);
  const long long ld = r / nc;
  const int n = degree_of(pk);
  const int mm = pk - n * (n + 1);
  const int m = mm < 0 ? -mm : mm;
  const double* f = dens + A.foff3[ld * 3 + c];
  const float fr = (float)f[n * (n + 1) + m];
  const float fi = m > 0 ? (float)f[n * (n + 1) - m] : 0.f;
  const float co = A.ph[((long long)m * nb + b) * 2], si = A.ph[((long long)m * nb + b) * 2 + 1];
  unsigned hi, lo;
  tf32_split(mm >= 0 ? fr * co - fi * si : fr * si + fi * co, hi, lo);
  Ghi[idx] = hi;
  Glo[idx] = lo;
}

// One block per (drop, latitude pair a, degree n).  The products are split by the parity of the input
// order, E = W[:, even m] G[even m, (b, c)] and O = W[:, odd m] G[odd m, (b, c)], so that no operand
// carries zero padding: K = the orders of one parity, N = (b, c) = 3 (p+1) columns.  The block stages
// W's columns of each parity already split into TF32 hi / lo parts, and the degree's rows of the
// phase-shifted coefficients G.  A warp owns one (part, parity, 16-row tile, half of N) and runs its
// k-steps once, building the A fragment once per k-step and reusing it over up to 13 column tiles.
constexpr int kRotMaxNt = 13;  // 8-column tiles per warp pass (N = 3 (p+1) takes one or two passes for p < 64)

__global__ void __launch_bounds__(kTcThreads) k_rot_tc(SelfGroup<float> A, const unsigned* __restrict__ Ghi,
                                                       const unsigned* __restrict__ Glo, float* __restrict__ EO) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = A.p;
  const int hb = p + 1;
  const long long bid = blockIdx.x;
  const int n = (int)(bid % (p + 1));
  const long long r = bid / (p + 1);
  const int na2 = (p + 2) / 2;
  const int a = (int)(r % na2);
  const long long ld = r / na2;
  const int NC3 = hb * 3;                // columns (b, c)
  const int NTN = (NC3 + 7) / 8;         // 8-column tiles
  // A operands: for part (re: C, rows m' = 0..n; im: S, rows m' = 1..n) and parity q, column kk is the
  // input order m = 2 kk + q (re) or m = 2 kk + q + ... (im: m = 1..n), stored [part][q][row][kk] as
  // TF32 hi and lo bit patterns; kq(part, q) columns, padded to a multiple of 8
  const int Mre = n + 1, Mim = n;
  const int kre0 = (n + 2) / 2, kre1 = (n + 1) / 2;  // even / odd orders among 0..n
  const int kim1 = (n + 1) / 2, kim0 = n / 2;        // odd / even orders among 1..n
  auto pad8 = [](int v) { return (v + 7) & ~7; };
  const int ka[2][2] = {{pad8(kre0), pad8(kre1)}, {pad8(kim0), pad8(kim1)}};
  unsigned* Ahi = reinterpret_cast<unsigned*>(smem_raw);
  long long aoff[2][2], acur = 0;
  for (int part = 0; part < 2; ++part)
    for (int q = 0; q < 2; ++q) {
      aoff[part][q] = acur;
      acur += (long long)(part ? Mim : Mre) * ka[part][q];
    }
  unsigned* Alo = Ahi + acur;
  unsigned* Gh = Alo + acur;                  // [n + mm][b][c], mm = -n..n: TF32 hi parts
  unsigned* Gl = Gh + (2 * n + 1) * NC3;      // and lo parts
  const long long boff = (long long)n * (n + 1) * (2 * n + 1) / 6 + (long long)(n - 1) * n * (2 * n - 1) / 6;
  const float* blk = A.wblk + (long long)a * A.wstride + boff;
  // the degree's rows of G go to shared memory by asynchronous 4-byte copies, all in flight at once
  const long long goff = ((ld * (p + 1) * (p + 1)) + (long long)n * n) * NC3;
  for (int i = threadIdx.x; i < (2 * n + 1) * NC3; i += blockDim.x) {
    const unsigned dh = (unsigned)__cvta_generic_to_shared(Gh + i), dl = (unsigned)__cvta_generic_to_shared(Gl + i);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dh), "l"(Ghi + goff + i) : "memory");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dl), "l"(Glo + goff + i) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  // W's columns of each parity, split into TF32 hi / lo: the loads of a thread's entries are issued
  // together (eight per batch) before any is split and stored
  for (int part = 0; part < 2; ++part)
    for (int q = 0; q < 2; ++q) {
      const int M = part ? Mim : Mre, K = ka[part][q];
      const int total = M * K;
      for (int i0 = threadIdx.x; i0 < total; i0 += 8 * blockDim.x) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * blockDim.x;
          v[u] = 0.f;
          if (i < total) {
            const int row = i / K, kk = i - row * K;
            // input order of column kk: m = 2 kk + q (re, m = 0..n); odd m = 2 kk + 1, even m = 2 kk + 2 (im)
            const int m = part ? (q ? 2 * kk + 1 : 2 * kk + 2) : 2 * kk + q;
            if (m <= n)
              v[u] = part ? __ldg(blk + (long long)(n + 1) * (n + 1) + (long long)(m - 1) * n + row)  // S
                          : __ldg(blk + (long long)m * (n + 1) + row);                                // C
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * blockDim.x;
          if (i < total) {
            unsigned hi, lo;
            tf32_split(v[u], hi, lo);
            Ahi[aoff[part][q] + i] = hi;
            Alo[aoff[part][q] + i] = lo;
          }
        }
      }
    }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const int mt[2] = {(Mre + 15) / 16, (Mim + 15) / 16};
  const int npass = (NTN + kRotMaxNt - 1) / kRotMaxNt;
  const int units = 2 * (mt[0] + mt[1]) * npass;
  for (int u = warp; u < units; u += kTcWarps) {
    const int pass = u % npass, uq = u / npass;
    const int q = uq & 1, mu = uq >> 1;
    const int t0 = pass * kRotMaxNt;
    const int part = mu >= mt[0] ? 1 : 0;
    const int tile = part ? mu - mt[0] : mu;
    const int M = part ? Mim : Mre, K = ka[part][q];
    const unsigned* Ah = Ahi + aoff[part][q];
    const unsigned* Al = Alo + aoff[part][q];
    const int r0 = tile * 16 + gq, r1 = r0 + 8;
    float d[kRotMaxNt][4];
#pragma unroll
    for (int t = 0; t < kRotMaxNt; ++t) d[t][0] = d[t][1] = d[t][2] = d[t][3] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 8) {
      const int c0 = k0 + tq, c1 = c0 + 4;
      unsigned ahi[4], alo[4];
      ahi[0] = r0 < M ? Ah[r0 * K + c0] : 0u;
      ahi[1] = r1 < M ? Ah[r1 * K + c0] : 0u;
      ahi[2] = r0 < M ? Ah[r0 * K + c1] : 0u;
      ahi[3] = r1 < M ? Ah[r1 * K + c1] : 0u;
      alo[0] = r0 < M ? Al[r0 * K + c0] : 0u;
      alo[1] = r1 < M ? Al[r1 * K + c0] : 0u;
      alo[2] = r0 < M ? Al[r0 * K + c1] : 0u;
      alo[3] = r1 < M ? Al[r1 * K + c1] : 0u;
      // B rows: column kk of the A operand is input order m (as above); its G row is n + m (re) or n - m (im)
      const int mk0 = part ? (q ? 2 * c0 + 1 : 2 * c0 + 2) : 2 * c0 + q;
      const int mk1 = part ? (q ? 2 * c1 + 1 : 2 * c1 + 2) : 2 * c1 + q;
      const long long g0 = (mk0 <= n) ? (long long)(n + (part ? -mk0 : mk0)) * NC3 : -1;
      const long long g1 = (mk1 <= n) ? (long long)(n + (part ? -mk1 : mk1)) * NC3 : -1;
#pragma unroll
      for (int t = 0; t < kRotMaxNt; ++t) {
        if (t0 + t < NTN) {
          const int j = (t0 + t) * 8 + gq;
          unsigned bhi[2], blo[2];
          const bool ok0 = g0 >= 0 && j < NC3, ok1 = g1 >= 0 && j < NC3;
          bhi[0] = ok0 ? Gh[g0 + j] : 0u;
          blo[0] = ok0 ? Gl[g0 + j] : 0u;
          bhi[1] = ok1 ? Gh[g1 + j] : 0u;
          blo[1] = ok1 ? Gl[g1 + j] : 0u;
          mma_tf32(d[t], alo, bhi);
          mma_tf32(d[t], ahi, blo);
          mma_tf32(d[t], ahi, bhi);
        }
      }
    }
    // D: rows r0 / r1 (output order m' = row, or row + 1 for the imaginary part), columns (b, c);
    // E (q = 0) and O (q = 1) interleave in the buffer's last index
#pragma unroll
    for (int t = 0; t < kRotMaxNt; ++t) {
      if (t0 + t < NTN) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int row = e < 2 ? r0 : r1, col = (t0 + t) * 8 + 2 * tq + (e & 1);
          if (row < M && col < NC3) {
            const int pk = part ? n * (n + 1) - (row + 1) : n * (n + 1) + row;
            EO[eo_row(ld, a, pk, p) + 2 * col + q] = d[t][e];
          }
        }
      }
    }
  }
}

// One block per target quadruple (drop, latitude pair a, longitude b): the E / O sums of every rotated
// coefficient contracted with the four targets' projected factors (as k_self_proj: real parts with
// the real planes, imaginary parts with the imaginary planes, whose signs the factors carry).
__global__ void __launch_bounds__(kTcThreads) k_contract_eo(SelfGroup<float> A, const float* __restrict__ EO,
                                                            double* __restrict__ vals) {
  __shared__ float red[kTcWarps][12];
  const int p = A.p;
  const int ntri = (p + 1) * (p + 2) / 2;
  const int nc = (p + 1) * (p + 1);
  const int ng = (p + 1) * (2 * p + 2);
  const int hb = p + 1, nb = 2 * p + 2, na2 = (p + 2) / 2;
  const long long bid = blockIdx.x;
  const long long ld = bid / ((long long)na2 * hb);
  const int r = (int)(bid - ld * na2 * hb);
  const int a = r / hb, b = r - a * hb;
  const int a2 = p - a;
  const bool quad = a2 != a;
  const float* eo = EO + eo_row(ld, a, 0, p) + (long long)b * 6;  // row pk at + pk * hb * 6
  const long long qstride = 12 * (long long)ntri;
  const float* Qk_[4] = {A.Q + (ld * ng + a * nb + b) * qstride, A.Q + (ld * ng + a * nb + b + hb) * qstride,
                         A.Q + (ld * ng + a2 * nb + b) * qstride, A.Q + (ld * ng + a2 * nb + b + hb) * qstride};
  float acc[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.f;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const int n = degree_of(i);
    const int o = i - n * n;
    const bool re = o <= n;
    const int mo = re ? o : o - n;
    const int t = n * (n + 1) / 2 + mo;
    const int ri = re ? 0 : 1;
    const int pk = re ? n * (n + 1) + mo : n * (n + 1) - mo;
    const float* e6 = eo + (long long)pk * hb * 6;
    const float2 v01 = *reinterpret_cast<const float2*>(e6);
    const float2 v23 = *reinterpret_cast<const float2*>(e6 + 2);
    const float2 v45 = *reinterpret_cast<const float2*>(e6 + 4);
    const float vp[3] = {v01.x + v01.y, v23.x + v23.y, v45.x + v45.y};
    const float vm[3] = {v01.x - v01.y, v23.x - v23.y, v45.x - v45.y};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k >= 2 && !quad) break;
      const float* Qk = Qk_[k] + t;
      float q[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) q[e] = __ldg(Qk + (2 * e + ri) * (long long)ntri);
      sym_mul_add_f(q, (k == 0 || k == 3) ? vp : vm, acc[k]);
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      for (int off = 16; off > 0; off >>= 1) acc[k][c] += __shfl_down_sync(0xffffffffu, acc[k][c], off);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) red[warp][k * 3 + c] = acc[k][c];
  __syncthreads();
  const int nt = quad ? 4 : 2;
  if (threadIdx.x < 3 * nt) {
    float v = 0.f;
    for (int w = 0; w < kTcWarps; ++w) v += red[w][threadIdx.x];
    const int k = threadIdx.x / 3, c = threadIdx.x - 3 * k;
    const int tl = (k < 2 ? a * nb : a2 * nb) + b + (k & 1) * hb;
    vals[A.val_off[ld] + (long long)c * ng + tl] = A.wts[ld] * (double)v;
  }
}

}  // namespace

// E/O floats of one drop of degree p
static long long eo_per_drop(int p) { return (long long)((p + 2) / 2) * (p + 1) * (long long)(p + 1) * (p + 1) * 6; }

// Drops per launch of a group: as many as keep the chunk's E/O sums within `budget` floats (at least one).
static long long chunk_drops(int p, long long budget) { return std::max(1LL, budget / eo_per_drop(p)); }

long long self_tc_eo_floats(const std::vector<SelfGroup<float>>& groups, long long budget) {
  long long n = 0;
  for (const auto& g : groups) n = std::max(n, std::min(g.ndrop, chunk_drops(g.p, budget)) * eo_per_drop(g.p));
  return n;
}

long long self_tc_g_floats(const std::vector<SelfGroup<float>>& groups, long long budget) {
  long long n = 0;
  for (const auto& g : groups)  // hi and lo parts
    n = std::max(n, 2 * std::min(g.ndrop, chunk_drops(g.p, budget)) * (long long)(g.p + 1) * (g.p + 1) * (g.p + 1) * 3);
  return n;
}

// shared memory of one k_rot_tc block at degree p: A hi / lo for both parts and parities (each padded
// to 8 columns) and the hi / lo parts of the degree-p rows of G
static size_t rot_tc_smem(int p) {
  const size_t acols = (size_t)(((p + 2) / 2 + 7) & ~7) + (((p + 1) / 2 + 7) & ~7);
  return sizeof(float) * (2 * (size_t)(p + 1) * acols * 2 + 2 * (2 * (size_t)p + 1) * (p + 1) * 3);
}

bool self_tc_fits(int p) { return rot_tc_smem(p) <= 227 * 1024; }

int launch_self_tc(const std::vector<SelfGroup<float>>& groups, const double* dens, double* vals, float* eo,
                   unsigned* gm, long long budget, cudaStream_t s) {
  for (const auto& g : groups) {
    const int p = g.p;
    const int ng = (p + 1) * (2 * p + 2), ntri = (p + 1) * (p + 2) / 2;
    if (g.ndrop * (long long)ng > 0x7fffffffLL) return BIE_EINVAL;
    const size_t smem = rot_tc_smem(p);
    if (!self_tc_fits(p)) return BIE_EINVAL;
    if (smem > 48 * 1024)
      BIE_CUDA_TRY(cudaFuncSetAttribute(k_rot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long per = chunk_drops(p, budget);
    for (long long d0 = 0; d0 < g.ndrop; d0 += per) {
      // the chunk's drops d0 .. d0 + nd - 1 of the group, as a group of their own
      SelfGroup<float> c = g;
      c.begin = 0;
      c.ndrop = std::min(per, g.ndrop - d0);
      c.foff3 = g.foff3 + 3 * d0;
      c.Q = g.Q + d0 * ng * 12LL * ntri;
      c.wts = g.wts + d0;
      c.val_off = g.val_off + d0;
      const long long ng3 = c.ndrop * (long long)(p + 1) * (p + 1) * (p + 1) * 3;
      k_phase_g<<<(unsigned)((ng3 + 255) / 256), 256, 0, s>>>(c, dens, gm, gm + ng3);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
      const long long nblk = c.ndrop * ((p + 2) / 2) * (long long)(p + 1);
      k_rot_tc<<<(unsigned)nblk, kTcThreads, smem, s>>>(c, gm, gm + ng3, eo);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
      k_contract_eo<<<(unsigned)nblk, kTcThreads, 0, s>>>(c, eo, vals);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
    }
  }
  return BIE_OK;
}

}  // namespace bie
