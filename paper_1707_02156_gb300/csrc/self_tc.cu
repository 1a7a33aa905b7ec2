// Singular self interaction, projected form, FP32 (Thm 1, Sec. 2.2, App. B) with the Wigner
// rotation on the tensor cores.
//
// The rotation of App. B at latitude beta_a, for the density's degree-n coefficients phase-shifted
// to longitude phi_b, g_m = e^{i m phi_b} rho_n^m, is a product with the real blocks of d^n(beta_a):
//     Re rho'_{n m'} = sum_{m=0..n} C[m'][m] Re g_m,   Im rho'_{n m'} = sum_{m=1..n} S[m'-1][m-1] Im g_m.
// Splitting the input orders m by parity gives the even and odd partial sums E, O, from which the
// four targets (theta_a, phi_b), (theta_a, phi_b + pi), (pi - theta_a, phi_b), (pi - theta_a,
// phi_b + pi) follow exactly (the symmetries of the CUDA-core kernel k_self_proj).  With every
// longitude b < p+1 of the latitude and the three components as columns, each (latitude, degree,
// parity) is one matrix product
//     E or O (m', (b, c)) = W(m', m of that parity) G(m of that parity, (b, c)),
// W = C (rows m' = 0..n) or S (rows m' = 1..n).  k_self_tc runs these products as mma.sync m16n8k8 in
// TF32 with the 3-pass split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (x = x_hi + x_lo, both TF32),
// accumulated in FP32 (about FP32 accuracy), from the phase-shifted coefficients that k_phase_g forms
// once per apply for every longitude; the sums stay in shared memory, where the same block contracts
// them with the projected kernel factors Q of the latitude pair's 4 (p+1) targets at that degree
// (Q streamed from HBM).  The per-degree sums of every target are added in a fixed order by
// k_self_tc_reduce, so results do not depend on scheduling.
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

// The phase-shifted coefficients g = e^{i m phi_b} rho_n^m of every longitude b < p+1, shared by all
// latitudes: Gm[ld][packed (n, mm)][b][c] = Re g (mm >= 0) or Im g (mm < 0) of |mm|, in FP32.
__global__ void k_phase_g(SelfGroup<float> A, const double* __restrict__ dens, float* __restrict__ Gm) {
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
  Gm[idx] = mm >= 0 ? fr * co - fi * si : fr * si + fi * co;
}

// One block per (drop, latitude pair a, degree n).  The products are split by the parity of the input
// order, E = W[:, even m] G[even m, (b, c)] and O = W[:, odd m] G[odd m, (b, c)], so that no operand
// carries zero padding: K = the orders of one parity, N = (b, c) = 3 (p+1) columns.  The block stages
// W's columns of each parity already split into TF32 hi / lo parts, and the degree's rows of the
// phase-shifted coefficients G.  A warp owns one (part, parity, 16-row tile, half of N) and runs its
// k-steps once, building the A fragment once per k-step and reusing it over up to 13 column tiles.
// The E / O sums go to shared memory; then each warp takes longitudes b and contracts the degree's
// 2n+1 rotated coefficients with the factors of b's four targets (lanes over the coefficients,
// a shuffle reduction), writing part[target][n][c].
constexpr int kRotMaxNt = 13;  // 8-column tiles per warp pass (N = 3 (p+1) takes one or two passes for p < 64)

__global__ void __launch_bounds__(kTcThreads) k_self_tc(SelfGroup<float> A, const float* __restrict__ Gm,
                                                        float* __restrict__ part) {
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
  float* Gs = reinterpret_cast<float*>(Alo + acur);  // [n + mm][b][c], mm = -n..n
  float* EOs = Gs + (2 * n + 1) * NC3;               // [n + mm'][b][c][parity]: E, O of the output orders
  const long long boff = (long long)n * (n + 1) * (2 * n + 1) / 6 + (long long)(n - 1) * n * (2 * n - 1) / 6;
  const float* blk = A.wblk + (long long)a * A.wstride + boff;
  // the degree's rows of G go to shared memory by asynchronous 4-byte copies, all in flight at once
  const float* gsrc = Gm + ((ld * (p + 1) * (p + 1)) + (long long)n * n) * NC3;
  for (int i = threadIdx.x; i < (2 * n + 1) * NC3; i += blockDim.x) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(Gs + i);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(gsrc + i) : "memory");
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
      const float* g0 = (mk0 <= n) ? Gs + (long long)(n + (part ? -mk0 : mk0)) * NC3 : nullptr;
      const float* g1 = (mk1 <= n) ? Gs + (long long)(n + (part ? -mk1 : mk1)) * NC3 : nullptr;
#pragma unroll
      for (int t = 0; t < kRotMaxNt; ++t) {
        if (t0 + t < NTN) {
          const int j = (t0 + t) * 8 + gq;
          const float b0v = (g0 && j < NC3) ? g0[j] : 0.f;
          const float b1v = (g1 && j < NC3) ? g1[j] : 0.f;
          unsigned bhi[2], blo[2];
          tf32_split(b0v, bhi[0], blo[0]);
          tf32_split(b1v, bhi[1], blo[1]);
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
            const int pl = part ? n - (row + 1) : n + row;  // local row n + m' (real) or n - m' (imaginary)
            EOs[pl * 2 * NC3 + 2 * col + q] = d[t][e];
          }
        }
      }
    }
  }
  __syncthreads();
  // contraction with the factors of the four targets of each longitude, at degree n
  const int ntri = (p + 1) * (p + 2) / 2, ng = (p + 1) * (2 * p + 2), nb = 2 * p + 2;
  const int a2 = p - a;
  const bool quad = a2 != a;
  const long long qstride = 12 * (long long)ntri;
  for (int b = warp; b < hb; b += kTcWarps) {
    const long long tl[4] = {(long long)a * nb + b, (long long)a * nb + b + hb, (long long)a2 * nb + b,
                             (long long)a2 * nb + b + hb};
    float acc[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.f;
    for (int o = lane; o < 2 * n + 1; o += 32) {
      const bool re = o <= n;
      const int mo = re ? o : o - n;
      const int t = n * (n + 1) / 2 + mo;
      const int ri = re ? 0 : 1;
      const float* v = EOs + (re ? n + mo : n - mo) * 2 * NC3 + b * 6;
      const float vp[3] = {v[0] + v[1], v[2] + v[3], v[4] + v[5]};
      const float vm[3] = {v[0] - v[1], v[2] - v[3], v[4] - v[5]};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= 2 && !quad) break;
        const float* Qk = A.Q + (ld * ng + tl[k]) * qstride + t;
        float qv[6];
#pragma unroll
        for (int e = 0; e < 6; ++e) qv[e] = __ldg(Qk + (2 * e + ri) * (long long)ntri);
        sym_mul_add_f(qv, (k == 0 || k == 3) ? vp : vm, acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        for (int off = 16; off > 0; off >>= 1) acc[k][c] += __shfl_down_sync(0xffffffffu, acc[k][c], off);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= 2 && !quad) break;
        float* pt = part + ((ld * ng + tl[k]) * (p + 1) + n) * 3;
        pt[0] = acc[k][0];
        pt[1] = acc[k][1];
        pt[2] = acc[k][2];
      }
  }
}

// vals = weight * (the per-degree sums of every target, added in degree order, in FP64)
__global__ void k_self_tc_reduce(SelfGroup<float> A, const float* __restrict__ part, double* __restrict__ vals) {
  const int p = A.p;
  const int ng = (p + 1) * (2 * p + 2);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= A.ndrop * (long long)ng) return;
  const long long ld = idx / ng;
  const int tl = (int)(idx - ld * ng);
  const float* pt = part + idx * (p + 1) * 3;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int n = 0; n <= p; ++n) {
    s0 += (double)pt[3 * n];
    s1 += (double)pt[3 * n + 1];
    s2 += (double)pt[3 * n + 2];
  }
  const double w = A.wts[ld];
  double* v = vals + A.val_off[ld] + tl;
  v[0] = w * s0;
  v[ng] = w * s1;
  v[2 * (long long)ng] = w * s2;
}

}  // namespace

// Per-degree partial sums of one drop of degree p (floats)
static long long part_per_drop(int p) { return (long long)(p + 1) * (2 * p + 2) * (p + 1) * 3; }

// Drops per launch of a group: as many as keep the chunk's partial sums within `budget` floats.
static long long chunk_drops(int p, long long budget) { return std::max(1LL, budget / part_per_drop(p)); }

long long self_tc_part_floats(const std::vector<SelfGroup<float>>& groups, long long budget) {
  long long n = 0;
  for (const auto& g : groups) n = std::max(n, std::min(g.ndrop, chunk_drops(g.p, budget)) * part_per_drop(g.p));
  return n;
}

long long self_tc_g_floats(const std::vector<SelfGroup<float>>& groups, long long budget) {
  long long n = 0;
  for (const auto& g : groups)
    n = std::max(n, std::min(g.ndrop, chunk_drops(g.p, budget)) * (long long)(g.p + 1) * (g.p + 1) * (g.p + 1) * 3);
  return n;
}

size_t self_tc_smem(int p) {
  // A hi / lo for both parts and parities (each padded to 8 columns), the degree-p rows of G, and
  // the E / O sums of degree p
  const size_t acols = (size_t)(((p + 2) / 2 + 7) & ~7) + (((p + 1) / 2 + 7) & ~7);
  return sizeof(float) * (2 * (size_t)(p + 1) * acols * 2 + (2 * (size_t)p + 1) * (p + 1) * 3 * 3);
}

int launch_self_tc(const std::vector<SelfGroup<float>>& groups, const double* dens, double* vals, float* part,
                   float* gm, long long budget, cudaStream_t s) {
  for (const auto& g : groups) {
    const int p = g.p;
    const int ng = (p + 1) * (2 * p + 2), ntri = (p + 1) * (p + 2) / 2;
    if (g.ndrop * (long long)ng > 0x7fffffffLL) return BIE_EINVAL;
    const size_t smem = self_tc_smem(p);
    if (smem > 227 * 1024) return BIE_EINVAL;
    if (smem > 48 * 1024)
      BIE_CUDA_TRY(cudaFuncSetAttribute(k_self_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
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
      k_phase_g<<<(unsigned)((ng3 + 255) / 256), 256, 0, s>>>(c, dens, gm);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
      const long long nblk = c.ndrop * ((p + 2) / 2) * (long long)(p + 1);
      k_self_tc<<<(unsigned)nblk, kTcThreads, smem, s>>>(c, gm, part);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
      const long long nt = c.ndrop * (long long)ng;
      k_self_tc_reduce<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(c, part, vals);
      count_launch();
      BIE_CUDA_TRY(cudaGetLastError());
    }
  }
  return BIE_OK;
}

}  // namespace bie
