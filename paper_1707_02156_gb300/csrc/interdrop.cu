// Inter-drop interactions (Sec. 2.1, 2.3): region classification with bounding spheres, and the
// regular (standard grid, Omega_0) and upsampled (grid of degree U(p+1)-1, Omega_1) pair sums of the
// single- and double-layer kernels, as a balanced work list of (target tile, source drop, grid,
// source range, target mask) items.
#include <cuda_runtime.h>

#include <type_traits>

#include "device.cuh"
#include "interdrop.h"
#include "internal.cuh"

namespace bie {
namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(long long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// region[t * ndrop + j]: 0 / 1 / 2 for Omega_0/1/2 of target t w.r.t. drop j, 3 = t inside drop j,
// 255 for j = own drop.  Distance = nearest point of j's upsampled grid (Sec. 2.3).
__global__ void k_classify(const double* __restrict__ rec_std, long long ntarget, const int* __restrict__ tdrop,
                           const long long* __restrict__ tloc, const long long* __restrict__ toff_std,
                           const int* __restrict__ ngd, int ndrop, const double* __restrict__ centre,
                           const double* __restrict__ bound, const double* __restrict__ h, double a_tilde,
                           const double* __restrict__ rec_up, const long long* __restrict__ up_off,
                           const long long* __restrict__ up_n, unsigned char* __restrict__ region) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ntarget * ndrop) return;
  const long long t = idx / ndrop;
  const int j = (int)(idx - t * ndrop);
  const int i = tdrop[t];
  if (i == j) {
    region[idx] = 255;
    return;
  }
  const long long ng = ngd[i];
  const double* ri = rec_std + 7 * toff_std[i];
  const double x0 = ri[tloc[t]], x1 = ri[ng + tloc[t]], x2 = ri[2 * ng + tloc[t]];
  const double dc0 = x0 - centre[3 * j], dc1 = x1 - centre[3 * j + 1], dc2 = x2 - centre[3 * j + 2];
  const double dcen = sqrt(dc0 * dc0 + dc1 * dc1 + dc2 * dc2);
  if (dcen - bound[j] > a_tilde * h[j]) {  // every grid point of j is farther than A h_j
    region[idx] = 0;
    return;
  }
  const long long N = up_n[j];
  const double* r = rec_up + 7 * up_off[j];
  double best = 1e300;
  long long bi = 0;
  for (long long s = 0; s < N; ++s) {
    const double d0 = x0 - r[s], d1 = x1 - r[N + s], d2 = x2 - r[2 * N + s];
    const double d = d0 * d0 + d1 * d1 + d2 * d2;
    if (d < best) {
      best = d;
      bi = s;
    }
  }
  const double dist = sqrt(best);
  const double side = (x0 - r[bi]) * r[3 * N + bi] + (x1 - r[N + bi]) * r[4 * N + bi] + (x2 - r[2 * N + bi]) * r[5 * N + bi];
  unsigned char code = dist <= h[j] ? 2 : (dist <= a_tilde * h[j] ? 1 : 0);
  if (side <= 0.0) code = 3;
  region[idx] = code;
}

constexpr int kChunk = 128;  // sources staged per pass

// Staged source record: (x, y, z, q0), (q1, q2, n0, n1), (n2, -, -, -) so that the inner loop reads
// it with 128-bit shared-memory loads (two for the single layer, three for the double layer).
template <typename R>
struct alignas(16) SrcRec {
  R v[12];
};

// One block per work-list block: the tile's 128 targets, TPT per thread (targets tid + u * 128/TPT),
// against the sources of its items, staged through shared memory.  The stresslet's factor -6 is
// applied with the item's weight.
template <typename R, int KIND, int TPT>
__global__ void __launch_bounds__(kTile / TPT) k_interdrop(
    const PairItem* __restrict__ items, const int* __restrict__ blk_item, const long long* __restrict__ tile_t0,
    const int* __restrict__ tile_n, const int* __restrict__ tile_drop, const long long* __restrict__ tgt_loc,
    const long long* __restrict__ toff_std, const int* __restrict__ ngd, const double* __restrict__ rec_std,
    const double* __restrict__ centre, const R* __restrict__ Xs, const R* __restrict__ Ns, const R* __restrict__ Qs,
    long long nstd, const R* __restrict__ Xu, const R* __restrict__ Nu, const R* __restrict__ Qu, long long nup,
    const double* __restrict__ wts, double* __restrict__ partial) {
  constexpr int NT = kTile / TPT;  // threads per block
  constexpr int NR = KIND ? 9 : 6;  // values used per source
  __shared__ SrcRec<R> src[kChunk];
  const int b = blockIdx.x;
  const int it0 = blk_item[b], it1 = blk_item[b + 1];
  const int tile = items[it0].tile;
  const int tid = threadIdx.x;
  const int nt = tile_n[tile];
  const int di = tile_drop[tile];
  double tx[TPT], ty[TPT], tz[TPT], acc[TPT][3];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int k = tid + u * NT;
    tx[u] = ty[u] = tz[u] = 0;
    acc[u][0] = acc[u][1] = acc[u][2] = 0;
    if (k < nt) {
      const long long t = tile_t0[tile] + k;
      const long long ng = ngd[di];
      const double* ri = rec_std + 7 * toff_std[di];
      const long long l = tgt_loc[t];
      tx[u] = ri[l];
      ty[u] = ri[ng + l];
      tz[u] = ri[2 * ng + l];
    }
  }
  for (int it = it0; it < it1; ++it) {
    const PairItem item = items[it];
    const int j = item.src_drop;
    bool act[TPT], any = false;
    R px[TPT], py[TPT], pz[TPT];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int k = tid + u * NT;
      act[u] = k < nt && ((item.mask[k >> 5] >> (k & 31)) & 1u);
      any = any || act[u];
      px[u] = (R)(tx[u] - centre[3 * j]);
      py[u] = (R)(ty[u] - centre[3 * j + 1]);
      pz[u] = (R)(tz[u] - centre[3 * j + 2]);
    }
    const R* X = item.grid ? Xu : Xs;
    const R* N = item.grid ? Nu : Ns;
    const R* Q = item.grid ? Qu : Qs;
    const long long ld = item.grid ? nup : nstd;
    R s[TPT][3];
#pragma unroll
    for (int u = 0; u < TPT; ++u) s[u][0] = s[u][1] = s[u][2] = 0;
    for (long long c0 = item.s0; c0 < item.s1; c0 += kChunk) {
      const int cn = (int)min((long long)kChunk, item.s1 - c0);
      for (int k = tid; k < cn; k += NT) {
        const long long sidx = c0 + k;
        SrcRec<R> r;
        r.v[0] = X[sidx];
        r.v[1] = X[ld + sidx];
        r.v[2] = X[2 * ld + sidx];
        r.v[3] = Q[sidx];
        r.v[4] = Q[ld + sidx];
        r.v[5] = Q[2 * ld + sidx];
        if (KIND) {
          r.v[6] = N[sidx];
          r.v[7] = N[ld + sidx];
          r.v[8] = N[2 * ld + sidx];
        } else {
          r.v[6] = r.v[7] = r.v[8] = 0;
        }
        r.v[9] = r.v[10] = r.v[11] = 0;
        src[k] = r;
      }
      __syncthreads();
      if (any) {
        for (int k = 0; k < cn; ++k) {
          R v[12];
          // 128-bit shared-memory loads of the record (the double-layer record needs all three)
          typedef typename std::conditional<sizeof(R) == 4, float4, double2>::type V;
          constexpr int per = 16 / sizeof(R);
          constexpr int nv = (NR + per - 1) / per;
#pragma unroll
          for (int q = 0; q < nv; ++q) *reinterpret_cast<V*>(v + q * per) = reinterpret_cast<const V*>(&src[k])[q];
          const R xs_ = v[0], ys_ = v[1], zs_ = v[2], q0 = v[3], q1 = v[4], q2 = v[5];
#pragma unroll
          for (int u = 0; u < TPT; ++u) {
            const R dx = px[u] - xs_, dy = py[u] - ys_, dz = pz[u] - zs_;
            const R ri = rsqrt_<R>(dx * dx + dy * dy + dz * dz);
            const R xq = dx * q0 + dy * q1 + dz * q2;
            if (KIND == 0) {  // Stokeslet
              const R c = xq * ri * ri * ri;
              s[u][0] += q0 * ri + c * dx;
              s[u][1] += q1 * ri + c * dy;
              s[u][2] += q2 * ri + c * dz;
            } else {  // stresslet, without its factor -6
              const R xn = dx * v[6] + dy * v[7] + dz * v[8];
              const R ri2 = ri * ri;
              const R c = xq * xn * ri2 * ri2 * ri;
              s[u][0] += c * dx;
              s[u][1] += c * dy;
              s[u][2] += c * dz;
            }
          }
        }
      }
      __syncthreads();
    }
    const double wj = KIND ? -6.0 * wts[j] : wts[j];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const double w = act[u] ? wj : 0.0;
      acc[u][0] += w * (double)s[u][0];
      acc[u][1] += w * (double)s[u][1];
      acc[u][2] += w * (double)s[u][2];
    }
  }
  double* pp = partial + (long long)b * 3 * kTile;
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int k = tid + u * NT;
    pp[k] = acc[u][0];
    pp[kTile + k] = acc[u][1];
    pp[2 * kTile + k] = acc[u][2];
  }
}

// ---- FP32 pair sums on packed lane pairs ----
// Two targets share one 64-bit register pair and every FP32 operation of their two pairs issues as
// one fma/mul/sub.rn.f32x2 instruction: half the issue slots of the scalar kernel for the same
// FP32-pipe work, which leaves room for the shared-memory loads and the two MUFU rsqrt of each
// source without starving the FMA pipe.  Rounding is that of the scalar operations (each lane is
// an IEEE round-to-nearest FP32 operation).
typedef unsigned long long fx2;  // lanes (lo, hi) = two FP32 values

__device__ __forceinline__ fx2 x2_pack(float lo, float hi) {
  fx2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void x2_unpack(fx2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ fx2 x2_sub(fx2 a, fx2 b) {
  fx2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ fx2 x2_mul(fx2 a, fx2 b) {
  fx2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ fx2 x2_fma(fx2 a, fx2 b, fx2 c) {
  fx2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ fx2 x2_rsqrt(fx2 v) {
  float lo, hi;
  x2_unpack(v, lo, hi);
  return x2_pack(rsqrtf(lo), rsqrtf(hi));
}

constexpr int kChunkX2 = 64;  // sources staged per pass of the packed kernel

// Staged source of the packed kernel: each value duplicated into both lanes, in the order
// x, y, z, q0, q1, q2, n0, n1, n2 (and one pad), read with 128-bit shared-memory loads (three for
// the single layer, five for the double layer).
struct alignas(16) SrcRecX2 {
  fx2 v[10];
};

// Same work list, layout and result as k_interdrop<float, KIND, TPT>; TPT even, the thread's
// targets tid + u * (128/TPT) taken two by two (u = 2w, 2w + 1 share lane pair w).  The tile's target
// coordinates (FP32, relative to their drop's centre) and the FP64 accumulators live in shared
// memory, not in registers, so that more warps fit per SM; the source loop takes two sources per iteration (2 x TPT/2 independent
// chains per thread).  PF = 1 software-pipelines the staging: the next chunk's sources are loaded
// into registers while the current chunk is summed, so the global-memory latency of the staging
// overlaps the arithmetic.
template <int KIND, int TPT, int PF, int CH = kChunkX2>
__global__ void __launch_bounds__(kTile / TPT) k_interdrop_x2(
    const PairItem* __restrict__ items, const int* __restrict__ blk_item, const long long* __restrict__ tile_t0,
    const int* __restrict__ tile_n, const int* __restrict__ tile_drop, const long long* __restrict__ tgt_loc,
    const long long* __restrict__ toff_std, const int* __restrict__ ngd, const double* __restrict__ rec_std,
    const double* __restrict__ centre, const float* __restrict__ Xs, const float* __restrict__ Ns,
    const float* __restrict__ Qs, long long nstd, const float* __restrict__ Xu, const float* __restrict__ Nu,
    const float* __restrict__ Qu, long long nup, const double* __restrict__ wts, double* __restrict__ partial) {
  static_assert(TPT % 2 == 0, "targets are taken in lane pairs");
  constexpr int NT = kTile / TPT;
  constexpr int NW = TPT / 2;  // lane pairs per thread
  constexpr int NV = KIND ? 9 : 6;
  constexpr int nv = (NV + 1) / 2;  // 128-bit loads per staged source
  static_assert(CH % NT == 0 && CH >= NT, "a chunk is a whole number of sources per thread");
  constexpr int RPT = CH / NT;  // staged sources per thread and chunk
  __shared__ SrcRecX2 src[CH];
  __shared__ float tgt[3][kTile];   // the tile's targets relative to their own drop's centre (FP32)
  __shared__ double acc[3][kTile];  // per-target sums over the block's items
  const int b = blockIdx.x;
  const int it0 = blk_item[b], it1 = blk_item[b + 1];
  const int tile = items[it0].tile;
  const int tid = threadIdx.x;
  const int nt = tile_n[tile];
  const int di = tile_drop[tile];
  const double ox = centre[3 * di], oy = centre[3 * di + 1], oz = centre[3 * di + 2];
  {
    const long long ng = ngd[di];
    const double* ri = rec_std + 7 * toff_std[di];
    for (int k = tid; k < kTile; k += NT) {
      double x = ox, y = oy, z = oz;
      if (k < nt) {
        const long long l = tgt_loc[tile_t0[tile] + k];
        x = ri[l];
        y = ri[ng + l];
        z = ri[2 * ng + l];
      }
      // |x - o| is about a drop radius, so its FP32 rounding (2^-24 of it) is far below that of the
      // target's position relative to a source drop's centre, which the pair sums round to FP32 anyway
      tgt[0][k] = (float)(x - ox);
      tgt[1][k] = (float)(y - oy);
      tgt[2][k] = (float)(z - oz);
      acc[0][k] = acc[1][k] = acc[2][k] = 0.0;
    }
  }
  // the block's shared arrays are written before any thread reads them (the first staging barrier
  // below comes after the target loads; each thread reads only its own targets' entries)
  __syncthreads();
  // sources c0 + tid + r NT of a chunk, r < RPT (zero past the item's end: zero weight)
  auto load_chunk = [&](float (&v)[RPT][NV], const float* X, const float* N, const float* Q, long long ld,
                        long long c0, long long s1) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const long long sidx = c0 + tid + r * NT;
#pragma unroll
      for (int q = 0; q < NV; ++q) v[r][q] = 0.f;
      if (sidx < s1) {
        v[r][0] = X[sidx];
        v[r][1] = X[ld + sidx];
        v[r][2] = X[2 * ld + sidx];
        v[r][3] = Q[sidx];
        v[r][4] = Q[ld + sidx];
        v[r][5] = Q[2 * ld + sidx];
        if (KIND) {
          v[r][6] = N[sidx];
          v[r][7] = N[ld + sidx];
          v[r][8] = N[2 * ld + sidx];
        }
      }
    }
  };
  auto store_chunk = [&](const float (&v)[RPT][NV]) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      SrcRecX2 rec;
#pragma unroll
      for (int q = 0; q < NV; ++q) rec.v[q] = x2_pack(v[r][q], v[r][q]);
#pragma unroll
      for (int q = NV; q < 10; ++q) rec.v[q] = 0ull;
      src[tid + r * NT] = rec;
    }
  };
  for (int it = it0; it < it1; ++it) {
    const int j = items[it].src_drop;
    unsigned act = 0u;  // bit u: target tid + u * NT is in this item
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int k = tid + u * NT;
      if (k < nt && ((items[it].mask[k >> 5] >> (k & 31)) & 1u)) act |= 1u << u;
    }
    // target relative to the source drop's centre: (x - o) + (o - c_j), the offset in FP64
    const double cx = ox - centre[3 * j], cy = oy - centre[3 * j + 1], cz = oz - centre[3 * j + 2];
    fx2 px[NW], py[NW], pz[NW], s[NW][3];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const int k0 = tid + 2 * w * NT, k1 = k0 + NT;
      px[w] = x2_pack((float)((double)tgt[0][k0] + cx), (float)((double)tgt[0][k1] + cx));
      py[w] = x2_pack((float)((double)tgt[1][k0] + cy), (float)((double)tgt[1][k1] + cy));
      pz[w] = x2_pack((float)((double)tgt[2][k0] + cz), (float)((double)tgt[2][k1] + cz));
      s[w][0] = s[w][1] = s[w][2] = 0ull;  // +0.0f in both lanes
    }
    const int grid = items[it].grid;
    const float* X = grid ? Xu : Xs;
    const float* N = grid ? Nu : Ns;
    const float* Q = grid ? Qu : Qs;
    const long long ld = grid ? nup : nstd;
    const long long s0 = items[it].s0, s1 = items[it].s1;
    float pre[RPT][NV];
    if (PF) load_chunk(pre, X, N, Q, ld, s0, s1);
    for (long long c0 = s0; c0 < s1; c0 += CH) {
      const int cn = (int)min((long long)CH, s1 - c0);
      if (!PF) load_chunk(pre, X, N, Q, ld, c0, s1);
      store_chunk(pre);
      __syncthreads();
      if (PF && c0 + CH < s1) load_chunk(pre, X, N, Q, ld, c0 + CH, s1);  // next chunk, in flight
      if (act) {
        const int cn2 = (cn + 1) & ~1;
        for (int k = 0; k < cn2; k += 2) {
          fx2 va[10], vb[10];
#pragma unroll
          for (int q = 0; q < nv; ++q) {
            *reinterpret_cast<ulonglong2*>(va + 2 * q) = reinterpret_cast<const ulonglong2*>(&src[k])[q];
            *reinterpret_cast<ulonglong2*>(vb + 2 * q) = reinterpret_cast<const ulonglong2*>(&src[k + 1])[q];
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const fx2* v = h ? vb : va;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
              const fx2 dx = x2_sub(px[w], v[0]), dy = x2_sub(py[w], v[1]), dz = x2_sub(pz[w], v[2]);
              const fx2 r2 = x2_fma(dz, dz, x2_fma(dy, dy, x2_mul(dx, dx)));
              const fx2 ri = x2_rsqrt(r2);
              const fx2 xq = x2_fma(dz, v[5], x2_fma(dy, v[4], x2_mul(dx, v[3])));
              const fx2 ri2 = x2_mul(ri, ri);
              if (KIND == 0) {  // Stokeslet: q/r + (xh.q) xh/r^3
                const fx2 c = x2_mul(x2_mul(xq, ri2), ri);
                s[w][0] = x2_fma(c, dx, x2_fma(v[3], ri, s[w][0]));
                s[w][1] = x2_fma(c, dy, x2_fma(v[4], ri, s[w][1]));
                s[w][2] = x2_fma(c, dz, x2_fma(v[5], ri, s[w][2]));
              } else {  // stresslet without its factor -6: (xh.q)(xh.n) xh/r^5
                const fx2 xn = x2_fma(dz, v[8], x2_fma(dy, v[7], x2_mul(dx, v[6])));
                const fx2 c = x2_mul(x2_mul(x2_mul(x2_mul(xq, xn), ri2), ri2), ri);
                s[w][0] = x2_fma(c, dx, s[w][0]);
                s[w][1] = x2_fma(c, dy, s[w][1]);
                s[w][2] = x2_fma(c, dz, s[w][2]);
              }
            }
          }
        }
      }
      __syncthreads();
    }
    const double wj = KIND ? -6.0 * wts[j] : wts[j];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const int k0 = tid + 2 * w * NT, k1 = k0 + NT;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float lo, hi;
        x2_unpack(s[w][c], lo, hi);
        if (act & (1u << (2 * w))) acc[c][k0] += wj * (double)lo;
        if (act & (1u << (2 * w + 1))) acc[c][k1] += wj * (double)hi;
      }
    }
  }
  double* pp = partial + (long long)b * 3 * kTile;
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int k = tid + u * NT;
    pp[k] = acc[0][k];
    pp[kTile + k] = acc[1][k];
    pp[2 * kTile + k] = acc[2][k];
  }
}

// ---- double-float pair sums ----
// A double-float value is an unevaluated sum hi + lo of two FP32 numbers (about 44 significant
// bits).  Sums use Knuth's TwoSum and products the FMA-based TwoProduct (both error-free
// transformations).  Results are left unnormalised (|lo| may exceed ulp(hi)/2 by a few units, which
// costs no accuracy in the short chains of one pair); the per-target accumulators are renormalised
// by Dekker's Fast2Sum after every staged chunk of sources.  1/sqrt starts from the FP32 estimate and
// takes one Newton step in double-float.  Every operation runs on the FP32 pipes.
struct df2 {
  float h, l;
};

__device__ inline df2 df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ inline df2 fast2sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ inline df2 df_add(df2 a, df2 b) {
  const float s = a.h + b.h;
  const float v = s - a.h;
  return {s, (a.h - (s - v)) + (b.h - v) + a.l + b.l};
}
__device__ inline df2 df_renorm(df2 a) {  // TwoSum of the two parts
  const float s = a.h + a.l;
  const float v = s - a.h;
  return {s, (a.h - (s - v)) + (a.l - v)};
}
__device__ inline df2 df_neg(df2 a) { return {-a.h, -a.l}; }
__device__ inline df2 df_mul(df2 a, df2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return {p, e};
}
__device__ inline df2 df_sqr(df2 a) {
  const float p = a.h * a.h;
  float e = fmaf(a.h, a.h, -p);
  e = fmaf(2.0f * a.h, a.l, e);
  return {p, e};
}
__device__ inline df2 df_rsqrt(df2 a) {
  const float y = rsqrtf(a.h);
  const float y2 = y * y;
  const df2 ay2 = df_mul(a, {y2, fmaf(y, y, -y2)});
  const float e = (1.0f - ay2.h) - ay2.l;  // 1 - a y^2, of the order of the estimate's error
  return fast2sum(y, 0.5f * y * e);
}

// Same work list and layout as k_interdrop; sources are read in FP64 and split into double-float
// pairs as they are staged through shared memory, targets are split once per item.
template <int KIND, int TPT>
__global__ void __launch_bounds__(kTile / TPT) k_interdrop_df(
    const PairItem* __restrict__ items, const int* __restrict__ blk_item, const long long* __restrict__ tile_t0,
    const int* __restrict__ tile_n, const int* __restrict__ tile_drop, const long long* __restrict__ tgt_loc,
    const long long* __restrict__ toff_std, const int* __restrict__ ngd, const double* __restrict__ rec_std,
    const double* __restrict__ centre, const double* __restrict__ Xs, const double* __restrict__ Ns,
    const double* __restrict__ Qs, long long nstd, const double* __restrict__ Xu, const double* __restrict__ Nu,
    const double* __restrict__ Qu, long long nup, const double* __restrict__ wts, double* __restrict__ partial) {
  constexpr int NT = kTile / TPT;
  constexpr int NV = KIND ? 9 : 6;  // staged values per source: x, q (and n)
  __shared__ df2 sv[NV][kChunk];
  const int b = blockIdx.x;
  const int it0 = blk_item[b], it1 = blk_item[b + 1];
  const int tile = items[it0].tile;
  const int tid = threadIdx.x;
  const int nt = tile_n[tile];
  const int di = tile_drop[tile];
  double tx[TPT], ty[TPT], tz[TPT], acc[TPT][3];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int k = tid + u * NT;
    tx[u] = ty[u] = tz[u] = 0;
    acc[u][0] = acc[u][1] = acc[u][2] = 0;
    if (k < nt) {
      const long long t = tile_t0[tile] + k;
      const long long ng = ngd[di];
      const double* ri = rec_std + 7 * toff_std[di];
      const long long l = tgt_loc[t];
      tx[u] = ri[l];
      ty[u] = ri[ng + l];
      tz[u] = ri[2 * ng + l];
    }
  }
  for (int it = it0; it < it1; ++it) {
    const PairItem item = items[it];
    const int j = item.src_drop;
    bool act[TPT], any = false;
    df2 px[TPT], py[TPT], pz[TPT];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int k = tid + u * NT;
      act[u] = k < nt && ((item.mask[k >> 5] >> (k & 31)) & 1u);
      any = any || act[u];
      px[u] = df_from(tx[u] - centre[3 * j]);
      py[u] = df_from(ty[u] - centre[3 * j + 1]);
      pz[u] = df_from(tz[u] - centre[3 * j + 2]);
    }
    const double* X = item.grid ? Xu : Xs;
    const double* N = item.grid ? Nu : Ns;
    const double* Q = item.grid ? Qu : Qs;
    const long long ld = item.grid ? nup : nstd;
    df2 s[TPT][3];
#pragma unroll
    for (int u = 0; u < TPT; ++u) s[u][0] = s[u][1] = s[u][2] = {0.0f, 0.0f};
    for (long long c0 = item.s0; c0 < item.s1; c0 += kChunk) {
      const int cn = (int)min((long long)kChunk, item.s1 - c0);
      for (int k = tid; k < cn; k += NT) {
        const long long sidx = c0 + k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sv[c][k] = df_from(X[c * ld + sidx]);
          sv[3 + c][k] = df_from(Q[c * ld + sidx]);
          if (KIND) sv[6 + c][k] = df_from(N[c * ld + sidx]);
        }
      }
      __syncthreads();
      if (any) {
        for (int k = 0; k < cn; ++k) {
          const df2 xs_ = sv[0][k], ys_ = sv[1][k], zs_ = sv[2][k];
          const df2 q0 = sv[3][k], q1 = sv[4][k], q2 = sv[5][k];
#pragma unroll
          for (int u = 0; u < TPT; ++u) {
            const df2 dx = df_add(px[u], df_neg(xs_)), dy = df_add(py[u], df_neg(ys_)),
                      dz = df_add(pz[u], df_neg(zs_));
            const df2 r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
            const df2 ri = df_rsqrt(r2);
            const df2 xq = df_add(df_add(df_mul(dx, q0), df_mul(dy, q1)), df_mul(dz, q2));
            if (KIND == 0) {  // Stokeslet
              const df2 ri3 = df_mul(df_sqr(ri), ri);
              const df2 c = df_mul(xq, ri3);
              s[u][0] = df_add(s[u][0], df_add(df_mul(q0, ri), df_mul(c, dx)));
              s[u][1] = df_add(s[u][1], df_add(df_mul(q1, ri), df_mul(c, dy)));
              s[u][2] = df_add(s[u][2], df_add(df_mul(q2, ri), df_mul(c, dz)));
            } else {  // stresslet
              const df2 n0 = sv[6][k], n1 = sv[7][k], n2 = sv[8][k];
              const df2 xn = df_add(df_add(df_mul(dx, n0), df_mul(dy, n1)), df_mul(dz, n2));
              const df2 ri2 = df_sqr(ri);
              const df2 ri5 = df_mul(df_sqr(ri2), ri);
              const df2 c = df_mul(df_mul(xq, xn), ri5);  // the factor -6 goes with the weight
              s[u][0] = df_add(s[u][0], df_mul(c, dx));
              s[u][1] = df_add(s[u][1], df_mul(c, dy));
              s[u][2] = df_add(s[u][2], df_mul(c, dz));
            }
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < TPT; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) s[u][c] = df_renorm(s[u][c]);
    }
    const double wj = KIND ? -6.0 * wts[j] : wts[j];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const double w = act[u] ? wj : 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[u][c] += w * ((double)s[u][c].h + (double)s[u][c].l);
    }
  }
  double* pp = partial + (long long)b * 3 * kTile;
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int k = tid + u * NT;
    pp[k] = acc[u][0];
    pp[kTile + k] = acc[u][1];
    pp[2 * kTile + k] = acc[u][2];
  }
}

// Per (tile, source drop j): the tile's targets in Omega_0, Omega_1 and Omega_2 of drop j as 128-bit
// masks, and whether any target lies inside drop j.  Consecutive threads take consecutive j, so the
// region reads of one target are coalesced.
__global__ void k_tile_masks(const unsigned char* __restrict__ region, int nd, const long long* __restrict__ tile_t0,
                             const int* __restrict__ tile_n, long long ntile, TileMask* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ntile * nd) return;
  const long long ti = idx / nd;
  const int j = (int)(idx - ti * nd);
  TileMask m{};
  const long long t0 = tile_t0[ti];
  const int n = tile_n[ti];
  for (int k = 0; k < n; ++k) {
    const unsigned char r = region[(t0 + k) * nd + j];
    if (r < 3) m.m[r][k >> 5] |= 1u << (k & 31);
    else if (r == 3) m.inside = 1;
  }
  out[idx] = m;
}

// vals += sum of the partials of the tile's blocks, in block order
__global__ void k_reduce_tiles(const double* __restrict__ partial, const int* __restrict__ tile_blk,
                               const long long* __restrict__ tile_t0, const int* __restrict__ tile_n,
                               const int* __restrict__ tile_drop, const long long* __restrict__ tgt_loc,
                               const long long* __restrict__ val_off, const int* __restrict__ ngd, int ntile,
                               double* __restrict__ vals) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)ntile * kTile) return;
  const int tile = (int)(idx / kTile), tid = (int)(idx - (long long)tile * kTile);
  if (tid >= tile_n[tile]) return;
  const int b0 = tile_blk[tile], b1 = tile_blk[tile + 1];
  if (b0 == b1) return;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int b = b0; b < b1; ++b) {
    const double* pp = partial + (long long)b * 3 * kTile;
    a0 += pp[tid];
    a1 += pp[kTile + tid];
    a2 += pp[2 * kTile + tid];
  }
  const int d = tile_drop[tile];
  const long long l = tgt_loc[tile_t0[tile] + tid];
  const long long ng = ngd[d];
  double* v = vals + val_off[d] + l;
  v[0] += a0;
  v[ng] += a1;
  v[2 * ng] += a2;
}

// Q[c][off_d + s] = wJ[s] * grid[d][c][s] for the nd drops of one degree group, whose source records
// rec [7][N] start at 7 * off_d (weight in row 6).
template <typename R>
__global__ void k_weight_sources(const R* __restrict__ grid, const double* __restrict__ rec,
                                 const long long* __restrict__ off, long long N, long long nd, R* __restrict__ Q,
                                 long long ldq) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nd * 3 * N) return;
  const long long d = idx / (3 * N);
  const long long r = idx - d * 3 * N;
  const int c = (int)(r / N);
  const long long s = r - c * N;
  const long long o = off[d];
  Q[c * ldq + o + s] = (R)rec[7 * o + 6 * N + s] * grid[idx];
}

// sum_s x.n wJ over one drop's records (for the volume), and max_s |x - c|, via atomics on doubles
__global__ void k_drop_stats(const double* __restrict__ rec, long long N, double cx, double cy, double cz,
                             double* __restrict__ out) {
  __shared__ double sv[kThreads], sm[kThreads];
  double v = 0, mx = 0;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    const double x = rec[s], y = rec[N + s], z = rec[2 * N + s];
    v += (x * rec[3 * N + s] + y * rec[4 * N + s] + z * rec[5 * N + s]) * rec[6 * N + s];
    const double dx = x - cx, dy = y - cy, dz = z - cz;
    mx = fmax(mx, sqrt(dx * dx + dy * dy + dz * dz));
  }
  sv[threadIdx.x] = v;
  sm[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sv[threadIdx.x] += sv[threadIdx.x + o];
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sv[0];
    out[2 * blockIdx.x + 1] = sm[0];
  }
}

// SoA source positions relative to the drop centre and normals, in precision R
template <typename R>
__global__ void k_source_geometry(const double* __restrict__ rec, long long N, double cx, double cy, double cz,
                                  R* __restrict__ X, R* __restrict__ Nn, long long ld) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  X[s] = (R)(rec[s] - cx);
  X[ld + s] = (R)(rec[N + s] - cy);
  X[2 * ld + s] = (R)(rec[2 * N + s] - cz);
  Nn[s] = (R)rec[3 * N + s];
  Nn[ld + s] = (R)rec[4 * N + s];
  Nn[2 * ld + s] = (R)rec[5 * N + s];
}

}  // namespace

int launch_classify(const double* rec_std, long long ntarget, const int* tdrop, const long long* tloc,
                    const long long* toff_std, const int* ngd, int ndrop, const double* centre, const double* bound,
                    const double* h, double a_tilde, const double* rec_up, const long long* up_off,
                    const long long* up_n, unsigned char* region, cudaStream_t s) {
  long long n = ntarget * ndrop;
  if (n == 0) return BIE_OK;
  k_classify<<<blocks_for(n), kThreads, 0, s>>>(rec_std, ntarget, tdrop, tloc, toff_std, ngd, ndrop, centre, bound, h,
                                                a_tilde, rec_up, up_off, up_n, region);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R, int TPT, int PF = 0, int CH = kChunkX2>
static void interdrop_kernel(int kind, int nblk, const PairItem* items, const int* blk_item, const long long* tile_t0,
                             const int* tile_n, const int* tile_drop, const long long* tgt_loc,
                             const long long* toff_std, const int* ngd, const double* rec_std, const double* centre,
                             const R* Xs, const R* Ns, const R* Qs, long long nstd, const R* Xu, const R* Nu,
                             const R* Qu, long long nup, const double* wts, double* partial, cudaStream_t s) {
  if constexpr (std::is_same<R, float>::value && TPT % 2 == 0) {
    // FP32 with two or more targets per thread: packed lane pairs
    if (kind == 0)
      k_interdrop_x2<0, TPT, PF, CH><<<nblk, kTile / TPT, 0, s>>>(items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc,
                                                              toff_std, ngd, rec_std, centre, Xs, Ns, Qs, nstd, Xu,
                                                              Nu, Qu, nup, wts, partial);
    else
      k_interdrop_x2<1, TPT, PF, CH><<<nblk, kTile / TPT, 0, s>>>(items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc,
                                                              toff_std, ngd, rec_std, centre, Xs, Ns, Qs, nstd, Xu,
                                                              Nu, Qu, nup, wts, partial);
    return;
  }
  if (kind == 0)
    k_interdrop<R, 0, TPT><<<nblk, kTile / TPT, 0, s>>>(items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc,
                                                        toff_std, ngd, rec_std, centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu,
                                                        nup, wts, partial);
  else
    k_interdrop<R, 1, TPT><<<nblk, kTile / TPT, 0, s>>>(items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc,
                                                        toff_std, ngd, rec_std, centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu,
                                                        nup, wts, partial);
}

template <typename R>
int launch_interdrop(int kind, int tpt, int nblk, const PairItem* items, const int* blk_item, const long long* tile_t0,
                     const int* tile_n, const int* tile_drop, const long long* tgt_loc, const long long* toff_std,
                     const int* ngd, const double* rec_std, const double* centre, const R* Xs, const R* Ns,
                     const R* Qs, long long nstd, const R* Xu, const R* Nu, const R* Qu, long long nup,
                     const double* wts, double* partial, cudaStream_t s) {
  if (nblk == 0) return BIE_OK;
  if (std::is_same<R, float>::value && (tpt == 12 || tpt == 14 || tpt == 24 || tpt == 34)) {
    // packed FP32: 12, 14 = 2 or 4 targets per thread with pipelined staging; 24, 34 = 4 targets per
    // thread with 32-source chunks, without and with pipelined staging
    if (tpt == 12)
      interdrop_kernel<R, 2, 1>(kind, nblk, items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc, toff_std, ngd,
                                rec_std, centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu, nup, wts, partial, s);
    else if (tpt == 14)
      interdrop_kernel<R, 4, 1>(kind, nblk, items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc, toff_std, ngd,
                                rec_std, centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu, nup, wts, partial, s);
    else if (tpt == 24)
      interdrop_kernel<R, 4, 0, 32>(kind, nblk, items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc, toff_std, ngd,
                                    rec_std, centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu, nup, wts, partial, s);
    else
      interdrop_kernel<R, 4, 1, 32>(kind, nblk, items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc, toff_std, ngd,
                                    rec_std, centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu, nup, wts, partial, s);
    count_launch();
    BIE_CUDA_TRY(cudaGetLastError());
    return BIE_OK;
  }
  if (tpt == 1)
    interdrop_kernel<R, 1>(kind, nblk, items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc, toff_std, ngd, rec_std,
                           centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu, nup, wts, partial, s);
  else if (tpt == 4)
    interdrop_kernel<R, 4>(kind, nblk, items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc, toff_std, ngd, rec_std,
                           centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu, nup, wts, partial, s);
  else
    interdrop_kernel<R, 2>(kind, nblk, items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc, toff_std, ngd, rec_std,
                           centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu, nup, wts, partial, s);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_interdrop_df(int kind, int nblk, const PairItem* items, const int* blk_item, const long long* tile_t0,
                        const int* tile_n, const int* tile_drop, const long long* tgt_loc, const long long* toff_std,
                        const int* ngd, const double* rec_std, const double* centre, const double* Xs,
                        const double* Ns, const double* Qs, long long nstd, const double* Xu, const double* Nu,
                        const double* Qu, long long nup, const double* wts, double* partial, cudaStream_t s) {
  if (nblk == 0) return BIE_OK;
  constexpr int TPT = 2;
  auto kern = kind == 0 ? k_interdrop_df<0, TPT> : k_interdrop_df<1, TPT>;
  kern<<<nblk, kTile / TPT, 0, s>>>(items, blk_item, tile_t0, tile_n, tile_drop, tgt_loc, toff_std, ngd, rec_std,
                                    centre, Xs, Ns, Qs, nstd, Xu, Nu, Qu, nup, wts, partial);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_tile_masks(const unsigned char* region, int nd, const long long* tile_t0, const int* tile_n,
                      long long ntile, TileMask* out, cudaStream_t s) {
  const long long n = ntile * nd;
  if (n == 0) return BIE_OK;
  k_tile_masks<<<blocks_for(n), kThreads, 0, s>>>(region, nd, tile_t0, tile_n, ntile, out);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_reduce_tiles(const double* partial, const int* tile_blk, const long long* tile_t0, const int* tile_n,
                        const int* tile_drop, const long long* tgt_loc, const long long* val_off, const int* ngd,
                        int ntile, double* vals, cudaStream_t s) {
  long long n = (long long)ntile * kTile;
  if (n == 0) return BIE_OK;
  k_reduce_tiles<<<blocks_for(n), kThreads, 0, s>>>(partial, tile_blk, tile_t0, tile_n, tile_drop, tgt_loc, val_off,
                                                     ngd, ntile, vals);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R>
int launch_weight_sources(const R* grid, const double* rec, const long long* off, long long N, long long nd, R* Q,
                          long long ldq, cudaStream_t s) {
  if (N == 0 || nd == 0) return BIE_OK;
  k_weight_sources<R><<<blocks_for(nd * 3 * N), kThreads, 0, s>>>(grid, rec, off, N, nd, Q, ldq);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_drop_stats(const double* rec, long long N, const double* c, double* out2x64, cudaStream_t s) {
  k_drop_stats<<<64, kThreads, 0, s>>>(rec, N, c[0], c[1], c[2], out2x64);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template <typename R>
int launch_source_geometry(const double* rec, long long N, const double* c, R* X, R* Nn, long long ld,
                           cudaStream_t s) {
  if (N == 0) return BIE_OK;
  k_source_geometry<R><<<blocks_for(N), kThreads, 0, s>>>(rec, N, c[0], c[1], c[2], X, Nn, ld);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

template int launch_interdrop<double>(int, int, int, const PairItem*, const int*, const long long*, const int*,
                                      const int*, const long long*, const long long*, const int*, const double*,
                                      const double*, const double*, const double*, const double*, long long,
                                      const double*, const double*, const double*, long long, const double*, double*,
                                      cudaStream_t);
template int launch_interdrop<float>(int, int, int, const PairItem*, const int*, const long long*, const int*, const int*,
                                     const long long*, const long long*, const int*, const double*, const double*,
                                     const float*, const float*, const float*, long long, const float*, const float*,
                                     const float*, long long, const double*, double*, cudaStream_t);
template int launch_weight_sources<double>(const double*, const double*, const long long*, long long, long long,
                                           double*, long long, cudaStream_t);
template int launch_weight_sources<float>(const float*, const double*, const long long*, long long, long long, float*,
                                          long long, cudaStream_t);
template int launch_source_geometry<double>(const double*, long long, const double*, double*, double*, long long,
                                            cudaStream_t);
template int launch_source_geometry<float>(const double*, long long, const double*, float*, float*, long long,
                                           cudaStream_t);

}  // namespace bie
