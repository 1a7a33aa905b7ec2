// Layer potentials at points off the drop surfaces (Sec. 1: the velocity anywhere in the fluid,
// from the interface densities), each (point, drop) pair by the rule of its region (Sec. 2.1-2.3).
// The kernels here put a chunk of points into the record layout of the drops' own targets, so that
// the inter-drop pair kernels, their tile reduction and the near-singular interpolation run on them
// unchanged; they classify the points, seed the closest-point search, gather the tile sums into the
// caller's layout and form the velocity.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "offsurface.h"

namespace bie {
namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(long long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// region[t * nd + j] for the points t0 .. t0 + n - 1 of pts [3][ld]: 0 / 1 / 2 for Omega_0/1/2 of
// drop j, 3 when the point lies inside drop j.  The tests are those of the drops' own targets: the
// distance to the nearest point of drop j's upsampled grid against h_j and A h_j (after the bounding-
// sphere test), inside when the point is on the inner side of the tangent plane there.  Two passes:
// one thread per (point, drop) settles the pairs outside the bounding sphere widened by A h_j and
// lists the others; then one warp per listed pair scans the upsampled grid, its lanes striding over
// the points (the first nearest point wins ties, as in a sequential scan).
__global__ void k_classify_points_far(const double* __restrict__ pts, long long ld, long long t0, long long n, int nd,
                                      const double* __restrict__ centre, const double* __restrict__ bound,
                                      const double* __restrict__ h, double a_tilde, unsigned char* __restrict__ region,
                                      unsigned* __restrict__ list, unsigned* __restrict__ count) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nd) return;
  const long long t = idx / nd;
  const int j = (int)(idx - t * nd);
  const double x0 = pts[t0 + t], x1 = pts[ld + t0 + t], x2 = pts[2 * ld + t0 + t];
  const double dc0 = x0 - centre[3 * j], dc1 = x1 - centre[3 * j + 1], dc2 = x2 - centre[3 * j + 2];
  if (sqrt(dc0 * dc0 + dc1 * dc1 + dc2 * dc2) - bound[j] > a_tilde * h[j]) {
    region[idx] = 0;
    return;
  }
  list[atomicAdd(count, 1u)] = (unsigned)idx;
}

__global__ void k_classify_points_near(const double* __restrict__ pts, long long ld, long long t0, int nd,
                                       const double* __restrict__ h, double a_tilde,
                                       const double* __restrict__ rec_up, const long long* __restrict__ up_off,
                                       const long long* __restrict__ up_n, const unsigned* __restrict__ list,
                                       const unsigned* __restrict__ count, unsigned char* __restrict__ region) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned total = *count;
  for (long long w = warp; w < total; w += nwarp) {
    const long long idx = list[w];
    const long long t = idx / nd;
    const int j = (int)(idx - t * nd);
    const double x0 = pts[t0 + t], x1 = pts[ld + t0 + t], x2 = pts[2 * ld + t0 + t];
    const long long N = up_n[j];
    const double* r = rec_up + 7 * up_off[j];
    double best = 1e300;
    long long bi = N;
    for (long long s = lane; s < N; s += 32) {
      const double d0 = x0 - r[s], d1 = x1 - r[N + s], d2 = x2 - r[2 * N + s];
      const double d = d0 * d0 + d1 * d1 + d2 * d2;
      if (d < best) {
        best = d;
        bi = s;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {  // smallest distance, then smallest index
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob < best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      const double dist = sqrt(best);
      const double side = (x0 - r[bi]) * r[3 * N + bi] + (x1 - r[N + bi]) * r[4 * N + bi] +
                          (x2 - r[2 * N + bi]) * r[5 * N + bi];
      unsigned char code = dist <= h[j] ? 2 : (dist <= a_tilde * h[j] ? 1 : 0);
      if (side <= 0.0) code = 3;
      region[idx] = code;
    }
  }
}

// rec[tile][7][128]: rows 0-2 the chunk's points (zero past its end), rows 3-6 zero; and the tile's
// centre (mean of its points) at centre[3 * (nd + tile)], to which the FP32 pair kernel refers them.
__global__ void k_point_records(const double* __restrict__ pts, long long ld, long long t0, long long n, int ntile,
                                int nd, double* __restrict__ rec, double* __restrict__ centre) {
  const int tile = blockIdx.x;
  const int k = threadIdx.x;  // blockDim.x == kTile
  const long long t = (long long)tile * kTile + k;
  __shared__ double sum[3][kTile];
  double* r = rec + (long long)tile * 7 * kTile;
  for (int c = 0; c < 3; ++c) {
    const double v = t < n ? pts[c * ld + t0 + t] : 0.0;
    r[c * kTile + k] = v;
    sum[c][k] = v;
  }
  for (int c = 3; c < 7; ++c) r[c * kTile + k] = 0.0;
  __syncthreads();
  for (int o = kTile / 2; o > 0; o >>= 1) {
    if (k < o)
      for (int c = 0; c < 3; ++c) sum[c][k] += sum[c][k + o];
    __syncthreads();
  }
  if (k == 0) {
    const long long m = n - (long long)tile * kTile;
    const double cnt = (double)(m < kTile ? m : kTile);
    for (int c = 0; c < 3; ++c) centre[3 * (nd + tile) + c] = sum[c][0] / cnt;
  }
}

// out[c][t0 + t] += vals[tile][c][k] for the chunk's points
__global__ void k_gather_points(const double* __restrict__ vals, long long t0, long long n, long long ld,
                                double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3 * n) return;
  const int c = (int)(idx / n);
  const long long t = idx - (long long)c * n;
  const long long tile = t / kTile, k = t - tile * kTile;
  out[c * ld + t0 + t] += vals[(tile * 3 + c) * kTile + k];
}

// the index of the standard-grid point of drop pairs[i].src_drop nearest to its point
__global__ void k_near_seed_points(const NearPair* __restrict__ pairs, int npair, const double* __restrict__ pts,
                                   long long ld, const double* __restrict__ rec_std, const long long* __restrict__ toff,
                                   const int* __restrict__ ngd, int* __restrict__ seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npair) return;
  const long long t = pairs[i].target;
  const int j = pairs[i].src_drop;
  const double x0 = pts[t], x1 = pts[ld + t], x2 = pts[2 * ld + t];
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

// out = u_inf + (S + D) / 2 (u_inf may be null)
__global__ void k_velocity(const double* __restrict__ uinf, const double* __restrict__ S, const double* __restrict__ D,
                           long long n, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = (uinf ? uinf[i] : 0.0) + 0.5 * (S[i] + D[i]);
}

}  // namespace

int launch_classify_points(const double* pts, long long ld, long long t0, long long n, int nd, const double* centre,
                           const double* bound, const double* h, double a_tilde, const double* rec_up,
                           const long long* up_off, const long long* up_n, unsigned char* region, unsigned* list,
                           unsigned* count, int sms, cudaStream_t s) {
  if (n * nd == 0) return BIE_OK;
  if (n * nd > 0xffffffffLL) return BIE_EINVAL;
  BIE_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
  k_classify_points_far<<<blocks_for(n * nd), kThreads, 0, s>>>(pts, ld, t0, n, nd, centre, bound, h, a_tilde, region,
                                                                list, count);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  k_classify_points_near<<<8 * sms, kThreads, 0, s>>>(pts, ld, t0, nd, h, a_tilde, rec_up, up_off, up_n, list, count,
                                                      region);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_point_records(const double* pts, long long ld, long long t0, long long n, int ntile, int nd, double* rec,
                         double* centre, cudaStream_t s) {
  if (ntile == 0) return BIE_OK;
  k_point_records<<<ntile, kTile, 0, s>>>(pts, ld, t0, n, ntile, nd, rec, centre);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_gather_points(const double* vals, long long t0, long long n, long long ld, double* out, cudaStream_t s) {
  if (n == 0) return BIE_OK;
  k_gather_points<<<blocks_for(3 * n), kThreads, 0, s>>>(vals, t0, n, ld, out);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_near_seed_points(const NearPair* pairs, int npair, const double* pts, long long ld, const double* rec_std,
                            const long long* toff, const int* ngd, int* seed, cudaStream_t s) {
  if (npair == 0) return BIE_OK;
  k_near_seed_points<<<(npair + 127) / 128, 128, 0, s>>>(pairs, npair, pts, ld, rec_std, toff, ngd, seed);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

int launch_velocity(const double* uinf, const double* S, const double* D, long long n, double* out, cudaStream_t s) {
  if (n == 0) return BIE_OK;
  k_velocity<<<blocks_for(n), kThreads, 0, s>>>(uinf, S, D, n, out);
  count_launch();
  BIE_CUDA_TRY(cudaGetLastError());
  return BIE_OK;
}

}  // namespace bie
