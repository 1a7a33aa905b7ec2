// Launchers of the off-surface evaluation (Sec. 1, with the region rules of Sec. 2.1-2.3).
#pragma once
#include <cuda_runtime.h>

#include "interdrop.h"
#include "near.h"

namespace bie {

// region[t * nd + j], t < n: the points t0 + t of pts [3][ld] against drop j (0 / 1 / 2 = Omega_0/1/2,
// 3 = inside drop j).  list: n * nd entries of scratch, count: one (device); n * nd < 2^32; sms: the
// device's multiprocessors (sizes the second pass)
int launch_classify_points(const double* pts, long long ld, long long t0, long long n, int nd, const double* centre,
                           const double* bound, const double* h, double a_tilde, const double* rec_up,
                           const long long* up_off, const long long* up_n, unsigned char* region, unsigned* list,
                           unsigned* count, int sms, cudaStream_t s);
// the n points t0.. of pts as target records rec [ntile][7][kTile] and the tiles' centres
// centre[3 * (nd + tile)]
int launch_point_records(const double* pts, long long ld, long long t0, long long n, int ntile, int nd, double* rec,
                         double* centre, cudaStream_t s);
// out[c][t0 + t] += vals[tile][c][k], t = tile * kTile + k < n
int launch_gather_points(const double* vals, long long t0, long long n, long long ld, double* out, cudaStream_t s);
// nearest standard-grid point of the pair's source drop to the pair's point (pairs[i].target indexes pts)
int launch_near_seed_points(const NearPair* pairs, int npair, const double* pts, long long ld, const double* rec_std,
                            const long long* toff, const int* ngd, int* seed, cudaStream_t s);
// out = uinf + (S + D) / 2 over n values (uinf may be null)
int launch_velocity(const double* uinf, const double* S, const double* D, long long n, double* out, cudaStream_t s);

}  // namespace bie
