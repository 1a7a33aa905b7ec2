// Work items and launchers of the inter-drop pair sums (Sec. 2.1, 2.3).
#pragma once
#include <cuda_runtime.h>

namespace bie {

constexpr int kTile = 128;  // targets per tile (one thread per target)

// One unit of inter-drop work: the targets of `tile` selected by `mask` against sources
// [s0, s1) of `grid` (0 standard, 1 upsampled) of drop `src_drop`.
struct PairItem {
  int tile;
  int src_drop;
  int grid;
  int pad;
  long long s0, s1;
  unsigned mask[4];
};

// targets of a tile per region of one source drop (bit k of m[r] = target k in region r)
struct TileMask {
  unsigned m[3][4];
  int inside;  // some target lies inside the source drop
};
int launch_tile_masks(const unsigned char* region, int nd, const long long* tile_t0, const int* tile_n,
                      long long ntile, TileMask* out, cudaStream_t s);
int launch_classify(const double* rec_std, long long ntarget, const int* tdrop, const long long* tloc,
                    const long long* toff_std, const int* ngd, int ndrop, const double* centre, const double* bound,
                    const double* h, double a_tilde, const double* rec_up, const long long* up_off,
                    const long long* up_n, unsigned char* region, cudaStream_t s);
// tpt: targets per thread (1, 2 or 4; chosen per geometry by timing, see autotune_interdrop); for FP32,
// 12 and 14 select the packed kernel with 2 or 4 targets per thread and pipelined source staging,
// 24 and 34 the packed kernel with 4 targets per thread and 32-source chunks (34: pipelined)
template <typename R>
int launch_interdrop(int kind, int tpt, int nblk, const PairItem* items, const int* blk_item, const long long* tile_t0,
                     const int* tile_n, const int* tile_drop, const long long* tgt_loc, const long long* toff_std,
                     const int* ngd, const double* rec_std, const double* centre, const R* Xs, const R* Ns,
                     const R* Qs, long long nstd, const R* Xu, const R* Nu, const R* Qu, long long nup,
                     const double* wts, double* partial, cudaStream_t s);
// the same pair sums in double-float arithmetic (FP32 pipes, about 44 bits) from FP64 sources
int launch_interdrop_df(int kind, int nblk, const PairItem* items, const int* blk_item, const long long* tile_t0,
                        const int* tile_n, const int* tile_drop, const long long* tgt_loc, const long long* toff_std,
                        const int* ngd, const double* rec_std, const double* centre, const double* Xs,
                        const double* Ns, const double* Qs, long long nstd, const double* Xu, const double* Nu,
                        const double* Qu, long long nup, const double* wts, double* partial, cudaStream_t s);
int launch_reduce_tiles(const double* partial, const int* tile_blk, const long long* tile_t0, const int* tile_n,
                        const int* tile_drop, const long long* tgt_loc, const long long* val_off, const int* ngd,
                        int ntile, double* vals, cudaStream_t s);
template <typename R>
int launch_weight_sources(const R* grid, const double* rec, const long long* off, long long N, long long nd, R* Q,
                          long long ldq, cudaStream_t s);
int launch_drop_stats(const double* rec, long long N, const double* c, double* out2x64, cudaStream_t s);
template <typename R>
int launch_source_geometry(const double* rec, long long N, const double* c, R* X, R* Nn, long long ld,
                           cudaStream_t s);

}  // namespace bie
