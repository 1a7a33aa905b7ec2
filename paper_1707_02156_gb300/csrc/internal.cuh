// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bie.h"

namespace bie {

void set_error(const std::string& msg);
void count_launch(int n = 1);  // kernel launches issued by the library (all threads)
int ctx_device(const bie_ctx* ctx);  // CUDA device ordinal of a context

#define BIE_CUDA_TRY(expr)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      ::bie::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));                    \
      return BIE_ECUDA;                                                                        \
    }                                                                                          \
  } while (0)

#define BIE_TRY(expr)              \
  do {                             \
    int s_ = (expr);               \
    if (s_ != BIE_OK) return s_;   \
  } while (0)

__host__ __device__ inline long long leg_row(int p, int m, int n, int nj) {
  long long before = (long long)m * (p + 1) - (long long)m * (m - 1) / 2;
  return (before + (n - m)) * nj;
}

// ---- transforms (transforms.cu) ----
// Legendre step of synthesis: H[f][m][j] = sum_n c_f(n,m) T[m][n][j] (complex, m >= 0), with an
// optional phi-derivative factor (i m)^dphi.  Coefficients of field f start at
// field_off ? field_off[f] : f * coef_stride.
template <typename CT, typename R>
int launch_leg_synth(const CT* coef, const long long* field_off, long long coef_stride, long long nfield, int p,
                     const R* T, int nj, R* H, int dphi, cudaStream_t s);
// phi step of synthesis: out[f][j][k] = Re sum_m fac_m H[f][m][j] e^{i m phi_k}, k < 2P+2
template <typename R, typename OT>
int launch_phi_synth(const R* H, long long nfield, int p, int P, const R* cs, OT* out,
                     const long long* out_off, long long out_stride, cudaStream_t s);
// analysis: grid (degree P) -> coefficients (degree p_out), FP64
int launch_analyze(const double* grid, const long long* grid_off, long long grid_stride, long long nfield, int P,
                   int p_out, const double* cs, const double* A, double* F, double* coef,
                   const long long* coef_off, long long coef_stride, cudaStream_t s);
// analysis of nfield fields on their own degree-p grids, for several degree groups in one launch
// (grid_off, coef_off per field; begin is set by the launcher)
struct AnaGroup {
  long long begin, nfield;
  const long long* grid_off;
  const long long* coef_off;
  const double* cs;
  const double* A;
  int p;
};
constexpr int kMaxAnaGroups = 8;
struct AnaGroups {
  int n;
  AnaGroup g[kMaxAnaGroups];
};
int launch_analyze_fused(const std::vector<AnaGroup>& groups, const double* grid, double* coef, cudaStream_t s);
// rotation (App. B): out[ld][a*nb+b][c] = blocks(a) applied to e^{i m alpha_b} coef[ld][c]
template <typename CT, typename R>
int launch_rotate(const CT* coef, const long long* field_off, int ncomp, long long ndrop, int p, const R* blocks,
                  long long blk_stride, int na, int nb, const R* ph, R* out, long long out_drop_stride,
                  cudaStream_t s);
// multiply coefficients by e^{i m gamma} (in place), ncomp fields per drop
int launch_phase(double* coef, long long nfield, int p, double gamma, cudaStream_t s);

// ---- pair sums and geometry (pairs.cu) ----
// Surface quantities from x, x_theta, x_phi grids [f=drop*3+c][j][k]: writes SoA source records
// [drop][7][N] = (x, n, wgt*J) with wgt the regular weight (pi/(P+1)) w_j, J = W/sin(theta_j).
int launch_surface(const double* X, const double* Xt, const double* Xp, long long ndrop, int P,
                   const double* wsin /*[j] = w_j pi/(P+1)/sin theta_j*/, double* rec, cudaStream_t s);
// Rotated-grid cache for ndrop drops of ng targets each: cache[t][7][nq] = (x0 - x', n',
// w^s_j W'/sin theta_j) on the degree-pq grid; x0 of drop ld's targets read from the standard-grid
// records at rec_std + rec_off[ld] ([7][ng] per drop; the drops need not be adjacent there).
template <typename R>
int launch_rotgeo(const double* X, const double* Xt, const double* Xp, long long ndrop, int ng, int pq,
                  const double* rec_std, const long long* rec_off, const double* wsq, R* cache, cudaStream_t s);
// Singular self interaction (Thm 1, Sec. 2.2), one block per target of ndrop drops of degree p:
// direct form against the rotated-geometry cache, or projected form against Q (see self.cu).
template <typename R>
int launch_self_direct(int kind, const double* dens, const long long* foff3, long long ndrop, int p, int pq,
                       const R* wblk, long long wstride, const R* ph, const R* T0, const R* cs, const R* cache,
                       const double* wts, const long long* val_off, double* vals, size_t smem_budget,
                       cudaStream_t s);
// Projected kernel factors Q[t][12][tri(n,m)] of ntarget targets (see self.cu), from the FP64
// rotated-geometry cache and the degree-pq grid's Legendre table T0 (degrees <= p, all nodes).
size_t kernel_proj_smem(int p, int pq);
int launch_kernel_proj(int kind, const double* cache, long long ntarget, int p, int pq, const double* cs,
                       const double* T0, double* Q64, float* Q32, cudaStream_t s);
// One degree group of the projected-form apply (device pointers; begin is set by the launcher).
template <typename R>
struct SelfGroup {
  long long begin;          // first block of the group
  long long ndrop;          // drops of the group
  const long long* foff3;   // [drop][3] offsets of the density coefficients
  const R* wblk;            // Wigner blocks of the group's latitudes, wstride apart
  long long wstride;
  const R* ph;              // cos, sin (m phi_b) of the degree-p grid
  const R* Q;               // projected kernel factors
  const double* wts;        // per-drop weight
  const long long* val_off; // per-drop offset into vals
  int p;
};
constexpr int kMaxSelfGroups = 8;
template <typename R>
struct SelfGroups {
  int n;
  SelfGroup<R> g[kMaxSelfGroups];
};
// out[i] = double-float split of in[i] (dff: dfloat.cuh)
struct dff;
int launch_split_dff(const double* in, dff* out, long long n, cudaStream_t s);
// All projected-form groups in one launch (eight groups per launch at most).
template <typename R, typename CT>
int launch_self_proj(std::vector<SelfGroup<R>> groups, const CT* dens, double* vals, cudaStream_t s);
// The FP32 projected form with the Wigner rotation on the tensor cores (self_tc.cu): per chunk of
// drops of one degree, the rotation products into eo (at most `budget` floats per chunk, at least one
// drop's worth), then the contraction with the factors.  self_tc_eo_floats = the buffer it needs.
long long self_tc_eo_floats(const std::vector<SelfGroup<float>>& groups, long long budget);
long long self_tc_g_floats(const std::vector<SelfGroup<float>>& groups, long long budget);
// whether k_rot_tc's shared memory at degree p fits one block (degrees up to 58)
bool self_tc_fits(int p);
int launch_self_tc(const std::vector<SelfGroup<float>>& groups, const double* dens, double* vals, float* eo,
                   unsigned* gm, long long budget, cudaStream_t s);
// interfacial force at N grid points from x derivatives [6][3][N] and Gamma derivatives [3][N]
int launch_force(const double* X, const double* Gm, long long N, double es, double xs, double* f, cudaStream_t s);
// out[i] = (float) in[i]
int launch_to_float(const double* in, float* out, long long n, cudaStream_t s);

// ---- surfactant transport (surfactant.cu) ----
// f_E and (fi non-null) inv_pe * lap Gamma at the N grid points of nd drops: X [6][nd*3][N] (x and
// its derivatives f, t, p, tt, tp, pp), U [3][nd*3][N] (u: f, t, p), Gm [6][nd][N]; fe, fi [nd][N]
int launch_surf_rates(const double* X, const double* U, const double* Gm, long long nd, long long N, double inv_pe,
                      double* fe, double* fi, cudaStream_t s);
// coefficients of the surface Laplacian L[5][nd][N] (s_tt, s_tp, s_pp, s_t, s_p) from X [6][nd*3][N]
int launch_lap_coef(const double* X, long long nd, long long N, double* L, cudaStream_t s);
// out[nd][N] = lap s from L and the fields S [6][nd][N] of s (kinds t..pp used)
int launch_lap_apply(const double* L, const double* S, long long nd, long long N, double* out, cudaStream_t s);
// per-drop integral on the grid of degree P (mode 0: volume from X kinds f, t, p; mode 1: mass of
// Gm [nd][N] from X kinds t, p), wsin[j] = (pi/(P+1)) w_j / sin(theta_j); out[nd] on the device
int launch_drop_integral(const double* X, const double* Gm, long long nd, int P, const double* wsin, int mode,
                         double* out, cudaStream_t s);
// out[d] = max |F| over the nper fields of drop d, F [nd*nper][N]
int launch_drop_absmax(const double* F, long long nd, int nper, long long N, double* out, cudaStream_t s);
// w = (y - a c) * inv_diag
int launch_implicit_combine(const double* y, const double* c, double a, const double* inv_diag, long long n,
                            double* w, cudaStream_t s);
// y = x * sc (elementwise)
int launch_mul(const double* x, const double* sc, long long n, double* y, cudaStream_t s);

// ---- angle reparametrisation (reparam.cu) ----
// zero-padded copies [d][c][(P+1)^2] of degree-p coefficients at src + off[d] + c (p+1)^2
int launch_pad_coef(const double* src, const long long* off, int p, int P, long long nd, int ncomp, double* dst,
                    cudaStream_t s);
// values (and, with derivs, theta and phi derivatives) of nf (1 or 3) expansions of degree P per drop at the
// N points (th, ph)[d][N]: out[d][f][kind][N]; ab = recursion coefficients (a, b) per (m, n), rows of order m
int launch_eval_points(const double* coef, int nf, int P, long long nd, long long N, const double* th,
                       const double* ph, const double* ab, int derivs, double* out, cudaStream_t s);
// norms[d][n][2] = (sum_m |x_n^m|, sum_m |x_n^m|^2), m = -n..n, of [d][3][(P+1)^2]
int launch_mode_norms(const double* coef, int P, long long nd, double* norms, cudaStream_t s);
// out = scale * a[d][n] * in, per drop and degree
int launch_scale_degrees(const double* in, const double* a, int P, long long nd, int ncomp, double scale, double* out,
                         cudaStream_t s);
// g = tangential part of gradE at the points (E = x0 and its derivatives there), gmax[d] = max |g|
int launch_rep_gradient(const double* E, const double* gradE, long long N, long long nd, double* g, double* gmax,
                        cudaStream_t s);
// forward Euler step of the angles of the active drops with the pseudo-velocity -g
int launch_rep_step(const double* E, const double* g, long long N, long long nd, const int* active, double dtau,
                    double* th, double* ph, cudaStream_t s);
// the degree-P grid's parameter points for nd drops, from the Gauss nodes t_j
int launch_grid_points(const double* nodes, int P, long long nd, double* th, double* ph, cudaStream_t s);

}  // namespace bie
