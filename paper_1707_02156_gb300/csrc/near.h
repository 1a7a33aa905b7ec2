// Near-singular (Omega_2) step of Sec. 2.3: records and launchers.
#pragma once
#include <cuda_runtime.h>

namespace bie {

// One (target, source drop) pair of the nearest region, with its closest point.
struct NearPair {
  long long target;  // global target index
  int src_drop;
  int pad;
  double d0;         // |x0 - x*|
  double theta_v;    // parameters of x* in the source drop's own parametrisation
  double phi_v;
};

int launch_near_seed(const NearPair* pairs, int npair, const double* rec_std, const long long* toff, const int* ngd,
                     const long long* tgt_loc, const int* tdrop, int* seed, cudaStream_t s);
// shape coefficients of each pair's source drop with its seed longitude's phases applied (ph:
// [pair][pmax+1][2] cos, sin of m alpha), to out + dst_off[pair] as [3][(p+1)^2]
int launch_near_phase_shift(const NearPair* pairs, int npair, const double* coef, const long long* coef_off,
                            const int* pdeg, int pmax, const double* ph, const long long* dst_off, double* out,
                            cudaStream_t s);
// the Legendre recursion's coefficients for degrees up to P (near_rec_table_doubles(P) doubles), which
// the closest-point Newton iteration reads
int near_rec_table_doubles(int P);
int launch_near_rec_table(int P, double* tab, cudaStream_t s);
int launch_near_newton(const NearPair* pairs, int npair, const double* xr, const int* pdeg, const long long* xr_off,
                       const double* x0, const double* tab, double* result, cudaStream_t s);
int launch_near_checkgrid(const NearPair* pairs, int npair, int L, const double* pts, const double* centre,
                          const double* bound, const double* h, double a_tilde, const double* rec_up,
                          const long long* up_off, const long long* up_n, int* grid, cudaStream_t s);
template <typename R>
int launch_near_checks(int kind, const NearPair* pairs, int npair, int L, const double* pts, const int* grid,
                       const double* centre, const long long* toff, const int* ngd, const long long* up_off,
                       const long long* up_n, const R* Xs, const R* Ns, const R* Qs, long long nstd, const R* Xu,
                       const R* Nu, const R* Qu, long long nup, const double* wts, double* cv, cudaStream_t s);
int launch_near_interp(const NearPair* pairs, const int* tbeg, int ntgt, int L, int kind, const double* selfcoef,
                       const double* dens, const long long* coef_off, const int* pdeg, const double* hdrop,
                       const double* wts, const double* cv, const int* tdrop, const long long* tgt_loc,
                       const long long* val_off, const int* ngd, double* vals, cudaStream_t s);

}  // namespace bie
