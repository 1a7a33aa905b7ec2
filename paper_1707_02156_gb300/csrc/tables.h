// Host-side plan tables for the SH Stokes layer operators (built once per degree, FP64).
#pragma once
#include <vector>

namespace bie {

// Gauss-Legendre nodes t_j (ascending) and weights on [-1,1], n points (Sec. 2.1 grid).
void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w);

// Offset of row (m, n) in an [m][n][j] table for 0 <= m <= n <= p with nj entries per row.
inline long long legendre_row(int p, int m, int n, int nj) {
  // rows of m' < m: sum_{m'<m} (p+1-m') = m(p+1) - m(m-1)/2
  long long before = (long long)m * (p + 1) - (long long)m * (m - 1) / 2;
  return (before + (n - m)) * nj;
}
inline long long legendre_size(int p, int nj) { return (long long)(p + 1) * (p + 2) / 2 * nj; }

// Normalised associated Legendre functions P~_n^m(cos theta_j) (App. A) on the Gauss grid of
// degree P, for 0 <= m <= n <= p, and their first and second theta derivatives.
// kind 0: value, 1: d/dtheta, 2: d2/dtheta2.  Layout [m][n][j], j = 0..P.
void legendre_table(int p, int P, int kind, std::vector<double>& out);

// Analysis table: (pi/(P+1)) w_j P~_n^m(t_j), same layout (forward transform of Sec. 2.1).
void analysis_table(int p, int P, std::vector<double>& out);

// cos(m phi_k), sin(m phi_k) for m = 0..p and k = 0..2P+1: layout [m][k][2].
void phase_table(int p, int P, std::vector<double>& out);

// Wigner rotation blocks for the rotated expansion g(s) = f(R_z(alpha) R_y(beta) s):
// per degree n, the real (n+1)x(n+1) block acting on Re(e^{i m alpha} f_n^m), m = 0..n,
// followed by the n x n block acting on the imaginary parts, m = 1..n (App. B, real symmetry).
// Both blocks are stored column-major (entry (m', m) at m (n+1) + m', resp. (m-1) n + (m'-1)), so
// threads computing consecutive outputs m' read consecutive addresses.
long long wigner_block_stride(int p);                 // doubles per beta
inline long long wigner_block_offset(int n) {         // offset of degree n inside one beta
  // sum_{k<n} (k+1)^2 + k^2
  long long s = 0;
  for (int k = 0; k < n; ++k) s += (long long)(k + 1) * (k + 1) + (long long)k * k;
  return s;
}
void wigner_blocks(int p, double beta, double* out);  // out: wigner_block_stride(p) doubles
// Dense small-d matrix d^n_{m'm}(beta), rows m' = -n..n, columns m = -n..n (for tests).
void wigner_small_d(int n, double beta, double* out);

// Singular weights w_j^s of Thm 1 on the grid of degree pq (with the regular factor
// pi/(pq+1) w_j; the integrand carries W/sin(theta_j)).
void singular_weights(int pq, std::vector<double>& out);

}  // namespace bie
