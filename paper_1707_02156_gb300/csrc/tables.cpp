// Host-side plan tables (FP64 results; long double where it is cheap).
//
// Gauss grid (Sec. 2.1), normalised associated Legendre functions (App. A recursion),
// their theta derivatives (ladder form of the App. A identities), Wigner small-d matrices
// (App. B) by the three-term recursion in the degree, singular weights (Thm 1).
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace bie {

typedef long double ld;

static const ld kPi = 3.141592653589793238462643383279502884L;

void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w) {
  t.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    // Newton on P_n from the Tricomi-type initial guess; node i counted from x = +1.
    ld x = std::cos(kPi * (i + 0.75L) / (n + 0.5L));
    ld dp = 0;
    for (int it = 0; it < 100; ++it) {
      ld p0 = 1, p1 = x;
      if (n == 0) p1 = 1;
      for (int k = 2; k <= n; ++k) {
        ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(x), p0 = P_{n-1}(x)
      dp = n * (x * p1 - p0) / (x * x - 1);
      ld dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-19L) {
        // one more evaluation of the derivative at the converged node
        p0 = 1;
        p1 = x;
        for (int k = 2; k <= n; ++k) {
          ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1);
        break;
      }
    }
    // ascending order: node i from the top goes to index n-1-i
    t[n - 1 - i] = (double)x;
    w[n - 1 - i] = (double)(2.0L / ((1 - x * x) * dp * dp));
  }
}

// P~_n^k(x) for 0 <= k <= n <= pmax into P[n*(pmax+1)+k].
static void legendre_all(int pmax, ld x, std::vector<ld>& P) {
  P.assign((size_t)(pmax + 1) * (pmax + 1), 0);
  ld s = std::sqrt(std::max((ld)0, 1 - x * x));
  auto at = [&](int n, int m) -> ld& { return P[(size_t)n * (pmax + 1) + m]; };
  at(0, 0) = std::sqrt(1.0L / (4 * kPi));
  for (int m = 1; m <= pmax; ++m) at(m, m) = -std::sqrt(1 + 1.0L / (2 * m)) * s * at(m - 1, m - 1);
  for (int m = 0; m < pmax; ++m) at(m + 1, m) = std::sqrt(2.0L * m + 3) * x * at(m, m);
  for (int m = 0; m <= pmax; ++m)
    for (int n = m + 2; n <= pmax; ++n) {
      ld a = std::sqrt((4.0L * n * n - 1) / ((ld)n * n - (ld)m * m));
      ld b = -std::sqrt(((ld)(n - 1) * (n - 1) - (ld)m * m) / (4.0L * (n - 1) * (n - 1) - 1));
      at(n, m) = a * (x * at(n - 1, m) + b * at(n - 2, m));
    }
}

void legendre_table(int p, int P, int kind, std::vector<double>& out) {
  std::vector<double> t, w;
  gauss_legendre(P + 1, t, w);
  const int nj = P + 1;
  out.assign(legendre_size(p, nj), 0.0);
  std::vector<ld> L;
  for (int j = 0; j < nj; ++j) {
    legendre_all(p, (ld)t[j], L);
    // signed-order access: P~_n^{-k} = (-1)^k P~_n^k, zero for |k| > n
    auto get = [&](int n, int k) -> ld {
      if (k > n || -k > n) return 0;
      if (k < 0) return ((-k) & 1 ? -1 : 1) * L[(size_t)n * (p + 1) - k];
      return L[(size_t)n * (p + 1) + k];
    };
    // ladder form: dP~_n^k/dtheta = (a_k P~_n^{k+1} - b_k P~_n^{k-1}) / 2
    auto dget = [&](int n, int k) -> ld {
      if (k > n || -k > n) return 0;
      ld a = std::sqrt((ld)(n - k) * (n + k + 1));
      ld b = std::sqrt((ld)(n + k) * (n - k + 1));
      return 0.5L * (a * get(n, k + 1) - b * get(n, k - 1));
    };
    for (int m = 0; m <= p; ++m)
      for (int n = m; n <= p; ++n) {
        ld v;
        if (kind == 0) {
          v = get(n, m);
        } else if (kind == 1) {
          v = dget(n, m);
        } else {
          ld a = std::sqrt((ld)(n - m) * (n + m + 1));
          ld b = std::sqrt((ld)(n + m) * (n - m + 1));
          v = 0.5L * (a * dget(n, m + 1) - b * dget(n, m - 1));
        }
        out[legendre_row(p, m, n, nj) + j] = (double)v;
      }
  }
}

void analysis_table(int p, int P, std::vector<double>& out) {
  std::vector<double> t, w;
  gauss_legendre(P + 1, t, w);
  legendre_table(p, P, 0, out);
  const int nj = P + 1;
  const ld fac = kPi / (P + 1);
  for (int m = 0; m <= p; ++m)
    for (int n = m; n <= p; ++n)
      for (int j = 0; j < nj; ++j) {
        long long i = legendre_row(p, m, n, nj) + j;
        out[i] = (double)(fac * (ld)w[j] * (ld)out[i]);
      }
}

void phase_table(int p, int P, std::vector<double>& out) {
  const int nk = 2 * P + 2;
  out.assign((size_t)(p + 1) * nk * 2, 0.0);
  for (int m = 0; m <= p; ++m)
    for (int k = 0; k < nk; ++k) {
      long long r = ((long long)m * k) % nk;  // m phi_k = pi r/(P+1) modulo 2 pi
      ld a = kPi * (ld)r / (P + 1);
      out[((size_t)m * nk + k) * 2 + 0] = (double)std::cos(a);
      out[((size_t)m * nk + k) * 2 + 1] = (double)std::sin(a);
    }
}

long long wigner_block_stride(int p) { return wigner_block_offset(p + 1); }

// d^j_{mp,m}(beta) at j0 = max(|m|,|mp|): the factorial sum of App. B has a single term there,
// K(mp, m) cos(beta/2)^e1 sin(beta/2)^e2 with a sign.  With j0 the larger of |m|, |mp|, K is the
// square root of a binomial coefficient, sqrt(C(2 j0, j0 + r)) with r = mp or m (whichever is not
// +-j0); it is formed as a product of ratios, exact to a few units of rounding.
static double start_const(int mp, int m) {
  const int j = std::max(std::abs(mp), std::abs(m));
  const int r = std::abs(mp) == j ? m : mp;
  const int k = std::min(j + r, j - r);  // C(2j, j + r) = C(2j, k)
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c = c * (double)(2 * j - k + i) / (double)i;
  return std::sqrt(c);
}

// d^j_{mp,m}(beta) for j = 0..p into col[j] (zero below j0), three-term recursion in j (double;
// the recursion is stable and loses about 1e-14 relative up to degree 64).
static void small_d_column(int p, int mp, int m, double cb, double ch, double sh, double* col) {
  for (int j = 0; j <= p; ++j) col[j] = 0.0;
  const int j0 = std::max(std::abs(m), std::abs(mp));
  if (j0 > p) return;
  {
    const int s = std::max(0, m - mp);
    const int e1 = 2 * (j0 - s) + m - mp, e2 = 2 * s - m + mp;
    const double v = start_const(mp, m) * std::pow(ch, (double)e1) * std::pow(sh, (double)e2);
    col[j0] = ((mp - m + s) & 1) ? -v : v;
  }
  const double mm = (double)m * m, pp = (double)mp * mp, mpm = (double)m * mp;
  for (int j = j0 + 1; j <= p; ++j) {
    if (j == 1) {  // j0 = 0, m = mp = 0
      col[1] = cb * col[0];
      continue;
    }
    const double jj = (double)j * j, j1 = (double)(j - 1) * (j - 1);
    const double a = (double)j * (2 * j - 1) / std::sqrt((jj - mm) * (jj - pp));
    const double t1 = (cb - mpm / ((double)j * (j - 1))) * col[j - 1];
    double t2 = 0;
    if (j - 2 >= j0) t2 = std::sqrt((j1 - mm) * (j1 - pp)) / ((double)(j - 1) * (2 * j - 1)) * col[j - 2];
    col[j] = a * (t1 - t2);
  }
}

void wigner_small_d(int n, double beta, double* out) {
  std::vector<double> col(n + 1);
  const double cb = std::cos(beta), ch = std::cos(beta / 2), sh = std::sin(beta / 2);
  for (int mp = -n; mp <= n; ++mp)
    for (int m = -n; m <= n; ++m) {
      small_d_column(n, mp, m, cb, ch, sh, col.data());
      out[(mp + n) * (2 * n + 1) + (m + n)] = col[n];
    }
}

void wigner_blocks(int p, double beta, double* out) {
  // rotated coefficient g_{n m'} = sum_m D_{m'm} e^{i m alpha} f_{n m}, D_{m'm} = d^n_{m m'}; the
  // blocks need the columns d^n_{+-m, m'} for m, m' >= 0 only
  const double cb = std::cos(beta), ch = std::cos(beta / 2), sh = std::sin(beta / 2);
  std::vector<double> cp(p + 1), cm(p + 1);
  for (int mp = 0; mp <= p; ++mp)
    for (int m = 0; m <= p; ++m) {
      small_d_column(p, m, mp, cb, ch, sh, cp.data());
      if (m > 0) small_d_column(p, -m, mp, cb, ch, sh, cm.data());
      const double sg = (m & 1) ? -1.0 : 1.0;
      for (int n = std::max(m, mp); n <= p; ++n) {
        double* C = out + wigner_block_offset(n);
        double* S = C + (size_t)(n + 1) * (n + 1);
        C[m * (n + 1) + mp] = m > 0 ? cp[n] + sg * cm[n] : cp[n];  // column-major: consecutive m' contiguous
        if (m > 0 && mp > 0) S[(m - 1) * n + (mp - 1)] = cp[n] - sg * cm[n];
      }
    }
}

void singular_weights(int pq, std::vector<double>& out) {
  std::vector<double> t, w;
  gauss_legendre(pq + 1, t, w);
  out.assign(pq + 1, 0.0);
  for (int j = 0; j <= pq; ++j) {
    ld x = t[j];
    ld p0 = 1, p1 = x, sum = 1 + (pq >= 1 ? x : 0);
    for (int n = 1; n < pq; ++n) {
      ld p2 = ((2 * n + 1) * x * p1 - n * p0) / (n + 1);
      p0 = p1;
      p1 = p2;
      sum += p2;
    }
    ld half = std::sqrt((1 - x) / 2);  // sin(theta_j / 2)
    out[j] = (double)(kPi / (pq + 1) * (ld)w[j] * 2 * half * sum);
  }
}

}  // namespace bie
