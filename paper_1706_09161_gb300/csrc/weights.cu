// Host-side FP64 construction of the fractional-operator matrices K_mu.
//
// Section 2.4 (Eqs. 1Dminus_discret, c+, c-, XXminus_discret): along one lattice
// line with nodes n, l = 0..N,
//   I+^g f(n dx) ~ dx^g / Gamma(2+g) sum_{l<=n} f(l dx) c+_{ln}(g)
//   I-^g f(n dx) ~ dx^g / Gamma(2+g) sum_{l>=n} f(l dx) c-_{ln}(g, N)
// and the fractional term of Eq. (CoeffA_FADE3D) is p I+(gC) + (1-p) I-(gC).
// c+ and c- are Toeplitz apart from their end columns (l = 0 for c+, l = N for c-):
//   interior  a(k) = (k+1)^s - 2 k^s + (k-1)^s,  k = |n-l| >= 1, s = g+1
//   end       b(m) = (1+g) m^g - m^s + (m-1)^s,  m = n (c+) or N-n (c-)
//   diagonal  1, except at the line's own end: I+ at n = 0 and I- at n = N integrate
//             over an empty interval (Eqs. Def_FracInt, Def_FracIntspe), so that entry
//             is 0 for g > 0; at g = 0 (alpha = 2) I^0 is the identity and it stays 1.
// The Caputo-type variant (Section 3.5, Eqs. Fg2, PSRLdD-a/b, Fg22) subtracts the
// boundary terms p f(0) (n dx)^g / Gamma(1+g) and (1-p) f(N dx) ((N-n) dx)^g / Gamma(1+g),
// i.e. columns 0 and N of K change; 0^0 = 1 keeps constants in the kernel at g = 0 too.
// Both a(k) and b(m) are small differences of powers; for k, m >= 2 they are summed
// from their binomial series instead (x = 1/k <= 1/2, so the series converges at least
// like 4^-j), which keeps every entry within a few units in the last place (the direct
// form loses ~2 log10(k) digits, and all of them as alpha -> 2).
#include <cmath>
#include <vector>

#include "lbm_internal.h"

namespace lbm {
namespace {

// a(k) = k^s * [(1+x)^s + (1-x)^s - 2], x = 1/k
//      = 2 k^s * sum_{j>=1} binom(s, 2j) x^{2j}
double interior_coeff(double g, long k) {
  const double s = g + 1.0;
  if (k < 2) return 2.0 * std::expm1(g * std::log(2.0));  // k = 1: 2^s - 2, (k-1)^s = 0
  const double x2 = 1.0 / (static_cast<double>(k) * static_cast<double>(k));
  double binom = 1.0;  // binom(s, m), advanced two orders per term
  double xp = 1.0;
  double sum = 0.0;
  for (int j = 1; j < 200; ++j) {
    const int m = 2 * j;
    // s - (m-2) and s - (m-1) as g - (m-3) and g - (m-2): no rounding of s = g + 1 first
    binom *= (g - (m - 3)) / (m - 1);
    binom *= (g - (m - 2)) / m;
    xp *= x2;
    const double term = binom * xp;
    sum += term;
    if (std::fabs(term) <= 1e-18 * std::fabs(sum)) break;
  }
  return 2.0 * std::pow(static_cast<double>(k), s) * sum;
}

// b(m) = (1+g) m^g - [m^s - (m-1)^s] = m^s * sum_{j>=2} (-1)^j binom(s, j) m^{-j}
double end_coeff(double g, long m) {
  const double s = g + 1.0;
  if (m < 2) return g;  // m = 1: (1+g) - 1 + 0
  const double x = 1.0 / static_cast<double>(m);
  double binom = s;  // binom(s, 1)
  double xp = x;
  double sum = 0.0;
  for (int j = 2; j < 200; ++j) {
    binom *= (g - (j - 2)) / j;  // s - (j-1), exact in g
    xp *= x;
    const double term = ((j & 1) ? -1.0 : 1.0) * binom * xp;
    sum += term;
    if (std::fabs(term) <= 1e-18 * std::fabs(sum)) break;
  }
  return std::pow(static_cast<double>(m), s) * sum;
}

// Digamma psi(x) for x > 0: shift up with psi(x) = psi(x+1) - 1/x until x >= 16, then
// the asymptotic expansion psi(x) ~ ln x - 1/(2x) - sum_n B_2n / (2n x^(2n)), n = 1..6
// (Abramowitz & Stegun 6.3.5 and 6.3.18); the first omitted term is below 1e-17.
double digamma(double x) {
  double acc = 0.0;
  while (x < 16.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double r = 1.0 / (x * x);
  const double series =
      r * (1.0 / 12 - r * (1.0 / 120 - r * (1.0 / 252 - r * (1.0 / 240 - r * (1.0 / 132 - r * (691.0 / 32760))))));
  return acc + std::log(x) - 0.5 / x - series;
}

// d/ds of k^s, i.e. k^s ln k (0 at k = 0 and k = 1)
double pow_log(double k, double s) { return (k <= 1.0) ? 0.0 : std::pow(k, s) * std::log(k); }

}  // namespace

double digamma_fn(double x) { return digamma(x); }

// dK/dalpha and dK/dp of the matrix built by build_frac_matrix (same layout).
// With gamma = 2 - alpha and K = s(gamma) (p W+ + (1-p) W-):
//   dK/dp     = s (W+ - W-)
//   dK/dalpha = -[ s'(gamma) (p W+ + (1-p) W-) + s (p dW+/dgamma + (1-p) dW-/dgamma) ],
//   s'(gamma) = s (ln dx - psi(2+gamma)),
//   d a(k)/dgamma = (k+1)^s ln(k+1) - 2 k^s ln k + (k-1)^s ln(k-1),
//   d b(m)/dgamma = m^g + (1+g) m^g ln m - m^s ln m + (m-1)^s ln(m-1).
// The direct second differences lose ~2 log10(k) digits, far below the precision the
// gradients are used at.
void build_frac_matrix_grad(double alpha, double p, double scale_g, int side, double dx, int variant, double* dKda,
                            double* dKdp) {
  const double g = 2.0 - alpha;
  const double s = g + 1.0;
  const long N = side - 1;
  const double scale = scale_g * std::pow(dx, g) / std::tgamma(2.0 + g);
  const double dscale = scale * (std::log(dx) - digamma(2.0 + g));
  std::vector<double> a(side + 1, 0.0), b(side + 1, 0.0), da(side + 1, 0.0), db(side + 1, 0.0);
  for (long k = 1; k <= N; ++k) {
    a[k] = interior_coeff(g, k);
    const double kd = static_cast<double>(k);
    da[k] = pow_log(kd + 1.0, s) - 2.0 * pow_log(kd, s) + pow_log(kd - 1.0, s);
  }
  for (long m = 1; m <= N; ++m) {
    b[m] = end_coeff(g, m);
    const double md = static_cast<double>(m);
    db[m] = std::pow(md, g) + (1.0 + g) * std::pow(md, g) * std::log(md) - pow_log(md, s) + pow_log(md - 1.0, s);
  }
  for (long n = 0; n <= N; ++n) {
    for (long l = 0; l <= N; ++l) {
      double wp = 0.0, wm = 0.0, dwp = 0.0, dwm = 0.0;
      if (l == n) {
        wp = (n > 0 || g == 0.0) ? 1.0 : 0.0;
        wm = (n < N || g == 0.0) ? 1.0 : 0.0;
      } else if (l < n) {
        wp = (l == 0) ? b[n] : a[n - l];
        dwp = (l == 0) ? db[n] : da[n - l];
      } else {
        wm = (l == N) ? b[N - n] : a[l - n];
        dwm = (l == N) ? db[N - n] : da[l - n];
      }
      dKdp[n * side + l] = scale * (wp - wm);
      dKda[n * side + l] = -(dscale * (p * wp + (1.0 - p) * wm) + scale * (p * dwp + (1.0 - p) * dwm));
    }
  }
  if (variant) {
    // K~ = K - B, B = scale_g [p e_0 (n dx)^g + (1-p) e_N ((N-n) dx)^g] / Gamma(1+g):
    // dB/dp from the two weights, dB/dalpha = -dB/dg = -B (ln(x) - psi(1+g)) per entry
    const double den = std::tgamma(1.0 + g);
    const double psi = digamma(1.0 + g);
    for (long n = 0; n <= N; ++n) {
      const double xl = n * dx, xr = (N - n) * dx;
      const double tl = scale_g * std::pow(xl, g) / den, tr = scale_g * std::pow(xr, g) / den;
      const double dtl = (xl > 0.0) ? tl * (std::log(xl) - psi) : 0.0;
      const double dtr = (xr > 0.0) ? tr * (std::log(xr) - psi) : 0.0;
      dKdp[n * side] -= tl;
      dKdp[n * side + N] += tr;
      dKda[n * side] += p * dtl;
      dKda[n * side + N] += (1.0 - p) * dtr;
    }
  }
}

void build_frac_matrix(double alpha, double p, double scale_g, int side, double dx, int variant, double* K) {
  const double g = 2.0 - alpha;          // order of the fractional integral
  const double s = g + 1.0;
  const long N = side - 1;
  const double scale = scale_g * std::pow(dx, g) / std::tgamma(2.0 + g);
  std::vector<double> a(side + 1, 0.0), b(side + 1, 0.0);
  for (long k = 1; k <= N; ++k) a[k] = interior_coeff(g, k);
  for (long m = 1; m <= N; ++m) b[m] = end_coeff(g, m);
  for (long n = 0; n <= N; ++n) {
    for (long l = 0; l <= N; ++l) {
      double wp = 0.0, wm = 0.0;
      if (l == n) {
        wp = (n > 0 || g == 0.0) ? 1.0 : 0.0;
        wm = (n < N || g == 0.0) ? 1.0 : 0.0;
      } else if (l < n) {
        wp = (l == 0) ? b[n] : a[n - l];
      } else {
        wm = (l == N) ? b[N - n] : a[l - n];
      }
      K[n * side + l] = scale * (p * wp + (1.0 - p) * wm);
    }
  }
  if (variant) {
    const double den = std::tgamma(1.0 + g);
    for (long n = 0; n <= N; ++n) {
      K[n * side] -= scale_g * p * std::pow(n * dx, g) / den;
      K[n * side + N] -= scale_g * (1.0 - p) * std::pow((N - n) * dx, g) / den;
    }
  }
}

}  // namespace lbm
