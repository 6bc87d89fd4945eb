// zmc_polyroots.cpp -- the root form of a real polynomial of degree <= 4, used to
// evaluate the product-polynomial family without cancellation.
//
// A factor q(u) = sum_k e_k u^k evaluated by Horner in FP32 loses relative
// accuracy wherever q is small against the terms it sums (near a root inside
// the box), by the factor sum_k |e_k u^k| / |q(u)|.  Written as
//     q(u) = lead * prod (u - r) * prod ((u - a)^2 + b^2)
// over its real roots r and complex pairs a +- ib, every factor is a difference
// with u (exact near its root by Sterbenz's lemma when r is split hi + lo) or a
// sum of non-negative terms, so the relative error stays at a few units in the
// last place everywhere.  The roots are found here in FP64 on the host:
//   1. real roots by isolation: the real roots of q' (recursively) cut the
//      line into intervals on which q is monotonic; each interval whose ends
//      differ in sign holds one root, found by bisection and polished by
//      Newton's method; a critical point where q vanishes (to rounding) is a
//      double root;
//   2. deflation by the real roots (synthetic division) leaves a polynomial
//      without real roots, of degree 0, 2 or 4: degree 2 gives a = -m1 / 2,
//      b^2 = m0 - a^2; degree 4 is split into two quadratics from its complex
//      roots (Aberth-Ehrlich iteration);
//   3. the form is verified by expanding it back: every coefficient within
//      1e-12 sum_k |e_k| of the original, else the caller keeps Horner.
#include <cmath>
#include <complex>
#include <cstring>

#include "zmc_runtime.h"

namespace zmc {
namespace {

// value and derivative of a monic-or-not polynomial c_0..c_g at x
inline double peval(const double *c, int g, double x) {
  double s = c[g];
  for (int k = g - 1; k >= 0; --k) s = s * x + c[k];
  return s;
}

inline double pabs(const double *c, int g, double x) {
  double s = std::fabs(c[g]);
  const double ax = std::fabs(x);
  for (int k = g - 1; k >= 0; --k) s = s * ax + std::fabs(c[k]);
  return s;
}

// Real roots of c_0..c_g (c_g != 0), ascending, into out; returns their count.
int real_roots(const double *c, int g, double *out) {
  if (g == 1) {
    out[0] = -c[0] / c[1];
    return 1;
  }
  double bound = 0.0;
  for (int k = 0; k < g; ++k) bound = std::max(bound, std::fabs(c[k] / c[g]));
  bound = 1.0 + bound;  // Cauchy: every root has |x| < bound
  // critical points: real roots of the derivative
  double d[4], crit[4];
  for (int k = 1; k <= g; ++k) d[k - 1] = k * c[k];
  const int nc = real_roots(d, g - 1, crit);
  double ends[6];
  int ne = 0;
  ends[ne++] = -bound;
  for (int k = 0; k < nc; ++k)
    if (crit[k] > -bound && crit[k] < bound) ends[ne++] = crit[k];
  ends[ne++] = bound;
  int n = 0;
  for (int k = 0; k + 1 < ne; ++k) {
    double lo = ends[k], hi = ends[k + 1];
    if (!(lo < hi)) continue;
    double flo = peval(c, g, lo), fhi = peval(c, g, hi);
    const bool touch_lo = k > 0 && std::fabs(flo) <= 1e-14 * pabs(c, g, lo);
    if (touch_lo) {
      // q vanishes at a critical point: a double root there (once)
      if (n == 0 || out[n - 1] != lo) {
        out[n++] = lo;
        out[n++] = lo;
      }
      continue;
    }
    if (flo == 0.0) {
      out[n++] = lo;
      continue;
    }
    if ((flo < 0.0) == (fhi < 0.0)) continue;
    // bisection to a small bracket, then Newton inside it
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo)); ++it) {
      const double mid = 0.5 * (lo + hi);
      const double fm = peval(c, g, mid);
      if (fm == 0.0) {
        lo = hi = mid;
        break;
      }
      if ((fm < 0.0) == (flo < 0.0)) {
        lo = mid;
        flo = fm;
      } else {
        hi = mid;
      }
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 3; ++it) {
      double dv = 0.0;
      const double v = peval(c, g, x);
      for (int j = g; j >= 1; --j) dv = dv * x + j * c[j];
      if (dv == 0.0) break;
      const double nx = x - v / dv;
      if (!(nx >= lo && nx <= hi)) break;
      x = nx;
    }
    out[n++] = x;
  }
  return n > g ? g : n;
}

// The two quadratic factors (u - a)^2 + b2 of a monic quartic without real
// roots (m_0..m_3), from its complex roots.
bool quartic_pairs(const double *m, double *a, double *b2) {
  using C = std::complex<double>;
  C z[4];
  double bound = 0.0;
  for (int k = 0; k < 4; ++k) bound = std::max(bound, std::fabs(m[k]));
  const double r = std::pow(1.0 + bound, 0.25);
  for (int k = 0; k < 4; ++k) z[k] = std::polar(r, 0.4 + k * 1.5707963267948966);
  for (int it = 0; it < 200; ++it) {
    double step = 0.0;
    for (int k = 0; k < 4; ++k) {
      C p = 1.0, dp = 0.0;
      for (int j = 3; j >= 0; --j) {
        dp = dp * z[k] + p;
        p = p * z[k] + m[j];
      }
      if (std::abs(dp) == 0.0) continue;
      const C ratio = p / dp;
      C sum = 0.0;
      for (int j = 0; j < 4; ++j)
        if (j != k) sum += 1.0 / (z[k] - z[j]);
      const C w = ratio / (1.0 - ratio * sum);
      z[k] -= w;
      step = std::max(step, std::abs(w) / std::max(1.0, std::abs(z[k])));
    }
    if (step < 1e-16) break;
  }
  // pair each root of positive imaginary part with its conjugate
  int np = 0;
  for (int k = 0; k < 4; ++k)
    if (z[k].imag() > 0.0) {
      if (np == 2) return false;
      a[np] = z[k].real();
      b2[np] = z[k].imag() * z[k].imag();
      ++np;
    }
  return np == 2;
}

}  // namespace

bool poly_root_form(const double *e_in, int g, RootForm *out) {
  std::memset(out, 0, sizeof *out);
  if (g < 0 || g > 4) return false;
  double e[5] = {0, 0, 0, 0, 0};
  for (int k = 0; k <= g; ++k) e[k] = e_in[k];
  while (g > 0 && e[g] == 0.0) --g;
  out->lead = e[g];
  if (g == 0 || e[g] == 0.0) return true;  // a constant (possibly zero)
  double m[5] = {0, 0, 0, 0, 0};
  for (int k = 0; k <= g; ++k) m[k] = e[k] / e[g];
  double roots[4];
  const int nr = real_roots(m, g, roots);
  // deflate: divide the monic polynomial by (u - r) for each real root
  double q[5];
  int gq = g;
  for (int k = 0; k <= g; ++k) q[k] = m[k];
  for (int j = 0; j < nr; ++j) {
    double carry = q[gq];
    double nq[5];
    nq[gq - 1] = carry;
    for (int k = gq - 1; k >= 1; --k) {
      carry = q[k] + carry * roots[j];
      nq[k - 1] = carry;
    }
    --gq;
    for (int k = 0; k <= gq; ++k) q[k] = nq[k];
    q[gq] = 1.0;
  }
  int s = 0;
  for (int j = 0; j < nr; ++j) {
    out->type[s] = 1;
    out->v[s++] = roots[j];
  }
  if (gq == 2) {
    const double a = -0.5 * q[1];
    const double b2 = q[0] - a * a;
    if (!(b2 > 0.0)) return false;
    out->type[s] = 2;
    out->v[s++] = a;
    out->type[s] = 3;
    out->v[s++] = b2;
  } else if (gq == 4) {
    double a[2], b2[2];
    if (!quartic_pairs(q, a, b2)) return false;
    for (int p = 0; p < 2; ++p) {
      out->type[s] = 2;
      out->v[s++] = a[p];
      out->type[s] = 3;
      out->v[s++] = b2[p];
    }
  } else if (gq != 0) {
    return false;
  }
  out->n = s;
  // verify: expand lead * prod(factors) and compare with e
  double c[5] = {1.0, 0, 0, 0, 0};
  int gc = 0;
  for (int k = 0; k < s; ++k) {
    if (out->type[k] == 1) {  // times (u - r)
      for (int j = gc + 1; j >= 0; --j) c[j] = (j > 0 ? c[j - 1] : 0.0) - out->v[k] * c[j];
      ++gc;
    } else if (out->type[k] == 2) {  // times (u^2 - 2a u + a^2 + b2)
      const double a = out->v[k], b2 = out->v[k + 1];
      const double c1 = -2.0 * a, c0 = a * a + b2;
      double nc[5] = {0, 0, 0, 0, 0};
      for (int j = 0; j <= gc; ++j) {
        nc[j + 2] += c[j];
        nc[j + 1] += c1 * c[j];
        nc[j] += c0 * c[j];
      }
      gc += 2;
      for (int j = 0; j <= gc; ++j) c[j] = nc[j];
    }
  }
  if (gc != g) return false;
  double scale = 0.0;
  for (int k = 0; k <= g; ++k) scale += std::fabs(e[k]);
  for (int k = 0; k <= g; ++k)
    if (!(std::fabs(out->lead * c[k] - e[k]) <= 1e-12 * scale)) return false;
  return true;
}

}  // namespace zmc
