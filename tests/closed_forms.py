"""Exact integrals of the four integrand families over a box (test helpers).

These are the analytic values the paper compares its Monte Carlo estimates to
(Fig. 1 caption: estimates against the analytical results), derived here in
closed form, independent of any sampling:

* HARMONIC (Eq. 1): the integral of exp(i k.x) over a box factorises,
  prod_i (exp(i k_i h_i) - exp(i k_i l_i)) / (i k_i) (or h_i - l_i when
  k_i = 0); a cos + b sin integrates to a Re + b Im of that product.
* ABSLIN (Eq. 2): for g(s) = |s| the k-fold antiderivative is
  G_k(s) = s^k |s| / (k+1)!, so with all c_i != 0,
  int_box |c.x| dx = (1/prod c_i) sum_{corners v} (prod_i sigma_i) G_d(c.v),
  sigma_i = +1 at h_i and -1 at l_i.  Dimensions with c_i = 0 contribute a
  factor h_i - l_i.  Evaluated in exact rational arithmetic.
* GAUSS: separable; each factor is sigma sqrt(pi/2) [erf((h-mu)/(sigma
  sqrt 2)) - erf((l-mu)/(sigma sqrt 2))].
* POLY: separable; each factor is sum_j c_j (h^{j+1} - l^{j+1}) / (j+1),
  exact in rationals.

``second_moment`` gives the integral of f^2 the same way, so the true
standard deviation of f over the box, and with it the spread a correct
estimator must show, is known exactly too.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import mpmath

mpmath.mp.dps = 40


def _box(row):
    d = int(row["dim"])
    return d, [float(v) for v in row["lo"][:d]], [float(v) for v in row["hi"][:d]]


def volume(row) -> float:
    d, lo, hi = _box(row)
    v = Fraction(1)
    for i in range(d):
        v *= Fraction(hi[i]) - Fraction(lo[i])
    return float(v)


def _expj_box(k, lo, hi):
    """int_box exp(i k.x) dx as an mpmath complex."""
    prod = mpmath.mpc(1)
    for ki, l, h in zip(k, lo, hi):
        ki, l, h = mpmath.mpf(ki), mpmath.mpf(l), mpmath.mpf(h)
        if ki == 0:
            prod *= h - l
        else:
            prod *= (mpmath.expj(ki * h) - mpmath.expj(ki * l)) / (1j * ki)
    return prod


def harmonic(row) -> float:
    d, lo, hi = _box(row)
    a, b = mpmath.mpf(float(row["p"][0])), mpmath.mpf(float(row["p"][1]))
    prod = _expj_box([float(v) for v in row["p"][2 : 2 + d]], lo, hi)
    return float(a * prod.real + b * prod.imag)


def abslin(row) -> float:
    d, lo, hi = _box(row)
    a = Fraction(float(row["p"][0]))
    c = [Fraction(float(v)) for v in row["p"][1 : 1 + d]]
    factor = Fraction(1)
    keep = []
    for i in range(d):
        if c[i] == 0:
            factor *= Fraction(hi[i]) - Fraction(lo[i])
        else:
            keep.append(i)
    m = len(keep)
    if m == 0:
        return 0.0
    total = Fraction(0)
    for corner in itertools.product((0, 1), repeat=m):
        s = Fraction(0)
        sign = 1
        for bit, i in zip(corner, keep):
            s += c[i] * (Fraction(hi[i]) if bit else Fraction(lo[i]))
            sign *= 1 if bit else -1
        total += sign * s**m * abs(s)
    prod_c = Fraction(1)
    for i in keep:
        prod_c *= c[i]
    return float(a * factor * total / (prod_c * math.factorial(m + 1)))


def _gauss_value(amp, sigma, mu, lo, hi):
    val = mpmath.mpf(amp)
    sigma = mpmath.mpf(sigma)
    s2 = sigma * mpmath.sqrt(2)
    for m, l, h in zip(mu, lo, hi):
        m = mpmath.mpf(m)
        val *= sigma * mpmath.sqrt(mpmath.pi / 2) * (
            mpmath.erf((mpmath.mpf(h) - m) / s2) - mpmath.erf((mpmath.mpf(l) - m) / s2))
    return val


def gauss(row) -> float:
    d, lo, hi = _box(row)
    return float(_gauss_value(float(row["p"][0]), float(row["p"][1]),
                              [float(v) for v in row["p"][2 : 2 + d]], lo, hi))


def _poly_coefs(row):
    d = int(row["dim"])
    deg = int(row["deg"])
    return [[Fraction(float(row["p"][5 * i + j])) for j in range(deg + 1)] for i in range(d)]


def _poly_box(coefs, lo, hi):
    val = Fraction(1)
    for cs, l, h in zip(coefs, lo, hi):
        l, h = Fraction(l), Fraction(h)
        val *= sum(c * (h ** (j + 1) - l ** (j + 1)) / (j + 1) for j, c in enumerate(cs))
    return val


def poly(row) -> float:
    d, lo, hi = _box(row)
    return float(_poly_box(_poly_coefs(row), lo, hi))


def exact(row) -> float:
    return (harmonic, abslin, gauss, poly)[int(row["family"])](row)


def second_moment(row) -> float:
    """int_box f(x)^2 dx, exactly."""
    fam = int(row["family"])
    d, lo, hi = _box(row)
    if fam == 0:
        a, b = mpmath.mpf(float(row["p"][0])), mpmath.mpf(float(row["p"][1]))
        k2 = [2.0 * float(v) for v in row["p"][2 : 2 + d]]
        p2 = _expj_box(k2, lo, hi)
        vol = mpmath.mpf(volume(row))
        # f^2 = (a^2+b^2)/2 + (a^2-b^2)/2 cos(2 k.x) + a b sin(2 k.x)
        return float((a * a + b * b) / 2 * vol + (a * a - b * b) / 2 * p2.real + a * b * p2.imag)
    if fam == 1:
        a = Fraction(float(row["p"][0]))
        c = [Fraction(float(v)) for v in row["p"][1 : 1 + d]]
        L = [Fraction(v) for v in lo]
        H = [Fraction(v) for v in hi]
        w = [H[i] - L[i] for i in range(d)]
        m1 = [(H[i] ** 2 - L[i] ** 2) / 2 for i in range(d)]
        m2 = [(H[i] ** 3 - L[i] ** 3) / 3 for i in range(d)]
        total = Fraction(0)
        for i in range(d):
            for j in range(d):
                term = c[i] * c[j]
                for t in range(d):
                    if i == j == t:
                        term *= m2[t]
                    elif t == i or t == j:
                        term *= m1[t]
                    else:
                        term *= w[t]
                total += term
        return float(a * a * total)
    if fam == 2:
        amp, sigma = float(row["p"][0]), float(row["p"][1])
        return float(_gauss_value(amp * amp, sigma / math.sqrt(2.0),
                                  [float(v) for v in row["p"][2 : 2 + d]], lo, hi))
    coefs = _poly_coefs(row)
    sq = []
    for cs in coefs:
        out = [Fraction(0)] * (2 * len(cs) - 1)
        for j1, c1 in enumerate(cs):
            for j2, c2 in enumerate(cs):
                out[j1 + j2] += c1 * c2
        sq.append(out)
    return float(_poly_box(sq, lo, hi))


def sigma_f(row) -> float:
    """Standard deviation of f(x) for x uniform on the box."""
    v = volume(row)
    m1 = exact(row) / v
    m2 = second_moment(row) / v
    return math.sqrt(max(m2 - m1 * m1, 0.0))


def fig1_closed_form(n: int) -> float:
    """Integral of cos(k.x) + sin(k.x) over [0,1]^4 with k = (n+50)/(2 pi) (1,1,1,1).

    Each factor is (e^{i kappa} - 1)/(i kappa) = e^{i kappa/2} sinc(kappa/2), so the
    product is (sin(kappa/2)/(kappa/2))^4 e^{2 i kappa}: the value is
    (sin(kappa/2)/(kappa/2))^4 (cos 2 kappa + sin 2 kappa).
    """
    kappa = (n + 50) / (2.0 * math.pi)
    s = math.sin(kappa / 2) / (kappa / 2)
    return s**4 * (math.cos(2 * kappa) + math.sin(2 * kappa))
