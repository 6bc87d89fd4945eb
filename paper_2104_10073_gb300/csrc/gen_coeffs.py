"""Fit the FP32 polynomials the kernels evaluate instead of library calls.

* cos(2 pi t) on 0 <= t <= 1/4 (+2^-24) turn, degree 5 in z = t^2 (absolute
  error): the harmonic family reduces its fixed-point phase to |t| <= 1/4 turn
  by the symmetries of cosine and evaluates R cos(2 pi t).
* 2^x on |x| <= 0.51 (relative error), degree 6: the Gaussian family's
  2^-Z = 2^-n 2^-r after n = rint(Z).

Every fit is a Remez exchange carried out in 50-digit arithmetic, then rounded to
binary32.  The script prints the maximum error of the rounded polynomials
evaluated in FP64 on a dense grid and writes ``zmc_coeffs.h``.

Run from the repository root:  python paper_2104_10073_gb300/csrc/gen_coeffs.py
"""
import os

import mpmath
import numpy as np

mpmath.mp.dps = 50
def remez(target, weight, n_coef, a, b, iters=30):
    """Minimax polynomial p(z) = sum c_j z^j of weight(z) * (target(z) - p(z)) on [a, b]."""
    m = n_coef + 1
    # Chebyshev extrema as the first reference
    ref = [a + (b - a) * (1 - mpmath.cos(mpmath.pi * i / (m - 1))) / 2 for i in range(m)]
    coef = None
    for _ in range(iters):
        A = mpmath.matrix(m, m)
        rhs = mpmath.matrix(m, 1)
        for i, z in enumerate(ref):
            for j in range(n_coef):
                A[i, j] = z**j
            A[i, n_coef] = (-1) ** i / weight(z)
            rhs[i] = target(z)
        sol = mpmath.lu_solve(A, rhs)
        coef = [sol[j] for j in range(n_coef)]

        def err(z):
            return weight(z) * (target(z) - sum(c * z**j for j, c in enumerate(coef)))

        # new reference: extrema of the error on a fine grid, one per sign run
        grid = [a + (b - a) * (1 - mpmath.cos(mpmath.pi * i / 4000)) / 2 for i in range(4001)]
        vals = [err(z) for z in grid]
        runs = []
        start = 0
        for i in range(1, len(grid) + 1):
            if i == len(grid) or mpmath.sign(vals[i]) != mpmath.sign(vals[start]):
                best = max(range(start, i), key=lambda k: abs(vals[k]))
                runs.append(best)
                start = i
        if len(runs) < m:
            break
        # keep m alternating extrema with the largest magnitudes
        while len(runs) > m:
            if abs(vals[runs[0]]) < abs(vals[runs[-1]]):
                runs.pop(0)
            else:
                runs.pop()
        ref = [grid[k] for k in runs]
    return coef


def main():
    zq = (mpmath.mpf(1) / 4 + mpmath.mpf(2) ** -24) ** 2
    cq = remez(lambda z: mpmath.cos(2 * mpmath.pi * mpmath.sqrt(z)), lambda z: 1, 6,
               mpmath.mpf(0), zq)
    cq32 = [np.float32(float(v)) for v in cq]
    t = np.linspace(0, 0.25 + 2.0**-24, 200001)
    z = t * t
    pc = sum(float(v) * z**j for j, v in enumerate(cq32))
    ec = np.max(np.abs(pc - np.cos(2 * np.pi * t)))
    xm = mpmath.mpf("0.51")
    e2 = remez(lambda x: mpmath.power(2, x), lambda x: 1 / mpmath.power(2, x), 7, -xm, xm)
    e32 = [np.float32(float(v)) for v in e2]
    x = np.linspace(-0.51, 0.51, 200001)
    pe = sum(float(v) * x**j for j, v in enumerate(e32))
    ee = np.max(np.abs(pe / np.exp2(x) - 1))
    print(f"max |cos err| {ec:.3e}  max |exp2 rel err| {ee:.3e}")
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_coeffs.py: Remez fits rounded to binary32.  Max error of the",
        "// rounded polynomials in exact arithmetic:",
        f"//   cos(2 pi t), 0 <= t <= 1/4 (degree 5 in t^2): {ec:.2e} absolute",
        f"//   2^x, |x| <= 0.51, degree 6:       {ee:.2e} relative",
        "#pragma once",
    ]
    for j, v in enumerate(cq32):
        lines.append(f"#define ZMC_COSQ_C{j} {float(v).hex()}f  // {float(v):.9e}")
    for j, v in enumerate(e32):
        lines.append(f"#define ZMC_EXP2_C{j} {float(v).hex()}f  // {float(v):.9e}")
    with open(os.path.join(here, "zmc_coeffs.h"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
