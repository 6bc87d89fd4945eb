"""Fit the FP32 polynomials the kernels evaluate instead of library calls.

* sin(2 pi t) / t on |t| <= 1/4 turn, degree 4 in z = t^2 (relative error):
  the harmonic family writes cos(2 pi x) = sin(2 pi (1/4 - |x|)) for its
  fixed-point phase x in [-1/2, 1/2) turn and evaluates t (R P)(t^2), which
  keeps the relative accuracy near the zeros.  Degree 4 approximates to 5e-9,
  far below the rounding of its coefficients to binary32 (4e-8; degree 5:
  2e-11 and 5e-8), so a fifth term would only cost an FMA.

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
    zq = (mpmath.mpf(1) / 4) ** 2

    def sinc2(z):
        t = mpmath.sqrt(z)
        return 2 * mpmath.pi if t == 0 else mpmath.sin(2 * mpmath.pi * t) / t

    sq = remez(sinc2, lambda z: 1 / sinc2(z), 5, mpmath.mpf(0), zq)
    sq32 = [np.float32(float(v)) for v in sq]
    t = np.linspace(1e-6, 0.25, 200001)
    z = t * t
    ps = t * sum(float(v) * z**j for j, v in enumerate(sq32))
    es = np.max(np.abs(ps / np.sin(2 * np.pi * t) - 1))
    print(f"max |sin rel err| {es:.3e}")
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_coeffs.py: Remez fits rounded to binary32.  Max error of the",
        "// rounded polynomials in exact arithmetic:",
        f"//   sin(2 pi t), |t| <= 1/4 (t times degree 4 in t^2): {es:.2e} relative",
        "#pragma once",
    ]
    for j, v in enumerate(sq32):
        lines.append(f"#define ZMC_SINQ_C{j} {float(v).hex()}f  // {float(v):.9e}")
    with open(os.path.join(here, "zmc_coeffs.h"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
