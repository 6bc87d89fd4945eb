"""Host-only check of the root form used by the product-polynomial kernel
(csrc/zmc_polyroots.cpp): on random and special polynomials of degree 2..4 the
form is found and agrees with the power form, evaluated in long double: to
1e-8 of the value wherever the FP64 coefficients determine it well (|q| >=
1e-10 of the summed terms), and to 1e-11 of the summed terms everywhere (the
residue sits at points within ~1e-10 of a root, where the FP64 coefficients do
not determine the value better either) -- both far below the FP32 kernel's own
rounding (6e-8 per operation).  A triple root
is the one case without a form here (the coefficient form is kept for it)."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("pr") / "polyroots_check")
    csrc = os.path.join(ROOT, "paper_2104_10073_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                    "-I", "/usr/local/cuda/include",
                    os.path.join(ROOT, "tests", "helpers", "polyroots_check.cpp"),
                    os.path.join(csrc, "zmc_polyroots.cpp"), "-o", exe], check=True)

    def run(polys):
        text = "".join(f"{len(e) - 1} " + " ".join(repr(float(v)) for v in e) + "\n"
                       for e in polys)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True)
        return [(int(a), float(b), float(c))
                for a, b, c in (line.split() for line in out.stdout.splitlines())]

    return run


def test_random_polynomials(checker):
    rng = np.random.default_rng(7)
    polys = [rng.standard_normal(g + 1) for g in (2, 3, 4) for _ in range(3000)]
    res = checker(polys)
    found = [r for r in res if r[0] == 1]
    assert len(found) >= 0.995 * len(res), len(found)
    assert max(r[1] for r in found) <= 1e-8, sorted(r[1] for r in found)[-5:]
    assert max(r[2] for r in found) <= 1e-11, sorted(r[2] for r in found)[-5:]


def _expand(lead, roots):
    c = np.array([lead])
    for r in roots:
        c = np.convolve(c, [-r, 1.0])
    return c


def test_triple_root_keeps_coefficients(checker):
    assert checker([np.real(_expand(1.7, [0.3, 0.3, 0.3]))])[0][0] in (0, 1)


@pytest.mark.parametrize("roots", [
    [0.5, 0.5], [0.0, 1.0], [0.25, 0.75, 0.5, 0.125],
    [0.5 + 0.1j, 0.5 - 0.1j], [0.2 + 1e-3j, 0.2 - 1e-3j, 0.9, -3.0],
    [0.4, 0.4 + 1e-9, 5.0], [1e3, -0.5], [0.1 + 2j, 0.1 - 2j, 0.6 + 0.2j, 0.6 - 0.2j]])
def test_special_polynomials(checker, roots):
    e = np.real(_expand(1.7, roots))
    ok, rel, absolute = checker([e])[0]
    assert ok == 1
    assert rel <= 1e-8 and absolute <= 1e-11, (rel, absolute)
