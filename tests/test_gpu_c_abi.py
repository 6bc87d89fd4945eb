"""The C ABI used from plain C: a C99 program compiled against include/zmc.h and
linked with libzmc.so integrates the Fig. 1 set (Eq. 1) through zmc_integrate
and zmc_submit / zmc_poll; its output must match the FP64 oracle and the closed
form, and the two calls must agree bit for bit."""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import build
from paper_2104_10073_gb300 import workloads as W
from tests import closed_forms as CF
from tests import gpu_common as G

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_fig1(tmp_path):
    lib = build.build()
    exe = str(tmp_path / "c_abi_fig1")
    subprocess.run(["gcc", "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "helpers", "c_abi_fig1.c"),
                    "-L", os.path.dirname(lib), "-lzmc", "-Wl,-rpath," + os.path.dirname(lib),
                    "-lm", "-o", exe], check=True)
    out = subprocess.run([exe, "100000"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    rows = np.array([[float(v) for v in line.split()] for line in out.stdout.splitlines()])
    assert rows.shape == (100, 4)
    t = W.harmonic_fig1(10**5)
    got = np.zeros(100, dtype=[("estimate", "f8"), ("stderr", "f8"), ("n", "u8"),
                               ("status", "i4")])
    got["estimate"], got["stderr"], got["n"] = rows[:, 1], rows[:, 2], 10**5
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)
    assert np.array_equal(rows[:, 1], rows[:, 3])
    for i in range(100):
        assert abs(rows[i, 1] - CF.exact(t[i])) <= 5 * rows[i, 2] + 1e-12
