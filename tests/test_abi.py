"""The C ABI library loads, exports what include/zmc.h declares, and validates
descriptors on the host (CPU only: no compute call needs a GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2104_10073_gb300 import build, zmc
from paper_2104_10073_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return zmc.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "zmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zmc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("zmc_create", "zmc_integrate", "zmc_submit", "zmc_poll", "zmc_destroy",
                     "zmc_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in zmc.EXPORTED, f"binding does not wrap {name}"


def test_struct_sizes(lib):
    assert lib.zmc_desc_size() == 464 == W.DESC_DTYPE.itemsize
    assert lib.zmc_result_size() == 32 == zmc.RESULT_DTYPE.itemsize
    assert ctypes.sizeof(zmc.zmc_options) == 72
    offs = {n: W.DESC_DTYPE.fields[n][1] for n in W.DESC_DTYPE.names}
    assert offs == {"family": 0, "dim": 4, "stream_id": 8, "deg": 12, "n_samples": 16,
                    "seed": 24, "lo": 32, "hi": 88, "p": 144}


def test_default_options(lib):
    o = zmc.zmc_default_options()
    assert o.mem_budget_bytes == 1 << 30 and o.quints_per_lane == 0 and o.device == 0


def _bad(mutator):
    t = W.harmonic_fig1(1000)[:3].copy()
    mutator(t[1])
    return zmc.zmc_validate(t)


@pytest.mark.parametrize("name,mut", [
    ("family", lambda r: r.__setitem__("family", 4)),
    ("dim0", lambda r: r.__setitem__("dim", 0)),
    ("dim8", lambda r: r.__setitem__("dim", 8)),
    ("nsamples0", lambda r: r.__setitem__("n_samples", 0)),
    ("lo_ge_hi", lambda r: r["lo"].__setitem__(2, 1.0)),
    ("nan_box", lambda r: r["hi"].__setitem__(0, np.nan)),
    ("inf_param", lambda r: r["p"].__setitem__(3, np.inf)),
    ("huge_phase", lambda r: r["p"].__setitem__(2, 1e9)),
    ("nsamples_above_2p62", lambda r: r.__setitem__("n_samples", 2**62 + 1)),
])
def test_validation_rejects(lib, name, mut):
    st, bad, msg = _bad(mut)
    assert st == zmc.ZMC_EINVAL and bad == 1, (name, st, bad, msg)
    assert msg


def test_validation_family_specific(lib):
    t = W.empty(2)
    W.gauss(t[0], 1.0, 0.0, [0.0], [0.0], [1.0], 10)
    W.poly(t[1], [[1.0, 2.0]], [0.0], [1.0], 10)
    st, bad, _ = zmc.zmc_validate(t)
    assert st == zmc.ZMC_EINVAL and bad == 0
    t[0]["p"][1] = 0.3
    t[1]["deg"] = 5
    st, bad, _ = zmc.zmc_validate(t)
    assert st == zmc.ZMC_EINVAL and bad == 1
    t[1]["deg"] = 1
    assert zmc.zmc_validate(t)[0] == zmc.ZMC_OK


def test_validation_accepts_abslin_at_any_scale(lib):
    """The abs-linear sum picks its fixed-point scale per integrand, for the
    64-bit sum (rows of < 256 samples) and the 32-bit one (>= 256); tiny, huge
    and mixed coefficient magnitudes, zero coefficients and boxes far from the
    origin are all valid for both."""
    for n in (10, 256, 10**6):
        for c in ([1e-20, -2e-20], [3e15, -1e15, 2e15], [1e8, 1e-8], [0.0, 1.0, 0.0],
                  [0.0, 0.0], [1e-300, 1.0], [1e30, -1e30]):
            for lo, hi in ((-1.0, 1.0), (1e6, 1e6 + 1.0)):
                t = W.empty(1)
                W.abslin(t[0], 1.0, c, [lo] * len(c), [hi] * len(c), n)
                st, bad, msg = zmc.zmc_validate(t)
                assert st == zmc.ZMC_OK, (n, c, lo, msg)


def test_validation_of_an_empty_table(lib):
    st, bad, _ = zmc.zmc_validate(W.empty(0))
    assert st == zmc.ZMC_OK and bad is None


def test_validation_accepts_paper_workloads(lib):
    for t in (W.harmonic_fig1(), W.abslin_eq2(), W.mixed(300)):
        assert zmc.zmc_validate(t)[0] == zmc.ZMC_OK


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_create()
    assert e.value.status == zmc.ZMC_ECUDA


def test_validation_reports_the_first_bad_row_of_a_large_table(lib):
    """Large tables are validated on several host threads; the reported row is
    still the first bad one, with its own message."""
    t = W.mixed(6000, gen_seed=3)
    t["dim"][4500] = 9
    t["n_samples"][3777] = 0
    t["lo"][5000][0] = t["hi"][5000][0]
    for _ in range(5):
        st, bad, msg = zmc.zmc_validate(t)
        assert st == zmc.ZMC_EINVAL and bad == 3777
        assert "3777" in msg and "n_samples" in msg
    t["n_samples"][3777] = 10
    st, bad, msg = zmc.zmc_validate(t)
    assert st == zmc.ZMC_EINVAL and bad == 4500 and "dim" in msg


def test_validation_rules_of_the_fp32_constants(lib):
    """The rules zmc.h lists beside zmc_desc for the derived FP32 constants: each
    is reported with its own reason."""
    def one(fill):
        t = W.empty(1)
        fill(t[0])
        return zmc.zmc_validate(t)

    # a harmonic span of more than 2^20 turns in one dimension
    st, _, msg = one(lambda r: W.harmonic(r, 1.0, 1.0, [2 * np.pi * 2**20 * 1.01], [0.0], [1.0], 10))
    assert st == zmc.ZMC_EINVAL and "2^20" in msg
    # just inside it is accepted
    st, _, _ = one(lambda r: W.harmonic(r, 1.0, 1.0, [2 * np.pi * 2**20 * 0.99], [0.0], [1.0], 10))
    assert st == zmc.ZMC_OK
    # a phase offset k.lo beyond 4e15 turns
    st, _, msg = one(lambda r: W.harmonic(r, 1.0, 1.0, [1.0], [1e17], [1e17 + 64.0], 10))
    assert st == zmc.ZMC_EINVAL and "phase" in msg
    # amplitudes whose scaled FP32 constants overflow (the scale stops at 2^-100)
    for fill in (lambda r: W.harmonic(r, 1e300, 0.0, [1.0], [0.0], [1.0], 10),
                 lambda r: W.gauss(r, 1e300, 0.5, [0.5], [0.0], [1.0], 10),
                 lambda r: W.abslin(r, 1e300, [1.0], [0.0], [1.0], 10),
                 lambda r: W.poly(r, [[1e300, 1.0]], [0.0], [1.0], 10)):
        st, _, msg = one(fill)
        assert st == zmc.ZMC_EINVAL and "range" in msg, msg
