"""The evaluation form the library picks per row (zmc_variant_of; CPU only):
the selection rules documented at zmc_variant_of in include/zmc.h."""
import numpy as np
import pytest

from paper_2104_10073_gb300 import build, zmc
from paper_2104_10073_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return zmc.lib()


def _form(fill):
    t = W.empty(1)
    fill(t[0])
    v = zmc.zmc_variant_of(t)[0]
    return int(v["family"]), int(v["dim"]), int(v["form"])


def test_harmonic_equal_rates():
    fig1 = zmc.zmc_variant_of(W.harmonic_fig1(1000))
    assert np.all(fig1["form"] == 1) and np.all(fig1["dim"] == 4) and np.all(fig1["family"] == 0)
    # the rates k_i (hi_i - lo_i) decide, not k alone: (2, 1) on widths (1, 2) is equal-rate
    assert _form(lambda r: W.harmonic(r, 1, 1, [2.0, 1.0], [0.0, -1.0], [1.0, 1.0], 10)) == (0, 2, 1)
    assert _form(lambda r: W.harmonic(r, 1, 1, [2.0, 2.0], [0.0, -1.0], [1.0, 1.0], 10)) == (0, 2, 0)
    # a rate stretched by 1e-9 takes the general phase
    t = W.harmonic_fig1(1000)[:1].copy()
    t["p"][0, 5] *= 1.0 + 1e-9
    assert int(zmc.zmc_variant_of(t)["form"][0]) == 0
    # one dimension has nothing to sum
    assert _form(lambda r: W.harmonic(r, 1, 1, [3.0], [0.0], [1.0], 10)) == (0, 1, 0)
    # negative and zero wave numbers, seven dimensions
    assert _form(lambda r: W.harmonic(r, 1, 0, [-5.0] * 7, [0.5] * 7, [1.0] * 7, 10)) == (0, 7, 1)
    assert _form(lambda r: W.harmonic(r, 1, 0, [0.0] * 3, [0.0] * 3, [1.0] * 3, 10)) == (0, 3, 1)


def test_abslin_sum_width_by_sample_count():
    for n, form in ((1, 0), (255, 0), (256, 1), (10**7, 1)):
        assert _form(lambda r: W.abslin(r, 1.0, [1.0, -1.0], [0.0, 0.0], [1.0, 1.0], n)) == \
            (1, 2, form)


def test_gauss_near_and_far():
    assert _form(lambda r: W.gauss(r, 1.0, 0.3, [0.5, 0.5], [0.0, 0.0], [1.0, 1.0], 10)) == (2, 2, 0)
    # mu two box widths above hi_0: outside [-1, 2] widths of lo
    assert _form(lambda r: W.gauss(r, 1.0, 0.3, [3.5, 0.5], [0.0, 0.0], [1.0, 1.0], 10)) == (2, 2, 1)


def test_poly_coefficient_and_root_forms():
    assert _form(lambda r: W.poly(r, [[2.0]], [0.0], [1.0], 10)) == (3, 1, 0)
    assert _form(lambda r: W.poly(r, [[1.0, 2.0]], [0.0], [1.0], 10)) == (3, 1, 1)
    # distinct real roots: root form, degree + 3
    assert _form(lambda r: W.poly(r, [[0.1, -1.0, 1.0]], [0.0], [1.0], 10)) == (3, 1, 5)
    assert _form(lambda r: W.poly(r, [[0.0, 1.0, -3.0, 2.0]], [0.0], [1.0], 10)) == (3, 1, 6)
    assert _form(lambda r: W.poly(r, [[1.0, 0.0, 0.0, 0.0, 1.0]], [0.0], [1.0], 10)) == (3, 1, 7)


def test_mixed_table_reaches_every_family_form_it_should():
    v = zmc.zmc_variant_of(W.mixed(2000))
    by_family = {f: set(v["form"][v["family"] == f].tolist()) for f in range(4)}
    assert by_family[0] == {0}  # random wave vectors: general phase
    assert by_family[1] == {1}  # every row has >= 10^4 samples
    assert 0 in by_family[2]
    assert {0, 1}.issubset(by_family[3]) and {5, 6, 7}.issubset(by_family[3])


def test_invalid_rows_are_reported():
    t = W.harmonic_fig1(10)[:3].copy()
    t[2]["dim"] = 9
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_variant_of(t)
    assert e.value.status == zmc.ZMC_EINVAL
    assert zmc.zmc_variant_of(W.empty(0)).shape == (0,)


def test_random_parity_tables_reach_every_form():
    """The seeded random tables of the GPU parity sweep (tests/test_gpu_fuzz.py),
    all together, reach every form the library has."""
    from tests.test_gpu_fuzz import table

    forms = set()
    for seed in range(10):
        v = zmc.zmc_variant_of(table(seed)[0])
        forms |= {(int(f), int(g)) for f, g in zip(v["family"], v["form"])}
    assert forms >= {(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1), (3, 2),
                     (3, 3), (3, 4), (3, 5), (3, 6), (3, 7)}, forms
