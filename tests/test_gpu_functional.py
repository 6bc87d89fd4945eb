"""Functional mode: one integrand form over a parameter lattice (GPU)."""
import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import closed_forms as CF
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


def _expand(base, slots, values, independent):
    t = np.repeat(base.reshape(1), len(values))
    for q, row in enumerate(values):
        for s, v in zip(slots, row):
            if s < 40:
                t[q]["p"][s] = v
            elif s < 47:
                t[q]["lo"][s - 40] = v
            else:
                t[q]["hi"][s - 47] = v
        if independent:
            t[q]["stream_id"] = int(base["stream_id"]) + q
    return t


@pytest.mark.parametrize("independent", [True, False])
def test_functional_equals_expanded_table(zctx, independent):
    base = W.empty(1)[0]
    W.harmonic(base, 1.0, 0.5, [2.0, -1.0, 3.0], [0.0, -0.5, 0.2], [1.0, 0.7, 1.1], 40000,
               seed=7, stream_id=100)
    kk = np.linspace(-12.0, 12.0, 61)
    hi2 = np.linspace(0.5, 2.0, 61)
    values = np.stack([kk, hi2], axis=1)
    slots = [zmc.slot_p(2), zmc.slot_hi(2)]
    got = zmc.zmc_integrate_functional(zctx.handle, base, slots, values, independent)
    table = _expand(base, slots, values, independent)
    ref = zmc.zmc_integrate(zctx.handle, table)
    assert np.array_equal(got["estimate"], ref["estimate"])
    want, _ = oracle.integrate(table)
    G.compare(table, got, want)
    for q in range(0, 61, 10):
        assert abs(got["estimate"][q] - CF.exact(table[q])) <= 5 * got["stderr"][q]


def test_common_random_numbers_give_smooth_differences(zctx):
    """With one stream for every point, neighbouring points share their samples:
    the difference of two close parameter points has far less noise than with
    independent streams."""
    base = W.empty(1)[0]
    W.gauss(base, 1.0, 0.3, [0.1, 0.2], [-0.5, -0.5], [1.0, 1.0], 20000, seed=3, stream_id=5)
    sig = np.array([[0.30], [0.301]])
    crn = zmc.zmc_integrate_functional(zctx.handle, base, [zmc.slot_p(1)], sig, False)
    ind = zmc.zmc_integrate_functional(zctx.handle, base, [zmc.slot_p(1)], sig, True)
    t = _expand(base, [1], sig, False)
    exact_diff = CF.exact(t[1]) - CF.exact(t[0])
    assert abs((crn["estimate"][1] - crn["estimate"][0]) - exact_diff) < 0.1 * crn["stderr"][0]
    assert abs(ind["estimate"][1] - ind["estimate"][0]) > 0.0


def test_functional_rejects_bad_slots(zctx):
    base = W.harmonic_fig1(1000)[0]
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_integrate_functional(zctx.handle, base, [54], [[1.0]])
    assert e.value.status == zmc.ZMC_EINVAL
