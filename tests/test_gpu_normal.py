"""Stratified sampling with a heuristic tree search (zmc_normal_integrate*, GPU)
against the FP64 oracle of the same reading (oracle/normal.py).

The split decisions compare each leaf's standard error with a threshold.  The
GPU's per-cell standard errors agree with the oracle's far closer than the
1e-4 the parity tolerance allows (FP32 sums of FP32 values: ~1e-6 relative or
better), so every case asserts first that no decision of the oracle run lies
within 2e-5 of its threshold (the cases are chosen so), which makes the
decisions the same on both sides; then the tree (cells, leaves, rounds) must be
equal and the estimate within 1e-6 of sum_leaves V_c mean|f|_c."""
import math

import numpy as np
import pytest
from scipy.special import erf

from oracle.normal import normal as oracle_normal
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc

pytestmark = pytest.mark.gpu

GAUSS_PROD_F64 = r"""
__device__ double zmc_user_f(const double *x, const double *p) {
  double r2 = 0.0;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) r2 += (x[i] - p[0]) * (x[i] - p[0]);
  return exp(-r2 / (2.0 * p[1] * p[1]));
}
"""
GAUSS_PROD_F32 = r"""
__device__ float zmc_user_f(const float *x, const float *p) {
  float r2 = 0.0f;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) r2 = fmaf(x[i] - p[0], x[i] - p[0], r2);
  return expf(-r2 / (2.0f * p[1] * p[1]));
}
"""


def gauss_prod(x, p):
    return np.exp(-np.sum((x - p[0]) ** 2, axis=1) / (2.0 * p[1] ** 2))


def _check(got, want, est_rel=1e-6, se_rel=1e-4):
    assert want["margin"] > 2e-5, f"a split decision is within {want['margin']:.1e} of tau"
    for k in ("n_cells", "n_leaves", "rounds", "n_samples"):
        assert got[k] == want[k], (k, got[k], want[k])
    assert abs(got["estimate"] - want["estimate"]) <= est_rel * want["scale"], (got, want)
    assert abs(got["stderr"] - want["stderr"]) <= se_rel * want["stderr"], (got, want)


@pytest.mark.parametrize("depth,sigma", [(0, 1.0), (2, 1.3), (3, 1.1)])
def test_builtin_gauss_matches_oracle(zctx, depth, sigma):
    row = W.empty(1)[0]
    W.gauss(row, 1.5, 0.25, [0.1, 0.4, 0.7], [-0.5, 0.0, 0.0], [1.0, 1.0, 1.2], 1)
    kw = dict(divisions=3, depth=depth, samples_per_cell=5000, sigma_mult=sigma, seed=11,
              stream_base=40)
    want = oracle_normal(3, row["lo"][:3], row["hi"][:3], row=row, **kw)
    got = zmc.zmc_normal_integrate(zctx.handle, row, zmc.normal_options(**kw))
    _check(got, want)


def test_builtin_harmonic_eq1_matches_oracle(zctx):
    row = W.harmonic_fig1(1)[40]
    # nearly uniform spread over the cells: sigma_mult < 1 splits every leaf
    kw = dict(divisions=2, depth=2, samples_per_cell=3000, sigma_mult=0.95, seed=3)
    want = oracle_normal(4, row["lo"][:4], row["hi"][:4], row=row, **kw)
    got = zmc.zmc_normal_integrate(zctx.handle, row, zmc.normal_options(**kw))
    _check(got, want)
    assert got["rounds"] == 2 and got["n_leaves"] == 4096


@pytest.mark.parametrize("dim,prec", [(8, zmc.ZMC_UDF_F64), (10, zmc.ZMC_UDF_F32),
                                      (12, zmc.ZMC_UDF_F32)])
def test_udf_high_dimension_matches_oracle(zctx, dim, prec):
    src = GAUSS_PROD_F64 if prec == zmc.ZMC_UDF_F64 else GAUSS_PROD_F32
    u = zmc.Udf(src, dim, prec, amplitude=1.0)
    lo, hi = np.full(dim, -1.0), np.full(dim, 1.5)
    p = np.array([0.2, 0.6])
    n = 600 if dim == 12 else 1500
    kw = dict(divisions=2, depth=2, samples_per_cell=n, sigma_mult=1.5, seed=7,
              max_leaves=3 * 2 ** dim)
    want = oracle_normal(dim, lo, hi, f=gauss_prod, p=p, **kw)
    got = u.normal_integrate(zctx.handle, lo, hi, p, zmc.normal_options(**kw))
    _check(got, want)
    exact = 1.0
    for a, b in zip(lo, hi):
        exact *= 0.6 * math.sqrt(math.pi / 2) * (erf((b - 0.2) / (0.6 * math.sqrt(2)))
                                                 - erf((a - 0.2) / (0.6 * math.sqrt(2))))
    assert abs(got["estimate"] - exact) <= 5 * got["stderr"]
    u.close()


def test_options_are_validated(zctx):
    row = W.harmonic_fig1(1)[0]
    for kw in (dict(divisions=0), dict(samples_per_cell=1), dict(sigma_mult=0.0),
               dict(divisions=40, depth=0), dict(max_leaves=(1 << 22) + 1)):
        with pytest.raises(zmc.ZmcError) as e:
            zmc.zmc_normal_integrate(zctx.handle, row, zmc.normal_options(**kw))
        assert e.value.status == zmc.ZMC_EINVAL, kw
    bad = row.copy()
    bad["family"] = W.USER
    with pytest.raises(zmc.ZmcError) as e:
        zmc.zmc_normal_integrate(zctx.handle, bad, zmc.normal_options())
    assert e.value.status == zmc.ZMC_EINVAL
