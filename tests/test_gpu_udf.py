"""User-defined integrands compiled at run time (GPU).

Two kinds of reference, both independent of the CUDA path:
* user forms of the built-in families (Eq. 1 harmonics, Gaussians) against the
  C oracle's own FP64 evaluation of those families on the same Philox samples;
* arbitrary functions against a plain FP64 numpy evaluation of the same formula
  at the oracle's sample points (oracle.samples), mean and M2 by their
  definitions.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_10073_gb300 import workloads as W
from paper_2104_10073_gb300 import zmc
from tests import gpu_common as G

pytestmark = pytest.mark.gpu

HARMONIC_F64 = r"""
__device__ double zmc_user_f(const double *x, const double *p) {
  double ph = 0.0;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) ph += p[2 + i] * x[i];
  return p[0] * cos(ph) + p[1] * sin(ph);
}
"""

HARMONIC_F32 = r"""
__device__ float zmc_user_f(const float *x, const float *p) {
  float ph = 0.0f;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) ph = fmaf(p[2 + i], x[i], ph);
  float s, c;
  sincosf(ph, &s, &c);
  return p[0] * c + p[1] * s;
}
"""

GAUSS_F32 = r"""
__device__ float zmc_user_f(const float *x, const float *p) {
  float r2 = 0.0f;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) {
    const float t = x[i] - p[2 + i];
    r2 = fmaf(t, t, r2);
  }
  return p[0] * expf(-r2 / (2.0f * p[1] * p[1]));
}
"""

# f(x) = p0 / (1 + sum_i p_{1+i} x_i^2) * (1 + p8 sin(x0 x1)): no built-in counterpart
RATIONAL_F64 = r"""
__device__ double zmc_user_f(const double *x, const double *p) {
  double q = 1.0;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) q += p[1 + i] * x[i] * x[i];
  return p[0] / q * (1.0 + p[8] * sin(x[0] * x[1]));
}
"""
RATIONAL_F32 = RATIONAL_F64.replace("double", "float").replace("sin(", "sinf(").replace(
    "1.0", "1.0f")


def rational_np(x, p):
    d = x.shape[1]
    q = 1.0 + np.sum(p[1:1 + d] * x * x, axis=1)
    return p[0] / q * (1.0 + p[8] * np.sin(x[:, 0] * x[:, 1]))


def _as_user(table):
    t = table.copy()
    t["family"] = W.USER
    t["deg"] = 0
    return t


def _numpy_results(table, fn):
    """FP64 estimate / stderr / mean|f| at the oracle's sample points."""
    out = np.zeros(len(table), dtype=[("estimate", "f8"), ("stderr", "f8"), ("mean_abs", "f8"),
                                      ("n", "u8")])
    for i, row in enumerate(table):
        n = int(row["n_samples"])
        _, x, _ = oracle.samples(row, 0, n)
        f = fn(x, row["p"])
        V = G.volume(row)
        mean = f.mean()
        m2 = float(np.sum((f - mean) ** 2))
        out["estimate"][i] = V * mean
        out["stderr"][i] = V * math.sqrt(m2 / (n * (n - 1))) if n > 1 else math.nan
        out["mean_abs"][i] = np.abs(f).mean()
        out["n"][i] = n
    return out


@pytest.fixture(scope="module")
def udfs():
    u = {
        "harm64": zmc.Udf(HARMONIC_F64, 4, zmc.ZMC_UDF_F64, amplitude=2.0),
        "harm32": zmc.Udf(HARMONIC_F32, 4, zmc.ZMC_UDF_F32, amplitude=2.0),
        "gauss32_3": zmc.Udf(GAUSS_F32, 3, zmc.ZMC_UDF_F32, amplitude=1.0),
        "rat64_5": zmc.Udf(RATIONAL_F64, 5, zmc.ZMC_UDF_F64, amplitude=8.0),
        "rat32_5": zmc.Udf(RATIONAL_F32, 5, zmc.ZMC_UDF_F32, amplitude=8.0),
    }
    yield u
    for v in u.values():
        v.close()


def test_f64_harmonic_matches_oracle_fig1(zctx, udfs):
    """Eq. 1 written by the user, FP64: the Fig. 1 set against the oracle."""
    t = W.harmonic_fig1(10**5)
    got = udfs["harm64"].integrate(zctx.handle, _as_user(t))
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)


def test_f32_harmonic_same_samples_as_builtin(zctx, udfs):
    """The user path draws exactly the built-in path's samples: the FP32 user
    harmonic agrees with the oracle (tolerance for FP32 sincosf of arguments up
    to |k.x| ~ 95, relative error ~1e-7 x |k.x|) and with the built-in family."""
    t = W.harmonic_fig1(10**5)[::7]
    got = udfs["harm32"].integrate(zctx.handle, _as_user(t))
    want, _ = oracle.integrate(t)
    G.compare(t, got, want, est_rel=2e-5, se_rel=1e-3)
    builtin = zmc.zmc_integrate(zctx.handle, t)
    G.compare(t, got, _with_mean_abs(builtin, want), est_rel=2e-5, se_rel=1e-3)


def _with_mean_abs(res, want):
    out = np.zeros(len(res), dtype=[("estimate", "f8"), ("stderr", "f8"), ("mean_abs", "f8"),
                                    ("n", "u8")])
    out["estimate"], out["stderr"], out["n"] = res["estimate"], res["stderr"], res["n"]
    out["mean_abs"] = want["mean_abs"]
    return out


def test_f32_gauss_matches_oracle(zctx, udfs):
    rng = np.random.default_rng(31)
    t = W.random_table(30, rng, n_lo=1, n_hi=60000, families=(W.GAUSS,), dims=(3,), seed=2)
    got = udfs["gauss32_3"].integrate(zctx.handle, _as_user(t))
    want, _ = oracle.integrate(t)
    G.compare(t, got, want)


@pytest.mark.parametrize("key,est_rel", [("rat64_5", 1e-6), ("rat32_5", 1e-6)])
def test_function_without_builtin_counterpart(zctx, udfs, key, est_rel):
    rng = np.random.default_rng(41)
    t = W.empty(16)
    for i in range(16):
        lo = rng.uniform(-1.0, 0.0, 5)
        hi = lo + rng.uniform(0.5, 2.0, 5)
        W.set_box(t[i], lo, hi)
        t[i]["family"], t[i]["dim"] = W.USER, 5
        t[i]["n_samples"] = int(rng.integers(1, 120000)) if i else 1
        t[i]["seed"], t[i]["stream_id"] = 77, 1000 + i
        t[i]["p"][0] = rng.uniform(0.5, 3.0)
        t[i]["p"][1:6] = rng.uniform(0.1, 2.0, 5)
        t[i]["p"][8] = rng.uniform(-0.5, 0.5)
    got = udfs[key].integrate(zctx.handle, t)
    want = _numpy_results(t, rational_np)
    G.compare(t, got, want, est_rel=est_rel)


def test_eval_samples_match_numpy(zctx, udfs):
    t = W.empty(1)
    W.set_box(t[0], [-0.5, 0.0, 0.2, -1.0, 0.3], [0.5, 1.5, 0.9, 1.0, 2.0])
    t[0]["family"], t[0]["dim"], t[0]["n_samples"] = W.USER, 5, 5000
    t[0]["seed"], t[0]["stream_id"] = 3, 9
    t[0]["p"][0], t[0]["p"][1:6], t[0]["p"][8] = 2.0, [0.3, 0.5, 1.0, 0.2, 0.7], 0.4
    _, x, _ = oracle.samples(t[0], 1234, 3000)
    want = rational_np(x, t[0]["p"])
    v64 = udfs["rat64_5"].eval_samples(zctx.handle, t[0], 1234, 3000)
    v32 = udfs["rat32_5"].eval_samples(zctx.handle, t[0], 1234, 3000)
    # FP64 evaluation rounded once to FP32; FP32 evaluation a few ulp more
    assert np.all(np.abs(v64 - want) <= 2.0**-23 * np.abs(want) + 1e-30)
    assert np.all(np.abs(v32 - want) <= 4e-6 * np.abs(want) + 1e-30)


def test_descriptor_validation(zctx, udfs):
    t = _as_user(W.harmonic_fig1(1000)[:2])
    bad = t.copy()
    bad["family"][1] = W.HARMONIC
    with pytest.raises(zmc.ZmcError) as e:
        udfs["harm64"].integrate(zctx.handle, bad)
    assert e.value.status == zmc.ZMC_EINVAL
    with pytest.raises(zmc.ZmcError) as e:
        udfs["gauss32_3"].integrate(zctx.handle, t)  # compiled for 3 dimensions
    assert e.value.status == zmc.ZMC_EINVAL
    bad = t.copy()
    bad["hi"][0][0] = bad["lo"][0][0]
    with pytest.raises(zmc.ZmcError) as e:
        udfs["harm64"].integrate(zctx.handle, bad)
    assert e.value.status == zmc.ZMC_EINVAL
    # the context is still usable
    got = udfs["harm64"].integrate(zctx.handle, t)
    assert np.all(got["status"] == 0)


ABSLIN_F32 = r"""
__device__ float zmc_user_f(const float *x, const float *p) {
  float s = 0.0f;
  for (int i = 0; i < ZMC_UDF_DIM; ++i) s = fmaf(p[1 + i], x[i], s);
  return p[0] * fabsf(s);
}
"""


def test_multi_function_batch_matches_references(zctx):
    """Three user functions of different forms and dimensions (Eq. 1 in 4-D,
    Eq. 2 in 2-D, the rational form in 5-D), their rows interleaved in one
    table and integrated in one call, against the oracle's families and the
    numpy reference; each row as when its function is integrated alone."""
    multi = zmc.Udf([HARMONIC_F32, ABSLIN_F32, RATIONAL_F32], [4, 2, 5], zmc.ZMC_UDF_F32,
                    [2.0, 8.0, 8.0])
    rng = np.random.default_rng(90)
    harm = W.harmonic_fig1(30000)[::9]
    absl = W.abslin_eq2(20000)[:10]
    absl = absl[absl["dim"] == 2]
    rat = W.empty(6)
    for i in range(6):
        lo = rng.uniform(-1.0, 0.0, 5)
        W.set_box(rat[i], lo, lo + rng.uniform(0.5, 2.0, 5))
        rat[i]["family"], rat[i]["dim"] = W.USER, 5
        rat[i]["n_samples"], rat[i]["seed"], rat[i]["stream_id"] = 40000 + i, 5, 500 + i
        rat[i]["p"][0], rat[i]["p"][1:6], rat[i]["p"][8] = 1.5, rng.uniform(0.1, 2.0, 5), 0.3
    parts = [(_as_user(harm), 0), (_as_user(absl), 1), (rat.copy(), 2)]
    rows = []
    for tab, k in parts:
        tab["deg"] = k
        rows.extend(list(tab))
    order = rng.permutation(len(rows))
    table = W.empty(len(rows))
    for j, i in enumerate(order):
        table[j] = rows[i]
    got = multi.integrate(zctx.handle, table)
    back = np.empty_like(got)
    back[order] = got
    n_h, n_a = len(harm), len(absl)
    want_h, _ = oracle.integrate(harm)
    want_a, _ = oracle.integrate(absl)
    G.compare(harm, back[:n_h], want_h, est_rel=2e-5, se_rel=1e-3)  # FP32 sincosf, |k.x| ~ 95
    G.compare(absl, back[n_h:n_h + n_a], want_a)
    G.compare(rat, back[n_h + n_a:], _numpy_results(rat, rational_np))
    alone = zmc.Udf(RATIONAL_F32, 5, zmc.ZMC_UDF_F32, 8.0)
    ra = alone.integrate(zctx.handle, _deg0(rat))
    # the same source compiled alone (another module): the same samples and
    # formula; FP32 code generation may differ between modules by an ulp
    assert np.allclose(ra["estimate"], back[n_h + n_a:]["estimate"], rtol=1e-6, atol=0)
    alone.close()
    bad = table.copy()
    bad["deg"][0] = 3  # no function 3
    with pytest.raises(zmc.ZmcError) as e:
        multi.integrate(zctx.handle, bad)
    assert e.value.status == zmc.ZMC_EINVAL
    multi.close()


def _deg0(t):
    t = t.copy()
    t["deg"] = 0
    return t
