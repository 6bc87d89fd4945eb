"""Seeded synthetic integrand tables (inputs only; no Monte Carlo arithmetic here).

Both the CUDA path (through the C ABI) and the FP64 CPU oracle consume the
tables built here, so this module holds nothing but the *definition* of the
inputs: families, dimensions, boxes, coefficients, sample budgets and Philox
keys.  It performs no sampling, no integrand evaluation and no reduction.

The row layout is the C ABI's ``zmc_desc`` (464 bytes, little endian):

    family u32 | dim u32 | stream_id u32 | deg u32 | n_samples u64 | seed u64 |
    lo f64[7] | hi f64[7] | p f64[40]

Family parameter layout in ``p`` (x is the point in the box, d = dim):

    HARMONIC (0)  a*cos(k.x) + b*sin(k.x)         p[0]=a, p[1]=b, p[2+i]=k_i
                  (paper, Eq. 1)
    ABSLIN   (1)  a*|c.x|                          p[0]=a, p[1+i]=c_i
                  (paper, Eq. 2)
    GAUSS    (2)  A*exp(-|x-mu|^2 / (2 sigma^2))   p[0]=A, p[1]=sigma, p[2+i]=mu_i
    POLY     (3)  prod_i sum_{j<=deg} c_ij x_i^j   p[5*i+j]=c_ij

Workloads (the paper's test problems and the scaled-up mixes built from them):

* :func:`harmonic_fig1` -- the 100 four-dimensional harmonics of the paper's
  GPU test (Sec. "Test on GPUs", Eq. 1, Fig. 1): a=b=1, box [0,1]^4,
  k_n = (n+50)/(2 pi) * (1,1,1,1), n = 1..100.
* :func:`abslin_eq2` -- the mixed-dimension abs-linear set of Eq. 2
  (n < 50: a_n|x1+x2| in 2-D, n >= 50: b_n|x1+x2-x3| in 3-D) with the
  coefficients and boxes drawn as stated in :func:`abslin_eq2`.
* :func:`mixed` -- the 10^4-integrand mix of all four families, dimensions
  1..7, log-uniform sample budgets 10^4..10^7 (the "10^4 different
  integrations" use case of the paper's closing comments).
* :func:`serving_stream` -- a Poisson stream of jobs, each a small mix.
"""
from __future__ import annotations

import math

import numpy as np

MAX_DIM = 7
N_PARAM = 40

HARMONIC, ABSLIN, GAUSS, POLY = 0, 1, 2, 3
USER = 4  # a user-defined integrand (zmc_udf_integrate)
FAMILY_NAMES = {HARMONIC: "harmonic", ABSLIN: "abslin", GAUSS: "gauss", POLY: "poly"}

DESC_DTYPE = np.dtype(
    [
        ("family", "<u4"),
        ("dim", "<u4"),
        ("stream_id", "<u4"),
        ("deg", "<u4"),
        ("n_samples", "<u8"),
        ("seed", "<u8"),
        ("lo", "<f8", (MAX_DIM,)),
        ("hi", "<f8", (MAX_DIM,)),
        ("p", "<f8", (N_PARAM,)),
    ],
    align=True,
)
assert DESC_DTYPE.itemsize == 464


def empty(n: int) -> np.ndarray:
    """A zero-filled table of ``n`` descriptors."""
    return np.zeros(n, dtype=DESC_DTYPE)


def set_box(row, lo, hi) -> None:
    d = len(lo)
    row["lo"][:d] = lo
    row["hi"][:d] = hi


def harmonic(row, a, b, k, lo, hi, n_samples, seed=0, stream_id=0) -> None:
    d = len(k)
    row["family"], row["dim"], row["deg"] = HARMONIC, d, 0
    row["n_samples"], row["seed"], row["stream_id"] = n_samples, seed, stream_id
    set_box(row, lo, hi)
    row["p"][0], row["p"][1] = a, b
    row["p"][2 : 2 + d] = k


def abslin(row, a, c, lo, hi, n_samples, seed=0, stream_id=0) -> None:
    d = len(c)
    row["family"], row["dim"], row["deg"] = ABSLIN, d, 0
    row["n_samples"], row["seed"], row["stream_id"] = n_samples, seed, stream_id
    set_box(row, lo, hi)
    row["p"][0] = a
    row["p"][1 : 1 + d] = c


def gauss(row, amp, sigma, mu, lo, hi, n_samples, seed=0, stream_id=0) -> None:
    d = len(mu)
    row["family"], row["dim"], row["deg"] = GAUSS, d, 0
    row["n_samples"], row["seed"], row["stream_id"] = n_samples, seed, stream_id
    set_box(row, lo, hi)
    row["p"][0], row["p"][1] = amp, sigma
    row["p"][2 : 2 + d] = mu


def poly(row, coef, lo, hi, n_samples, seed=0, stream_id=0) -> None:
    """``coef`` has shape (d, deg+1); coef[i][j] multiplies x_i**j."""
    coef = np.asarray(coef, dtype=np.float64)
    d, g1 = coef.shape
    row["family"], row["dim"], row["deg"] = POLY, d, g1 - 1
    row["n_samples"], row["seed"], row["stream_id"] = n_samples, seed, stream_id
    set_box(row, lo, hi)
    for i in range(d):
        row["p"][5 * i : 5 * i + g1] = coef[i]


# ---------------------------------------------------------------- paper workloads


def harmonic_fig1(n_samples: int = 10**5, seeds=(0,)) -> np.ndarray:
    """The 100 harmonics of the paper's GPU test (Eq. 1, Fig. 1).

    One block of 100 rows per Philox key in ``seeds``; within a block, row
    n-1 is f_n with stream_id n-1.  ``seeds=range(10)`` gives the paper's ten
    independent evaluations in one table.
    """
    seeds = list(seeds)
    t = empty(100 * len(seeds))
    for r, seed in enumerate(seeds):
        for n in range(1, 101):
            kn = (n + 50) / (2.0 * math.pi)
            harmonic(t[r * 100 + n - 1], 1.0, 1.0, [kn] * 4, [0.0] * 4, [1.0] * 4,
                     n_samples, seed=seed, stream_id=n - 1)
    return t


def _box(rng, d):
    lo = rng.uniform(-1.0, 0.0, size=d)
    width = rng.uniform(0.5, 2.0, size=d)
    return lo, lo + width


def abslin_eq2(n_samples: int = 10**6, gen_seed: int = 2104, seed: int = 0) -> np.ndarray:
    """The mixed-dimension abs-linear set of Eq. 2.

    n = 1..49: a_n |x1 + x2| on a 2-D box; n = 50..100: b_n |x1 + x2 - x3| on a
    3-D box.  The paper gives neither coefficients nor boxes; they are drawn
    here as a_n, b_n ~ U[0.5, 2], lo ~ U[-1, 0]^d, width ~ U[0.5, 2]^d from
    ``numpy.random.default_rng(gen_seed)``, row by row in n order.
    """
    rng = np.random.default_rng(gen_seed)
    t = empty(100)
    for n in range(1, 101):
        c = [1.0, 1.0] if n < 50 else [1.0, 1.0, -1.0]
        a = rng.uniform(0.5, 2.0)
        lo, hi = _box(rng, len(c))
        abslin(t[n - 1], a, c, lo, hi, n_samples, seed=seed, stream_id=n - 1)
    return t


def _mixed_row(rng, row, n_samples, seed, stream_id):
    fam = int(rng.integers(0, 4))
    d = int(rng.integers(1, MAX_DIM + 1))
    lo, hi = _box(rng, d)
    if fam == HARMONIC:
        a, b = rng.uniform(0.5, 2.0, size=2)
        k = rng.uniform(-30.0, 30.0, size=d)
        harmonic(row, a, b, k, lo, hi, n_samples, seed, stream_id)
    elif fam == ABSLIN:
        a = rng.uniform(0.5, 2.0)
        c = rng.choice([-1.0, 1.0], size=d)
        abslin(row, a, c, lo, hi, n_samples, seed, stream_id)
    elif fam == GAUSS:
        mu = rng.uniform(lo, hi)
        sigma = rng.uniform(0.05, 0.5)
        gauss(row, 1.0, sigma, mu, lo, hi, n_samples, seed, stream_id)
    else:
        deg = int(rng.integers(0, 5))
        coef = rng.standard_normal(size=(d, deg + 1))
        poly(row, coef, lo, hi, n_samples, seed, stream_id)


def log_uniform_budget(rng, lo_exp=4.0, hi_exp=7.0) -> int:
    return int(round(10.0 ** rng.uniform(lo_exp, hi_exp)))


def mixed(n_fn: int = 10**4, gen_seed: int = 2104, seed: int = 0,
          lo_exp: float = 4.0, hi_exp: float = 7.0) -> np.ndarray:
    """``n_fn`` integrands drawn uniformly over the four families.

    Per row: family ~ U{harmonic, abslin, gauss, poly}, d ~ U{1..7},
    lo ~ U[-1, 0]^d, width ~ U[0.5, 2]^d; harmonic a, b ~ U[0.5, 2],
    k ~ U[-30, 30]^d; abs-linear a ~ U[0.5, 2], c_i ~ U{-1, +1}; Gaussian
    amplitude 1, mu ~ U(box), sigma ~ U[0.05, 0.5]; polynomial degree
    ~ U{0..4} (same in every dimension), coefficients ~ N(0, 1).  The sample
    budget is round(10^U[lo_exp, hi_exp]), the Philox key is ``seed`` and the
    stream id is the row index.
    """
    rng = np.random.default_rng(gen_seed)
    t = empty(n_fn)
    for i in range(n_fn):
        n = log_uniform_budget(rng, lo_exp, hi_exp)
        _mixed_row(rng, t[i], n, seed, i)
    return t


def mixed_block(rng, n_fn: int, seed: int, lo_exp: float = 4.0, hi_exp: float = 7.0,
                stream_base: int = 0) -> np.ndarray:
    """``n_fn`` rows drawn like :func:`mixed`, vectorised (same distributions,
    drawn array by array, so the rows differ from :func:`mixed`'s)."""
    t = empty(n_fn)
    fam = rng.integers(0, 4, size=n_fn)
    dim = rng.integers(1, MAX_DIM + 1, size=n_fn)
    t["family"] = fam
    t["dim"] = dim
    t["stream_id"] = stream_base + np.arange(n_fn)
    t["seed"] = seed
    t["n_samples"] = np.round(10.0 ** rng.uniform(lo_exp, hi_exp, size=n_fn)).astype(np.uint64)
    active = np.arange(MAX_DIM)[None, :] < dim[:, None]
    lo = rng.uniform(-1.0, 0.0, size=(n_fn, MAX_DIM))
    hi = lo + rng.uniform(0.5, 2.0, size=(n_fn, MAX_DIM))
    t["lo"] = np.where(active, lo, 0.0)
    t["hi"] = np.where(active, hi, 0.0)
    p = np.zeros((n_fn, N_PARAM))
    ab = rng.uniform(0.5, 2.0, size=(n_fn, 2))
    k = rng.uniform(-30.0, 30.0, size=(n_fn, MAX_DIM))
    c = rng.choice([-1.0, 1.0], size=(n_fn, MAX_DIM))
    sigma = rng.uniform(0.05, 0.5, size=n_fn)
    mu = rng.uniform(lo, hi)
    deg = rng.integers(0, 5, size=n_fn)
    coef = rng.standard_normal(size=(n_fn, MAX_DIM, 5))
    h = fam == HARMONIC
    p[h, 0], p[h, 1] = ab[h, 0], ab[h, 1]
    p[h, 2:2 + MAX_DIM] = np.where(active[h], k[h], 0.0)
    a = fam == ABSLIN
    p[a, 0] = ab[a, 0]
    p[a, 1:1 + MAX_DIM] = np.where(active[a], c[a], 0.0)
    g = fam == GAUSS
    p[g, 0], p[g, 1] = 1.0, sigma[g]
    p[g, 2:2 + MAX_DIM] = np.where(active[g], mu[g], 0.0)
    q = fam == POLY
    mask = active[:, :, None] & (np.arange(5)[None, None, :] <= deg[:, None, None])
    p[q, :5 * MAX_DIM] = np.where(mask[q], coef[q], 0.0).reshape(-1, 5 * MAX_DIM)
    t["p"] = p
    t["deg"] = np.where(q, deg, 0)
    return t


def serving_stream(rate_hz: float, duration_s: float, arrival_seed: int = 5,
                   max_fns: int = 1000, lo_exp: float = 4.0, hi_exp: float = 7.0):
    """Poisson job arrivals at ``rate_hz`` over ``duration_s`` seconds.

    Returns a list of (arrival_time_s, table).  Each job holds U{1..max_fns}
    integrands drawn like :func:`mixed` (by :func:`mixed_block`), with the job
    index as Philox key.
    """
    rng = np.random.default_rng(arrival_seed)
    jobs = []
    t = 0.0
    j = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n_fn = int(rng.integers(1, max_fns + 1))
        jr = np.random.default_rng([arrival_seed, j])
        jobs.append((t, mixed_block(jr, n_fn, seed=j, lo_exp=lo_exp, hi_exp=hi_exp)))
        j += 1
    return jobs


def random_table(n_fn: int, rng, n_lo: int = 1, n_hi: int = 5000, families=(0, 1, 2, 3),
                 dims=range(1, 8), seed: int = 0) -> np.ndarray:
    """Small mixed tables for parity tests: uniform budgets in [n_lo, n_hi]."""
    t = empty(n_fn)
    fams = list(families)
    dims = list(dims)
    for i in range(n_fn):
        fam = fams[int(rng.integers(0, len(fams)))]
        d = dims[int(rng.integers(0, len(dims)))]
        n = int(rng.integers(n_lo, n_hi + 1))
        lo, hi = _box(rng, d)
        if fam == HARMONIC:
            harmonic(t[i], rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0),
                     rng.uniform(-30.0, 30.0, size=d), lo, hi, n, seed, i)
        elif fam == ABSLIN:
            abslin(t[i], rng.uniform(0.5, 2.0), rng.choice([-1.0, 1.0], size=d), lo, hi,
                   n, seed, i)
        elif fam == GAUSS:
            gauss(t[i], 1.0, rng.uniform(0.05, 0.5), rng.uniform(lo, hi), lo, hi, n, seed, i)
        else:
            deg = int(rng.integers(0, 5))
            poly(t[i], rng.standard_normal(size=(d, deg + 1)), lo, hi, n, seed, i)
    return t


def total_samples(table: np.ndarray) -> int:
    return int(np.sum(table["n_samples"].astype(np.uint64)))
