"""FP64 CPU oracle for multi-function direct Monte Carlo (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It loads ``libzmc_oracle.so`` built from
``zmc_oracle.c`` with the host C compiler and shares no code with the CUDA
implementation.  Every function follows the paper's direct Monte Carlo method
(Sec. "Solution method"; Eq. 1 and Eq. 2 for the integrand families); the
header of ``zmc_oracle.c`` states the steps.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "zmc_oracle.c")
LIB = os.path.join(HERE, "libzmc_oracle.so")

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")

CFLAGS = ["-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
          "-shared"]


def compile_oracle(src: str, out: str) -> str:
    """Compile an oracle source file with gcc (C99, no FMA contraction, OpenMP)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        compile_oracle(SRC, LIB)
    return LIB


def _col(table, name, dtype):
    return np.ascontiguousarray(table[name], dtype=dtype)


def _row_args(row):
    return (int(row["family"]), int(row["dim"]), int(row["stream_id"]), int(row["deg"]),
            int(row["seed"]), np.ascontiguousarray(row["lo"], dtype=np.float64),
            np.ascontiguousarray(row["hi"], dtype=np.float64),
            np.ascontiguousarray(row["p"], dtype=np.float64))


class Oracle:
    """ctypes front end of one compiled oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.zo_philox_many.argtypes = [ctypes.c_size_t, _u32p, _u32p, _u32p]
        lib.zo_philox_many.restype = None
        lib.zo_integrate.argtypes = [ctypes.c_size_t, _u32p, _u32p, _u32p, _u32p, _u64p, _u64p,
                                     _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int]
        lib.zo_integrate.restype = ctypes.c_int
        row = [ctypes.c_uint32] * 4 + [ctypes.c_uint64, _f64p, _f64p, _f64p, ctypes.c_uint64,
                                       ctypes.c_uint64]
        lib.zo_moments.argtypes = row + [_f64p]
        lib.zo_moments.restype = None
        lib.zo_samples.argtypes = row + [_u32p, _f64p, _f64p]
        lib.zo_samples.restype = None
        self.lib = lib

    def philox4x32_10(self, ctr, key) -> np.ndarray:
        """Philox4x32-10 of counters ``ctr`` (n, 4) under keys ``key`` (n, 2)."""
        ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
        key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
        assert ctr.shape[0] == key.shape[0]
        out = np.zeros_like(ctr)
        self.lib.zo_philox_many(ctr.shape[0], ctr.reshape(-1), key.reshape(-1),
                                out.reshape(-1))
        return out

    def integrate(self, table, threads: int = 0):
        """Direct MC of every row of ``table`` (a ``zmc_desc`` structured array).

        Returns ``(result, threads_used)``; result has fields ``estimate``,
        ``stderr``, ``mean_abs`` (mean |f| over the samples) and ``n``.
        """
        n = len(table)
        est, err, mabs = np.zeros(n), np.zeros(n), np.zeros(n)
        used = self.lib.zo_integrate(
            n, _col(table, "family", np.uint32), _col(table, "dim", np.uint32),
            _col(table, "stream_id", np.uint32), _col(table, "deg", np.uint32),
            _col(table, "n_samples", np.uint64), _col(table, "seed", np.uint64),
            _col(table, "lo", np.float64).reshape(-1), _col(table, "hi", np.float64).reshape(-1),
            _col(table, "p", np.float64).reshape(-1), est, err, mabs, int(threads))
        res = np.zeros(n, dtype=[("estimate", "f8"), ("stderr", "f8"), ("mean_abs", "f8"),
                                 ("n", "u8")])
        res["estimate"], res["stderr"], res["mean_abs"] = est, err, mabs
        res["n"] = table["n_samples"]
        return res, used

    def moments(self, row, s_begin: int, s_end: int) -> np.ndarray:
        """Welford (n, mean, M2, sum|f|) of one row over samples [s_begin, s_end)."""
        out = np.zeros(4)
        self.lib.zo_moments(*_row_args(row), int(s_begin), int(s_end), out)
        return out

    def samples(self, row, s_begin: int, count: int):
        """Raw 23-bit fields, points and values of samples [s_begin, s_begin+count)."""
        d = int(row["dim"])
        words = np.zeros((count, d), dtype=np.uint32)
        x = np.zeros((count, d))
        fx = np.zeros(count)
        self.lib.zo_samples(*_row_args(row), int(s_begin), int(count), words.reshape(-1),
                            x.reshape(-1), fx)
        return words, x, fx

    def points(self, dim: int, lo, hi, seed: int, stream_id: int, s_begin: int, count: int):
        """Sample points x (count, dim) of samples [s_begin, s_begin+count) of the
        stream (seed, stream_id) on the box [lo, hi] of any dimension: the same
        generator and map as ``samples``, without an integrand."""
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        assert len(lo) == len(hi) == dim
        words = np.zeros((count, dim), dtype=np.uint32)
        x = np.zeros((count, dim))
        fx = np.zeros(count)
        self.lib.zo_samples(4, int(dim), int(stream_id), 0, int(seed), lo, hi, np.zeros(40),
                            int(s_begin), int(count), words.reshape(-1), x.reshape(-1), fx)
        return x


_lock = threading.Lock()
_default = None


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def philox4x32_10(ctr, key):
    return default().philox4x32_10(ctr, key)


def integrate(table, threads: int = 0):
    return default().integrate(table, threads)


def moments(row, s_begin, s_end):
    return default().moments(row, s_begin, s_end)


def samples(row, s_begin, count):
    return default().samples(row, s_begin, count)


def points(dim, lo, hi, seed, stream_id, s_begin, count):
    return default().points(dim, lo, hi, seed, stream_id, s_begin, count)
