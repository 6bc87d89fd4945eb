"""ctypes binding of ``libzmc.so`` (C ABI declared in ``include/zmc.h``).

Argument marshalling only: every step of the integration runs in the library's
CUDA kernels.  Function names are the C entry points'.  Descriptor tables are
numpy structured arrays with the ``zmc_desc`` layout
(:data:`paper_2104_10073_gb300.workloads.DESC_DTYPE`), passed by pointer.

There is no fallback: if the library cannot be loaded, :func:`lib` raises.
PyTorch is used only to provide device memory (an optional arena tensor) and
the CUDA stream the library runs on (see :class:`Context`).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libzmc.so")

# zmc_status
ZMC_OK, ZMC_EINVAL, ZMC_ENOMEM, ZMC_EAGAIN, ZMC_ETIMEOUT = 0, 1, 2, 3, 4
ZMC_ECUDA, ZMC_ENOTFOUND, ZMC_ECLOSED, ZMC_ENOSYS = 5, 6, 7, 8
STATUS_NAMES = {0: "ZMC_OK", 1: "ZMC_EINVAL", 2: "ZMC_ENOMEM", 3: "ZMC_EAGAIN",
                4: "ZMC_ETIMEOUT", 5: "ZMC_ECUDA", 6: "ZMC_ENOTFOUND", 7: "ZMC_ECLOSED",
                8: "ZMC_ENOSYS"}
ZMC_STAGE_SAMPLE, ZMC_STAGE_MERGE, ZMC_STAGE_ALL = 1, 2, 3
ZMC_TUNE_GEOMETRY, ZMC_TUNE_CHUNK = 1, 2  # zmc_options.autotune flags
ZMC_USER = 4
DEFAULT_QUINTS_PER_LANE = 104  # the library's default chunk: 160 x 104 = 16640 samples
SERVING_QUINTS_PER_LANE = 26  # ... and for a serving context: 4160 samples
ZMC_UDF_F32, ZMC_UDF_F64 = 0, 1

RESULT_DTYPE = np.dtype([("estimate", "<f8"), ("stderr", "<f8"), ("n", "<u8"),
                         ("status", "<i4"), ("reserved", "<i4")])
assert RESULT_DTYPE.itemsize == 32
MOMENTS_DTYPE = np.dtype([("mean", "<f8"), ("m2", "<f8"), ("n", "<u8"), ("status", "<i4"),
                          ("reserved", "<i4")])


class zmc_options(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("arena", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("max_chunks_per_iter", ctypes.c_uint32),
                ("autotune", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("quints_per_lane", ctypes.c_uint32), ("tune_cache_path", ctypes.c_char_p),
                ("serving", ctypes.c_uint32), ("serving_share", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("serving_cut_backlog", ctypes.c_uint64)]


class zmc_plan_info(ctypes.Structure):
    _fields_ = [("n_fn", ctypes.c_uint64), ("n_chunks", ctypes.c_uint64),
                ("n_samples", ctypes.c_uint64), ("grid", ctypes.c_uint32),
                ("block", ctypes.c_uint32), ("quints_per_lane", ctypes.c_uint32),
                ("sms", ctypes.c_uint32), ("family_grid", ctypes.c_uint32 * 4),
                ("family_block", ctypes.c_uint32 * 4), ("tune_source", ctypes.c_int32 * 4),
                ("family_unroll", ctypes.c_uint32 * 4), ("chunk_tune_source", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


class zmc_normal_opts(ctypes.Structure):
    _fields_ = [("divisions", ctypes.c_uint32), ("depth", ctypes.c_uint32),
                ("samples_per_cell", ctypes.c_uint64), ("sigma_mult", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("stream_base", ctypes.c_uint32),
                ("max_leaves", ctypes.c_uint32)]


class zmc_normal_result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("stderr_", ctypes.c_double),
                ("n_samples", ctypes.c_uint64), ("n_cells", ctypes.c_uint64),
                ("n_leaves", ctypes.c_uint64), ("rounds", ctypes.c_uint32),
                ("status", ctypes.c_int32)]


class zmc_serving_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "completed", "cancelled", "queued", "running", "iterations",
        "samples_done", "arena_used_bytes", "arena_bytes", "shared_iterations",
        "max_jobs_per_iter")]


class ZmcError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_P = ctypes.c_void_p
_SIGS = {
    "zmc_default_options": ([ctypes.POINTER(zmc_options)], ctypes.c_int),
    "zmc_create": ([ctypes.POINTER(zmc_options), ctypes.POINTER(_P)], ctypes.c_int),
    "zmc_destroy": ([_P], ctypes.c_int),
    "zmc_last_error": ([_P], ctypes.c_char_p),
    "zmc_integrate": ([_P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "zmc_integrate_plain": ([_P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "zmc_integrate_moments": ([_P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "zmc_integrate_functional": ([_P, _P, _P, ctypes.c_uint32, _P, ctypes.c_size_t,
                                  ctypes.c_uint32, _P], ctypes.c_int),
    "zmc_submit": ([_P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "zmc_poll": ([_P, ctypes.c_uint64, _P, ctypes.c_int32], ctypes.c_int),
    "zmc_cancel": ([_P, ctypes.c_uint64], ctypes.c_int),
    "zmc_checkpoint": ([_P, ctypes.c_uint64, _P, ctypes.c_int32], ctypes.c_int),
    "zmc_submit_resume": ([_P, _P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)],
                          ctypes.c_int),
    "zmc_poll_any": ([_P, _P, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)],
                     ctypes.c_int),
    "zmc_serving_stats_get": ([_P, ctypes.POINTER(zmc_serving_stats)], ctypes.c_int),
    "zmc_plan_create": ([_P, _P, ctypes.c_size_t, ctypes.POINTER(_P)], ctypes.c_int),
    "zmc_plan_run": ([_P, ctypes.c_uint32], ctypes.c_int),
    "zmc_plan_run_plain": ([_P], ctypes.c_int),
    "zmc_plan_results": ([_P, _P], ctypes.c_int),
    "zmc_plan_device_results": ([_P, ctypes.POINTER(_P)], ctypes.c_int),
    "zmc_plan_info_get": ([_P, ctypes.POINTER(zmc_plan_info)], ctypes.c_int),
    "zmc_plan_destroy": ([_P], ctypes.c_int),
    "zmc_philox4x32_10": ([_P, _P, _P, _P, ctypes.c_size_t], ctypes.c_int),
    "zmc_philox_rate": ([_P, ctypes.c_uint64, _P], ctypes.c_int),
    "zmc_eval_samples": ([_P, _P, ctypes.c_uint64, ctypes.c_uint32, _P], ctypes.c_int),
    "zmc_validate": ([_P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "zmc_variant_of": ([_P, ctypes.c_size_t, _P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "zmc_serving_fill": ([_P, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                          ctypes.c_uint64, _P], ctypes.c_int),
    "zmc_integrate_noalloc": ([_P, ctypes.c_size_t, _P, _P], ctypes.c_int),
    "zmc_udf_create": ([ctypes.c_char_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                        ctypes.POINTER(_P)], ctypes.c_int),
    "zmc_udf_create_multi": ([_P, _P, ctypes.c_uint32, ctypes.c_uint32, _P, ctypes.POINTER(_P)],
                             ctypes.c_int),
    "zmc_udf_integrate": ([_P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "zmc_udf_eval_samples": ([_P, _P, _P, ctypes.c_uint64, ctypes.c_uint32, _P], ctypes.c_int),
    "zmc_udf_log": ([_P], ctypes.c_char_p),
    "zmc_udf_destroy": ([_P], ctypes.c_int),
    "zmc_normal_default_options": ([ctypes.POINTER(zmc_normal_opts)], ctypes.c_int),
    "zmc_normal_integrate": ([_P, _P, ctypes.POINTER(zmc_normal_opts),
                              ctypes.POINTER(zmc_normal_result)], ctypes.c_int),
    "zmc_normal_integrate_udf": ([_P, _P, _P, _P, _P, ctypes.POINTER(zmc_normal_opts),
                                  ctypes.POINTER(zmc_normal_result)], ctypes.c_int),
    "zmc_desc_size": ([], ctypes.c_size_t),
    "zmc_result_size": ([], ctypes.c_size_t),
}
EXPORTED = tuple(_SIGS)

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load ``libzmc.so`` (raises if it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} not built; run paper_2104_10073_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            if L.zmc_desc_size() != W.DESC_DTYPE.itemsize:
                raise RuntimeError("zmc_desc layout mismatch")
            if L.zmc_result_size() != RESULT_DTYPE.itemsize:
                raise RuntimeError("zmc_result layout mismatch")
            _lib = L
    return _lib


def _check(status, where):
    if status != ZMC_OK:
        raise ZmcError(status, where, lib().zmc_last_error(None).decode())


def _table(desc) -> np.ndarray:
    t = np.ascontiguousarray(desc, dtype=W.DESC_DTYPE)
    if t.ndim != 1:
        t = t.reshape(-1)
    return t


# ------------------------------------------------------------------ thin wrappers
def zmc_default_options() -> zmc_options:
    """The library defaults (zmc_default_options)."""
    o = zmc_options()
    _check(lib().zmc_default_options(ctypes.byref(o)), "zmc_default_options")
    return o


def zmc_create(opt: zmc_options | None = None) -> int:
    """Create a context from a zmc_options (zmc_create); returns the handle."""
    h = ctypes.c_void_p()
    _check(lib().zmc_create(ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)),
           "zmc_create")
    return h.value


def zmc_destroy(ctx: int) -> None:
    """Release a context (zmc_destroy)."""
    _check(lib().zmc_destroy(ctx), "zmc_destroy")


def zmc_last_error(ctx: int | None = None) -> str:
    """The reason of the last failure on this thread (zmc_last_error)."""
    return lib().zmc_last_error(ctx).decode()


def zmc_integrate(ctx: int, desc) -> np.ndarray:
    """Blocking batched integration of a descriptor table (zmc_integrate); one
    RESULT_DTYPE row per descriptor."""
    t = _table(desc)
    out = np.zeros(len(t), dtype=RESULT_DTYPE)
    _check(lib().zmc_integrate(ctx, t.ctypes.data, len(t), out.ctypes.data), "zmc_integrate")
    return out


def zmc_integrate_plain(ctx: int, desc) -> np.ndarray:
    """The same results computed the plain way, one FP64 launch per integrand
    (zmc_integrate_plain)."""
    t = _table(desc)
    out = np.zeros(len(t), dtype=RESULT_DTYPE)
    _check(lib().zmc_integrate_plain(ctx, t.ctypes.data, len(t), out.ctypes.data),
           "zmc_integrate_plain")
    return out


def zmc_integrate_moments(ctx: int, desc, s_begin, s_end) -> np.ndarray:
    """(mean, m2, n) of each row over its sample range [s_begin, s_end)."""
    t = _table(desc)
    b = np.ascontiguousarray(np.asarray(s_begin, dtype=np.uint64).reshape(-1))
    e = np.ascontiguousarray(np.asarray(s_end, dtype=np.uint64).reshape(-1))
    assert len(b) == len(e) == len(t)
    out = np.zeros(len(t), dtype=MOMENTS_DTYPE)
    _check(lib().zmc_integrate_moments(ctx, t.ctypes.data, b.ctypes.data, e.ctypes.data, len(t),
                                       out.ctypes.data), "zmc_integrate_moments")
    return out


def slot_p(j: int) -> int:
    """Functional-mode slot of parameter p[j] (ZMC_SLOT_P)."""
    return j


def slot_lo(i: int) -> int:
    """Functional-mode slot of lo[i] (ZMC_SLOT_LO)."""
    return 40 + i


def slot_hi(i: int) -> int:
    """Functional-mode slot of hi[i] (ZMC_SLOT_HI)."""
    return 47 + i


def zmc_integrate_functional(ctx: int, base_row, slots, values, independent_streams=True):
    """Results of ``base_row`` at each parameter point: row q of ``values``
    (n_points x len(slots)) sets the given slots (see slot_p / slot_lo / slot_hi)."""
    t = _table(np.asarray(base_row).reshape(1))
    sl = np.ascontiguousarray(np.asarray(slots, dtype=np.uint32).reshape(-1))
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(-1, len(sl)))
    out = np.zeros(v.shape[0], dtype=RESULT_DTYPE)
    _check(lib().zmc_integrate_functional(ctx, t.ctypes.data, sl.ctypes.data, len(sl),
                                          v.ctypes.data, v.shape[0],
                                          1 if independent_streams else 0, out.ctypes.data),
           "zmc_integrate_functional")
    return out


def zmc_submit(ctx: int, desc) -> int:
    """Queue a table on a serving context (zmc_submit); returns the job id."""
    t = _table(desc)
    jid = ctypes.c_uint64()
    _check(lib().zmc_submit(ctx, t.ctypes.data, len(t), ctypes.byref(jid)), "zmc_submit")
    return jid.value


def zmc_poll(ctx: int, job_id: int, n: int, wait_ms: int = -1):
    """Returns (status, results-or-None); ZMC_EAGAIN / ZMC_ETIMEOUT are not errors."""
    out = np.zeros(n, dtype=RESULT_DTYPE)
    st = lib().zmc_poll(ctx, job_id, out.ctypes.data, wait_ms)
    if st in (ZMC_EAGAIN, ZMC_ETIMEOUT):
        return st, None
    if st == ZMC_OK:
        return st, out
    return st, None


def zmc_poll_any(ctx: int, cap: int = 1024, wait_ms: int = -1):
    """(status, list of finished job ids); each finished job is reported once."""
    ids = np.zeros(cap, dtype=np.uint64)
    n = ctypes.c_size_t(0)
    st = lib().zmc_poll_any(ctx, ids.ctypes.data, cap, wait_ms, ctypes.byref(n))
    return st, [int(v) for v in ids[:n.value]]


def zmc_cancel(ctx: int, job_id: int) -> None:
    """Cancel a queued or running job (zmc_cancel)."""
    _check(lib().zmc_cancel(ctx, job_id), "zmc_cancel")


def zmc_checkpoint(ctx: int, job_id: int, n: int, wait_ms: int = -1):
    """(status, moments-or-None): stop a job and take the moments of the samples
    each of its n integrands has taken; ZMC_EAGAIN / ZMC_ETIMEOUT are not errors."""
    out = np.zeros(n, dtype=MOMENTS_DTYPE)
    st = lib().zmc_checkpoint(ctx, job_id, out.ctypes.data, wait_ms)
    return st, (out if st == ZMC_OK else None)


def zmc_submit_resume(ctx: int, desc, from_moments) -> int:
    """Submit ``desc`` continuing from ``from_moments`` (a zmc_checkpoint result,
    or zmc_integrate_moments over samples [0, n) of the same streams)."""
    t = _table(desc)
    m = np.ascontiguousarray(np.asarray(from_moments, dtype=MOMENTS_DTYPE).reshape(-1))
    assert len(m) == len(t)
    jid = ctypes.c_uint64()
    _check(lib().zmc_submit_resume(ctx, t.ctypes.data, m.ctypes.data, len(t), ctypes.byref(jid)),
           "zmc_submit_resume")
    return jid.value


def zmc_serving_stats_get(ctx: int) -> dict:
    """Counters of the serving loop (zmc_serving_stats_get) as a dict."""
    s = zmc_serving_stats()
    _check(lib().zmc_serving_stats_get(ctx, ctypes.byref(s)), "zmc_serving_stats_get")
    return {name: getattr(s, name) for name, _ in s._fields_}


def zmc_plan_create(ctx: int, desc) -> int:
    """Precompute and upload a table once (zmc_plan_create); returns the plan."""
    t = _table(desc)
    h = ctypes.c_void_p()
    _check(lib().zmc_plan_create(ctx, t.ctypes.data, len(t), ctypes.byref(h)),
           "zmc_plan_create")
    return h.value


def zmc_plan_run(plan: int, stages: int = ZMC_STAGE_ALL) -> None:
    """Enqueue the plan's stages on the context stream (zmc_plan_run)."""
    _check(lib().zmc_plan_run(plan, stages), "zmc_plan_run")


def zmc_plan_run_plain(plan: int) -> None:
    """Enqueue the plain FP64 form of the plan (zmc_plan_run_plain)."""
    _check(lib().zmc_plan_run_plain(plan), "zmc_plan_run_plain")


def zmc_plan_results(plan: int, n: int) -> np.ndarray:
    """Wait and copy the plan's n results to the host (zmc_plan_results)."""
    out = np.zeros(n, dtype=RESULT_DTYPE)
    _check(lib().zmc_plan_results(plan, out.ctypes.data), "zmc_plan_results")
    return out


def zmc_plan_device_results(plan: int) -> int:
    """Device address of the plan's results (zmc_plan_device_results)."""
    p = ctypes.c_void_p()
    _check(lib().zmc_plan_device_results(plan, ctypes.byref(p)), "zmc_plan_device_results")
    return p.value


def zmc_plan_info_get(plan: int) -> dict:
    """Sizes and launch geometry of a plan (zmc_plan_info_get) as a dict."""
    i = zmc_plan_info()
    _check(lib().zmc_plan_info_get(plan, ctypes.byref(i)), "zmc_plan_info_get")
    out = {}
    for name, _ in i._fields_:
        v = getattr(i, name)
        out[name] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def zmc_plan_destroy(plan: int) -> None:
    """Release a plan (zmc_plan_destroy)."""
    _check(lib().zmc_plan_destroy(plan), "zmc_plan_destroy")


def zmc_philox4x32_10(ctx: int, ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters (n, 4) under keys (n, 2) by the device routine
    of the sampling path (zmc_philox4x32_10)."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    out = np.zeros_like(ctr)
    _check(lib().zmc_philox4x32_10(ctx, ctr.ctypes.data, key.ctypes.data, out.ctypes.data,
                                   ctr.shape[0]), "zmc_philox4x32_10")
    return out


def zmc_philox_rate(ctx: int, n_blocks: int = 1 << 35) -> float:
    """Philox4x32-10 blocks per second of the generator alone (zmc_philox_rate)."""
    r = ctypes.c_double()
    _check(lib().zmc_philox_rate(ctx, n_blocks, ctypes.byref(r)), "zmc_philox_rate")
    return r.value


def zmc_eval_samples(ctx: int, row, s_begin: int, count: int) -> np.ndarray:
    """FP32 values of samples [s_begin, s_begin + count) of one descriptor, by
    the sampling path's own generation, map and evaluation (zmc_eval_samples)."""
    t = _table(np.asarray(row).reshape(1))
    out = np.zeros(count, dtype=np.float32)
    _check(lib().zmc_eval_samples(ctx, t.ctypes.data, int(s_begin), int(count),
                                  out.ctypes.data), "zmc_eval_samples")
    return out


def zmc_integrate_noalloc(desc, out_device_ptr: int, stream_ptr: int | None) -> int:
    """Status of one call of the no-allocation entry point: ``desc`` stays on the
    host, results go to the caller's device array ``out_device_ptr`` (n rows of
    32 bytes) asynchronously on ``stream_ptr``; nothing is allocated."""
    t = _table(desc)
    return lib().zmc_integrate_noalloc(t.ctypes.data, len(t), out_device_ptr, stream_ptr)


def zmc_validate(desc):
    """(status, first bad row or None, message); host only."""
    t = _table(desc)
    bad = ctypes.c_size_t(0)
    st = lib().zmc_validate(t.ctypes.data, len(t), ctypes.byref(bad))
    if st == ZMC_OK:
        return st, None, ""
    return st, bad.value, zmc_last_error()


def zmc_variant_of(desc) -> np.ndarray:
    """The evaluation form the library picks per row (zmc_variant_of): a
    structured array (family, dim, form); host only."""
    t = _table(desc)
    codes = np.zeros(len(t), dtype=np.uint32)
    bad = ctypes.c_size_t(0)
    _check(lib().zmc_variant_of(t.ctypes.data, len(t), codes.ctypes.data, ctypes.byref(bad)),
           "zmc_variant_of")
    out = np.zeros(len(t), dtype=[("family", "u4"), ("dim", "u4"), ("form", "u4")])
    out["family"] = (codes >> 4) & 0xF
    out["dim"] = codes & 0xF
    out["form"] = codes >> 8
    return out


def zmc_serving_fill(chunks_left, budget: int, share: int = 0, cut_backlog: int = 0,
                     chunk_samples: int = 4160) -> np.ndarray:
    """Chunks each live job (oldest first) contributes to one serving launch
    (zmc_serving_fill); host only."""
    left = np.ascontiguousarray(chunks_left, dtype=np.uint64)
    take = np.zeros(len(left), dtype=np.uint64)
    _check(lib().zmc_serving_fill(left.ctypes.data, len(left), budget, share, cut_backlog,
                                  chunk_samples, take.ctypes.data), "zmc_serving_fill")
    return take


# ------------------------------------------------------------------ convenience
def normal_options(**kw) -> zmc_normal_opts:
    """zmc_normal_opts with the library defaults, overridden by keyword."""
    o = zmc_normal_opts()
    _check(lib().zmc_normal_default_options(ctypes.byref(o)), "zmc_normal_default_options")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _normal_dict(r: zmc_normal_result) -> dict:
    return {"estimate": r.estimate, "stderr": r.stderr_, "n_samples": r.n_samples,
            "n_cells": r.n_cells, "n_leaves": r.n_leaves, "rounds": r.rounds}


def zmc_normal_integrate(ctx: int, base_row, opts: zmc_normal_opts) -> dict:
    """Stratified sampling with tree refinement of one built-in integrand."""
    t = _table(np.asarray(base_row).reshape(1))
    r = zmc_normal_result()
    _check(lib().zmc_normal_integrate(ctx, t.ctypes.data, ctypes.byref(opts), ctypes.byref(r)),
           "zmc_normal_integrate")
    return _normal_dict(r)


class Udf:
    """A user-defined integrand compiled at run time (NVRTC); see zmc_udf_create.

    ``source`` defines ``zmc_user_f(const float *x, const float *p)`` (precision
    ZMC_UDF_F32) or the ``double`` form (ZMC_UDF_F64).  Compiling needs no GPU."""

    def __init__(self, source, dim, precision: int = ZMC_UDF_F32, amplitude=0.0):
        """``source`` / ``dim`` / ``amplitude``: one function, or lists of them
        (zmc_udf_create_multi: a row selects function k with its ``deg`` field)."""
        h = _P()
        if isinstance(source, str):
            _check(lib().zmc_udf_create(source.encode(), dim, precision, amplitude,
                                        ctypes.byref(h)), "zmc_udf_create")
            dims = [dim]
        else:
            srcs = [s.encode() for s in source]
            arr = (ctypes.c_char_p * len(srcs))(*srcs)
            dims = [int(d) for d in dim]
            d = np.ascontiguousarray(dims, dtype=np.uint32)
            amps = np.ascontiguousarray(
                amplitude if np.ndim(amplitude) else [amplitude] * len(srcs), dtype=np.float64)
            _check(lib().zmc_udf_create_multi(ctypes.cast(arr, _P), d.ctypes.data, len(srcs),
                                              precision, amps.ctypes.data, ctypes.byref(h)),
                   "zmc_udf_create_multi")
        self.handle = h.value
        self.dims = dims
        self.dim = dims[0]
        self.precision = precision

    @property
    def log(self) -> str:
        return lib().zmc_udf_log(self.handle).decode()

    def integrate(self, ctx: int, desc) -> np.ndarray:
        t = _table(desc)
        out = np.zeros(len(t), dtype=RESULT_DTYPE)
        _check(lib().zmc_udf_integrate(ctx, self.handle, t.ctypes.data, len(t), out.ctypes.data),
               "zmc_udf_integrate")
        return out

    def eval_samples(self, ctx: int, row, s_begin: int, count: int) -> np.ndarray:
        t = _table(np.asarray(row).reshape(1))
        out = np.zeros(count, dtype=np.float32)
        _check(lib().zmc_udf_eval_samples(ctx, self.handle, t.ctypes.data, s_begin, count,
                                          out.ctypes.data), "zmc_udf_eval_samples")
        return out

    def normal_integrate(self, ctx: int, lo, hi, p, opts: zmc_normal_opts) -> dict:
        """Stratified sampling with tree refinement over the box [lo, hi]."""
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        pp = np.zeros(40)
        pv = np.asarray(p, dtype=np.float64).reshape(-1)
        pp[:len(pv)] = pv
        assert len(lo) == len(hi) == self.dim
        r = zmc_normal_result()
        _check(lib().zmc_normal_integrate_udf(ctx, self.handle, lo.ctypes.data, hi.ctypes.data,
                                              pp.ctypes.data, ctypes.byref(opts),
                                              ctypes.byref(r)), "zmc_normal_integrate_udf")
        return _normal_dict(r)

    def close(self):
        if self.handle:
            lib().zmc_udf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A library context whose device memory and stream come from PyTorch.

    ``arena_bytes`` of device memory are taken from PyTorch's caching allocator
    (one uint8 tensor kept alive by this object) and the library runs on
    ``stream`` (default: a new ``torch.cuda.Stream``).
    """

    def __init__(self, arena_bytes: int = 1 << 30, device: int = 0, stream=None,
                 serving: bool = False, quints_per_lane: int = 0,
                 max_chunks_per_iter: int = 0, serving_share: int = 0,
                 serving_cut_backlog: int = 0,
                 use_torch_memory: bool = True, autotune: bool | int = False,
                 tune_cache_path: str | None = None):
        import torch

        self.torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        opt = zmc_default_options()
        opt.mem_budget_bytes = arena_bytes
        opt.device = device
        opt.stream = self.stream.cuda_stream
        opt.serving = 1 if serving else 0
        opt.quints_per_lane = quints_per_lane
        opt.max_chunks_per_iter = max_chunks_per_iter
        opt.serving_share = serving_share
        opt.serving_cut_backlog = serving_cut_backlog
        # True: launch geometry only; an int: ZMC_TUNE_* flags
        opt.autotune = (ZMC_TUNE_GEOMETRY if autotune is True
                        else int(autotune) if autotune else 0)
        self._tune_path = tune_cache_path.encode() if tune_cache_path else None
        opt.tune_cache_path = self._tune_path
        self.arena = None
        if use_torch_memory:
            self.arena = torch.empty(arena_bytes + 256, dtype=torch.uint8,
                                     device=f"cuda:{device}")
            base = self.arena.data_ptr()
            opt.arena = (base + 255) & ~255
        self.handle = zmc_create(opt)

    def close(self):
        if self.handle:
            zmc_destroy(self.handle)
            self.handle = None
            self.arena = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
