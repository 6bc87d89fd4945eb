"""Build ``libzmc.so`` (the C ABI library) in-tree with nvcc for sm_103a.

The translation units (one per integrand family's sampling path and quint-loop
unroll, the plain form, the shared kernels, the host runtime, serving, the
allocation-free entry point, the tuning cache) compile in parallel and link into
one shared library with the CUDA runtime linked statically, so the library needs
only the NVIDIA driver at run time.  Output:
``paper_2104_10073_gb300/libzmc.so``.  Rebuilds only when a source is newer.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "libzmc.so")
BUILD = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FAMILY_SOURCES = ["zmc_fam_harmonic.cu", "zmc_fam_abslin.cu", "zmc_fam_gauss.cu",
                  "zmc_fam_poly.cu"]
SOURCES = [*FAMILY_SOURCES, "zmc_plain.cu", "zmc_kernels.cu", "zmc_runtime.cpp",
           "zmc_serving.cpp", "zmc_noalloc.cu", "zmc_tune.cpp", "zmc_udf.cpp", "zmc_normal.cpp",
           "zmc_pool.cpp", "zmc_polyroots.cpp"]
UNROLLS = (1, 2)  # each family file is compiled once per quint-loop unroll
HEADERS = ["zmc_internal.h", "zmc_runtime.h", "zmc_coeffs.h", "zmc_device.cuh",
           "zmc_udf_kernel.cuh", "zmc_udf_layout.h"]
# Headers whose text zmc_udf.cpp hands to NVRTC (symbol name, path).
JIT_HEADERS = [("kJitZmcH", os.path.join(INCLUDE, "zmc.h")),
               ("kJitZmcInternalH", os.path.join(CSRC, "zmc_internal.h")),
               ("kJitZmcDeviceCuh", os.path.join(CSRC, "zmc_device.cuh")),
               ("kJitZmcUdfKernelCuh", os.path.join(CSRC, "zmc_udf_kernel.cuh")),
               ("kJitZmcUdfLayoutH", os.path.join(CSRC, "zmc_udf_layout.h"))]


def _units():
    """(source, object stem, extra flags) of every translation unit."""
    units = []
    for src in SOURCES:
        stem = os.path.splitext(src)[0]
        if src in FAMILY_SOURCES:
            # -fmad=false: no multiply-add is fused unless the source says fmaf, so
            # the sampling arithmetic is exactly as written whatever the unroll
            units += [(src, f"{stem}_u{u}", [f"-DZMC_FAM_UNROLL={u}", "-fmad=false"])
                      for u in UNROLLS]
        else:
            units.append((src, stem, []))
    return units


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _flags(extra=()):
    # ZMC_NVCC_DEFINES: optional space-separated -D tuning knobs (launch bounds,
    # multiply form) for sweeps; the defaults are the tuned values.
    defs = os.environ.get("ZMC_NVCC_DEFINES", "").split()
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
            "-I", CSRC, "-I", BUILD, *defs, *extra]


def _write_jit_sources() -> None:
    """_build/zmc_jit_sources.h: the headers of the run-time compiled path as
    C string constants (raw literals, one per header)."""
    out = ["// Generated by build.py from the headers named below; do not edit.", "#pragma once"]
    for sym, path in JIT_HEADERS:
        text = open(path).read()
        assert ')zmcjit"' not in text
        out.append(f"// {os.path.relpath(path, ROOT)}")
        out.append(f'static const char {sym}[] = R"zmcjit({text})zmcjit";')
    data = "\n".join(out) + "\n"
    path = os.path.join(BUILD, "zmc_jit_sources.h")
    if not os.path.exists(path) or open(path).read() != data:
        with open(path, "w") as f:
            f.write(data)


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(INCLUDE, "zmc.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def _flags_stamp() -> str:
    """The compile flags the library was last built with (tuning knobs included)."""
    return os.path.join(BUILD, "flags.txt")


def build(force: bool = False, verbose: bool = False) -> str:
    flags = " ".join(_flags())
    stamp = _flags_stamp()
    same_flags = os.path.exists(stamp) and open(stamp).read() == flags
    if (not force and same_flags and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= _newest_input()):
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    _write_jit_sources()
    nvcc = _nvcc()

    def compile_one(unit):
        src, stem, extra = unit
        obj = os.path.join(BUILD, stem + ".o")
        cmd = [nvcc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd.insert(1, "-Xptxas=-v" if verbose else "-Xptxas=-O3")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    units = _units()
    # the slowest unit (the polynomial family) first, so it overlaps the rest
    units.sort(key=lambda u: u[0] != "zmc_fam_poly.cu")
    with ThreadPoolExecutor(max_workers=len(units)) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-cudart", "static", *objs, "-o", tmp,
           "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    with open(stamp, "w") as f:
        f.write(flags)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
