import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


@pytest.fixture(scope="session")
def torch_philox(tmp_path_factory):
    """Callable (seed, subsequence, offset) triples -> words, backed by PyTorch's
    header-only ``at::philox_engine`` compiled for the host."""
    import numpy as np
    import torch

    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    exe = str(tmp_path_factory.mktemp("tpd") / "torch_philox_dump")
    src = os.path.join(ROOT, "tests", "helpers", "torch_philox_dump.cpp")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe], check=True)

    def run(triples):
        text = "\n".join(f"{int(s)} {int(q)} {int(o)}" for s, q, o in triples) + "\n"
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True)
        return np.array([[int(v) for v in line.split()] for line in out.stdout.splitlines()],
                        dtype=np.uint32).reshape(-1, 4)

    return run


@pytest.fixture(scope="session")
def zctx():
    """A library context on cuda:0 (device memory and stream from PyTorch)."""
    import torch

    from paper_2104_10073_gb300 import build, zmc

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    ctx = zmc.Context(arena_bytes=4 << 30)
    yield ctx
    ctx.close()


@pytest.fixture(scope="session")
def sq_ctx(zctx):
    """A blocking context with a serving context's chunk length, whose results
    can be compared bit for bit with served ones."""
    from paper_2104_10073_gb300 import zmc

    ctx = zmc.Context(arena_bytes=2 << 30, quints_per_lane=zmc.SERVING_QUINTS_PER_LANE)
    yield ctx
    ctx.close()


@pytest.fixture(scope="session")
def curand_philox(tmp_path_factory):
    """Callable (ctr (n,4), key (n,2)) -> words, backed by cuRAND's device Philox."""
    import numpy as np

    exe = str(tmp_path_factory.mktemp("cpd") / "curand_philox_dump")
    src = os.path.join(ROOT, "tests", "helpers", "curand_philox_dump.cu")
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", src, "-o", exe],
                   check=True)

    def run(ctr, key):
        lines = [" ".join(str(int(v)) for v in list(c) + list(k)) for c, k in zip(ctr, key)]
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True)
        return np.array([[int(v) for v in ln.split()] for ln in out.stdout.splitlines()],
                        dtype=np.uint32).reshape(-1, 4)

    return run
