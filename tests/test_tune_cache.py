"""The autotuner's JSON cache, on the host (CPU only): every entry survives a
load / store / reload round trip, malformed entries are skipped, and the key
names the family kernel's registers per thread (its build)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cache_round_trip(tmp_path):
    exe = str(tmp_path / "rt")
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2104_10073_gb300", "csrc"), "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "helpers", "tune_cache_roundtrip.cpp"),
                    os.path.join(ROOT, "paper_2104_10073_gb300", "csrc", "zmc_tune.cpp"),
                    "-o", exe], check=True)
    src = tmp_path / "in.json"
    src.write_text('{"version": 1, "entries": {\n'
                   '  "NVIDIA GB300|152|0|16|4": {"block": 256, "blocks_per_sm": 2, "ms": 2.0},\n'
                   '  "NVIDIA GB300|152|1|16|6": {"block": 128, "blocks_per_sm": 4, "ms": 0.7},\n'
                   '  "bad|1|1|1|1": {"block": 96, "blocks_per_sm": 2, "ms": 1.0},\n'
                   '  "NVIDIA GB300|152|3|16|7": {"block": 128, "blocks_per_sm": 4}\n'
                   '}}\n')
    out = subprocess.run([exe, str(src), str(tmp_path / "out.json")], capture_output=True,
                         text=True, check=True).stdout.splitlines()
    assert out[-1] == "key: GPU X|10|2|16|5|r115"
    out = out[:-1]
    assert sorted(out) == sorted(["NVIDIA GB300|152|0|16|4 256 2",
                                  "NVIDIA GB300|152|1|16|6 128 4",
                                  "NVIDIA GB300|152|3|16|7 128 4",
                                  "GPU X|10|2|16|5 128 3"])
