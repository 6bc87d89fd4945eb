"""The autotuner's JSON cache, on the host (CPU only): every entry, geometry or
chunk length and unroll, survives a load / store / reload round trip, malformed
entries and files of the older format are skipped, and the geometry key names
the chunk length, the unroll and the family kernel's registers per thread (its
build)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    path = str(tmp_path_factory.mktemp("tune") / "rt")
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2104_10073_gb300", "csrc"), "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "helpers", "tune_cache_roundtrip.cpp"),
                    os.path.join(ROOT, "paper_2104_10073_gb300", "csrc", "zmc_tune.cpp"),
                    "-o", path], check=True)
    return path


def _run(exe, tmp_path, text):
    src = tmp_path / "in.json"
    src.write_text(text)
    out = subprocess.run([exe, str(src), str(tmp_path / "out.json")], capture_output=True,
                         text=True, check=True).stdout.splitlines()
    return out[:-1], out[-1]


def test_cache_round_trip(exe, tmp_path):
    entries, key = _run(exe, tmp_path, '{"version": 2, "entries": {\n'
                        '  "G|152|0|q104|u1|4|r128": {"block": 256, "blocks_per_sm": 2, "ms": 2.0},\n'
                        '  "G|152|1|q104|u2|6|r126": {"block": 128, "blocks_per_sm": 4, "ms": 0.7},\n'
                        '  "bad|1|1|1|1": {"block": 96, "blocks_per_sm": 2, "ms": 1.0},\n'
                        '  "chunk|G|152|m1": {"quints": 208, "unroll": [1, 2, 1, 2], "ms": 4.5},\n'
                        '  "chunk|bad|q": {"quints": 100, "unroll": [1, 1, 1, 1], "ms": 4.5},\n'
                        '  "chunk|bad|u": {"quints": 26, "unroll": [1, 3, 1, 1], "ms": 4.5},\n'
                        '  "G|152|3|q104|u1|7|r128": {"block": 128, "blocks_per_sm": 4}\n'
                        '}}\n')
    assert key == "key: GPU X|10|2|q16|u2|5|r115"
    assert sorted(entries) == sorted(["G|152|0|q104|u1|4|r128 256 2",
                                      "G|152|1|q104|u2|6|r126 128 4",
                                      "G|152|3|q104|u1|7|r128 128 4",
                                      "chunk|G|152|m1 q208 u1212",
                                      "GPU X|10|2|q16|u1|5|r115 128 3",
                                      "chunk|GPU X|10|m5 q52 u1211"])


def test_older_format_is_retuned(exe, tmp_path):
    entries, _ = _run(exe, tmp_path, '{"version": 1, "entries": {\n'
                      '  "NVIDIA GB300|152|0|16|4": {"block": 256, "blocks_per_sm": 2, "ms": 2.0}\n'
                      '}}\n')
    assert sorted(entries) == sorted(["GPU X|10|2|q16|u1|5|r115 128 3",
                                      "chunk|GPU X|10|m5 q52 u1211"])
