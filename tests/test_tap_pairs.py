"""CPU check of the packed FP32 convolution form: the tap pairs that let one
packed FMA update two outputs (csrc/taps.h) give every output exactly the
taps of the scalar form, for every filter kind and chunk width
(tests/tap_pairs_check.cpp, compiled with g++ against the library's header)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime_api.h")):
            return os.path.join(d, "include")
    return None


def test_tap_pairs_reproduce_scalar_taps():
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    csrc = os.path.join(ROOT, "paper_0904_1543_gb300", "csrc")
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "tap_pairs_check")
        cmd = [cxx, "-O1", "-std=c++17", "-I", csrc, "-I", os.path.join(ROOT, "include"),
               "-I", inc, os.path.join(HERE, "tap_pairs_check.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
        assert r.returncode == 0 and "OK" in r.stdout, r.stdout[-3000:] + r.stderr[-2000:]
