"""CPU checks of the digit arithmetic behind WVL_F64_EMU (the tensor-core
FP64 passes): the digit split, the accumulator schedule of every filter of
the method, and one window evaluated in integer arithmetic exactly as the
kernels do, against a long-double convolution.  The C++ check program
(tests/emu_host_check.cpp) includes the library's own header and links the
library for its filters."""
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


def test_emu_digit_arithmetic():
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    import paper_0904_1543_gb300 as W
    W.lib()                                   # builds libwvl.so if needed
    pkg = os.path.join(ROOT, "paper_0904_1543_gb300")
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "emu_host_check")
        cmd = [cxx, "-O2", "-std=c++17", "-I", os.path.join(pkg, "csrc"),
               "-I", os.path.join(ROOT, "include"), "-I", inc,
               os.path.join(HERE, "emu_host_check.cpp"), "-o", exe,
               "-L", pkg, "-lwvl", f"-Wl,-rpath,{pkg}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and "OK" in r.stdout, r.stdout[-3000:] + r.stderr[-2000:]
