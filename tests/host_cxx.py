"""Compiles the host-only C++ test drivers under tests/ against the library's
host sources with g++ (no GPU, no nvcc: the drivers use only host code)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1312_5561_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def compile_driver(main_cpp, sources, out, csrc=CSRC):
    """g++ -fopenmp tests/<main_cpp> + csrc/<sources> -> out; skips the test
    when g++ or the CUDA runtime headers (included by the library's internal
    header) are missing."""
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("needs g++ and the CUDA runtime headers")
    cmd = ["g++", "-O2", "-fopenmp", "-std=c++17", "-I", csrc, "-I", os.path.join(ROOT, "include"), "-I", inc,
           os.path.join(ROOT, "tests", main_cpp), *[os.path.join(csrc, s) for s in sources], "-o", str(out)]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    return str(out)
