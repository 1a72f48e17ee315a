"""The fused kernels' source built for the host (CUDA qualifiers mapped to
plain C++, each kernel run over its launch grid one thread at a time): the
z-marching 3x3x3 max and mean of the viscosity (k_nu_maxsmooth) equals the two
gather kernels it replaces bit for bit.  This checks the march's windows and
halo planes on the CPU, beyond the GPU tests' FP32 tolerance."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def test_nu_maxsmooth_equals_max_then_smooth(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "nu_maxsmooth")
    src = os.path.join(HERE, "host_emulation", "nu_maxsmooth.cpp")
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CUDA_INC, "-o", exe, src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    assert r.stdout.count("0 differing values") == 6, r.stdout
