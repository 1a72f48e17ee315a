"""The fused kernels' source built for the host (CUDA qualifiers mapped to
plain C++, each kernel run over its launch grid one thread at a time), checked
bit for bit on the CPU, beyond the GPU tests' FP32 tolerance:
- the z-marching 3x3x3 max and mean of the viscosity (k_nu_maxsmooth) equals
  the two gather kernels it replaces (the march's windows and halo planes);
- the Courant maxima taken inside the stage-1 kernels (k_nu_raw, k_nu_maxsmooth,
  the mass and energy k_div) equal those of the separate pass k_courant_part
  (the block reductions and the per-cell formulas);
- the right-hand side formed with one cell per thread equals the one formed
  with four x-cells per thread, for the benchmark's physics and for every
  option at once, on a uniform and on a stretched z mesh;
- the op graph with its merged nodes (stencil pairs and sums, folded sums and
  scalings), with one-cell and with four-x-cell kernels, gives the same
  forward values bit for bit as the graph of one node per primitive, and a
  reverse sweep equal to rounding, in FP64 and FP32."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def _build_and_run(tmp_path, name):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / name)
    src = os.path.join(HERE, "host_emulation", name + ".cpp")
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CUDA_INC, "-o", exe, src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    return r.stdout


def test_nu_maxsmooth_equals_max_then_smooth(tmp_path):
    out = _build_and_run(tmp_path, "nu_maxsmooth")
    assert out.count("0 differing values") == 6, out


def test_courant_maxima_in_stage_kernels_equal_separate_pass(tmp_path):
    out = _build_and_run(tmp_path, "courant_fused")
    assert out.count(", 0 differing") == 5, out


def test_one_cell_and_four_cell_threads_give_the_same_rhs(tmp_path):
    out = _build_and_run(tmp_path, "rhs_mappings")
    assert out.count(" 0 differing values, 0 non-finite") == 16, out


def test_merged_op_graph_equals_one_node_per_primitive(tmp_path):
    out = _build_and_run(tmp_path, "graph_fusion")
    assert out.count("forward 0 differing values, 0 non-finite") == 16, out
    assert "FAIL" not in out, out
    # the four-x-cell kernels ran on the boxes whose nx is a multiple of 4
    import re
    four = [int(m) for m in re.findall(r"four-cell \((\d+) four-cell launches\)", out)]
    assert len(four) == 8 and sum(1 for f in four if f > 0) == 6, out
    # the merges keep taking out more than a third of the nodes (the
    # adjoint's launches and arrays scale with them; 39-43% now)
    for a, b in re.findall(r": (\d+) -> (\d+) nodes", out):
        assert int(b) <= 0.65 * int(a), (a, b)
