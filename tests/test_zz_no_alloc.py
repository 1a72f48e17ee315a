"""stagger_diagnostics_noalloc: the diagnostics entry point for callers that
cannot allocate device memory (a memory pool that owns the whole device, a
monitoring tool that must leave the footprint of the run unchanged, code with
no library context).  It keeps its scratch in a fixed array of the library's
device image.  Checked through the C ABI against stagger_diagnostics on two
calls in a row, including a second state, so nothing stale carries over from
the shared scratch.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    return S


def _noalloc(S, sim, state):
    out = (ctypes.c_double * 10)()
    rc = S.lib.stagger_diagnostics_noalloc(ctypes.byref(sim.grid), ctypes.byref(sim.params),
                                           S._dev(state), out,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, list(out)


def _close(a, b):
    # The same FP64 partials summed in another order: each sum agrees to
    # 1e-12 of the largest sum (sum rho); max |div B| and the non-finite
    # count do not depend on the order and must be equal.
    scale = max(abs(b[0]), abs(b[4]), 1.0)
    for i in (0, 1, 2, 3, 4, 5, 6, 8):
        assert abs(a[i] - b[i]) <= 1e-12 * scale, (i, a[i], b[i])
    assert a[7] == b[7] and a[9] == b[9]


def test_noalloc_diagnostics_match_twice(S):
    import workloads as inputs
    w = inputs.orszag_tang_3d(48)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, nu1=0.04, nu2=1.0, nu3=0.04,
                                                     do_quench=1))
    ref1 = sim.diagnostics(dev)
    rc, a = _noalloc(S, sim, dev)
    assert rc == S.OK
    _close(a, ref1)
    # Second call in a row on a different state: the shared scratch must not
    # leak the first call's values.
    sim.step(dev, None)
    ref2 = sim.diagnostics(dev)
    rc, b = _noalloc(S, sim, dev)
    assert rc == S.OK
    _close(b, ref2)
    assert a != b
    sim.close()


def test_noalloc_rejects_grids_beyond_its_scratch(S):
    g = S.Grid(512, 512, 512, 1 / 512, 1 / 512, 1 / 512)
    p = S.default_params()
    dummy = torch.zeros(8, device="cuda")
    ptrs = S.P8F(*[ctypes.cast(dummy.data_ptr(), ctypes.POINTER(ctypes.c_float))] * 8)
    out = (ctypes.c_double * 10)()
    assert S.lib.stagger_diagnostics_noalloc(ctypes.byref(g), ctypes.byref(p), ptrs, out, None) == S.EINVAL
    g = S.Grid(256, 256, 256, 1 / 256, 1 / 256, 1 / 256)   # exactly at the limit: accepted sizes
    big = [torch.ones(256, 256, 256, device="cuda") for _ in range(8)]
    p = S.default_params()
    rc = S.lib.stagger_diagnostics_noalloc(ctypes.byref(g), ctypes.byref(p), S._dev(big), out, None)
    torch.cuda.synchronize()
    assert rc == S.OK and out[0] == pytest.approx(256 ** 3)
