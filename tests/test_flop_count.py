"""The stored operation counts per zone per step (tests/golden/flops_per_zone.json,
written by tests/golden/count_flops.py from the oracle's operator list) are
current, every operation the oracle executes is classified, and the counts
meet the hand counts of pieces whose arithmetic is fixed by the paper."""
import importlib.util
import json
import os

import pytest
import torch

HERE = os.path.dirname(os.path.abspath(__file__))


def _mod():
    spec = importlib.util.spec_from_file_location("count_flops",
                                                  os.path.join(HERE, "golden", "count_flops.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


@pytest.mark.parametrize("workload", ["turbulence", "ideal"])
def test_stored_counts_are_current(workload):
    m = _mod()
    stored = json.load(open(os.path.join(HERE, "golden", "flops_per_zone.json")))[workload]
    res, unknown = m.count(workload)
    assert not unknown, unknown
    for k in ("arith", "select", "transc", "flops"):
        assert res[k] == pytest.approx(stored[k], abs=2e-3), (k, res[k], stored[k])


def test_counter_on_operators_of_known_cost():
    """eq. (interp) costs 3 additions + 3 multiplies + 2 additions = 8 flops
    per point, eq. (deriv) 3 subtractions + 3 multiplies + 2 additions + 1
    division = 9; the RK update f + b dt q one multiply-add per field."""
    import oracle
    m = _mod()
    f = torch.rand(4, 5, 6, dtype=torch.float64)
    with m.Counter() as c:
        oracle.up(f, "x")
    assert c.c["arith"] == 8 * f.numel() and c.c["select"] == 0
    with m.Counter() as c:
        oracle.ddup(f, "y", 0.1)
    assert c.c["arith"] == 9 * f.numel()
    with m.Counter() as c:
        oracle.max3(f, "z")
    assert c.c["select"] == 2 * f.numel() and c.c["arith"] == 0
