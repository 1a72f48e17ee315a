"""Floating-point operation count per zone per RK3 step, taken from the FP64
oracle's own operator list.

Every aten operation the oracle executes during one Courant step is counted
by its number of output (or, for reductions, input) elements:
  arith   add, sub, mul, div, neg, reciprocal (one flop per element; a fused
          multiply-add on the GPU is two of these)
  select  abs, maximum, minimum, clamp, where, comparisons (one ALU op each)
  transc  exp, log, log1p, sqrt, pow with a non-integer exponent (one special
          function each; counted apart from the flops)
Data movement (roll, copies, casts) counts nothing.  The counts divided by
the number of cells are the algorithmic operation counts per zone per step of
the workloads below; they do not depend on the grid size beyond the few
reductions of the Courant step.

Run from the repository root:  python tests/golden/count_flops.py
It writes tests/golden/flops_per_zone.json; it calls only oracle/.
"""
from __future__ import annotations

import json
import os
import sys

import torch
from torch.utils._python_dispatch import TorchDispatchMode

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "flops_per_zone.json")

ARITH = {"add", "sub", "mul", "div", "neg", "reciprocal", "rsub"}
SELECT = {"abs", "maximum", "minimum", "clamp", "clamp_min", "clamp_max", "where", "gt", "lt",
          "ge", "le", "eq", "ne", "max", "min", "amax", "amin", "logical_not", "logical_or",
          "bitwise_or", "bitwise_not", "isfinite"}
TRANSC = {"exp", "log", "log1p", "sqrt", "rsqrt"}
REDUCE = {"sum", "mean"}           # n - 1 additions (+1 division for mean) per reduction
FREE = {"roll", "clone", "copy_", "_to_copy", "detach", "view", "reshape", "alias", "t",
        "lift_fresh", "zeros_like", "full_like", "empty_like", "ones_like", "zeros", "full",
        "scalar_tensor", "expand", "slice", "select", "unsqueeze", "squeeze", "_unsafe_view",
        "as_strided", "empty", "fill_", "zero_", "resize_", "item", "_local_scalar_dense",
        "lift_fresh_copy", "permute", "contiguous", "index", "cat", "stack", "clone"}


class Counter(TorchDispatchMode):
    def __init__(self):
        super().__init__()
        self.c = {"arith": 0, "select": 0, "transc": 0}
        self.unknown = set()

    def __torch_dispatch__(self, func, types, args=(), kwargs=None):
        kwargs = kwargs or {}
        out = func(*args, **kwargs)
        name = func.overloadpacket.__name__.rstrip("_")
        t = out if torch.is_tensor(out) else (out[0] if isinstance(out, (tuple, list)) and out
                                              and torch.is_tensor(out[0]) else None)
        n = t.numel() if t is not None else 0
        if name in ARITH:
            self.c["arith"] += n
        elif name == "pow":
            e = args[1] if len(args) > 1 else kwargs.get("exponent")
            if isinstance(e, (int, float)) and float(e) == 2.0:
                self.c["arith"] += n                    # a square: one multiply
            else:
                self.c["transc"] += n
        elif name in SELECT:
            if name in ("max", "min", "amax", "amin") and t is not None and t.numel() == 1:
                self.c["select"] += max(args[0].numel() - 1, 0)   # a full reduction
            else:
                self.c["select"] += n
        elif name in TRANSC:
            self.c["transc"] += n
        elif name in REDUCE:
            self.c["arith"] += args[0].numel()
        elif name not in FREE:
            self.unknown.add(name)
        return out


def count(workload: str, n: int = 12):
    """Operation counts per zone of one Courant RK3 step of a workload:
    'turbulence' (Richtmyer-Morton viscosity, energy diffusion, resistivity,
    quench: the benchmark's physics) or 'ideal' (all diffusion off)."""
    import oracle
    import workloads
    w = workloads.turbulence(n)
    g = oracle.Grid(*w.shape, *w.spacing)
    if workload == "turbulence":
        p = oracle.Params(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=True)
    elif workload == "ideal":
        p = oracle.Params()
    else:
        raise ValueError(workload)
    f = [torch.tensor(a) for a in w.fields]
    with Counter() as c:
        oracle.step(f, g, p)
    cells = n ** 3
    res = {k: v / cells for k, v in c.c.items()}
    res["flops"] = res["arith"] + res["select"]
    return res, sorted(c.unknown)


def main():
    data = {"_source": "tests/golden/count_flops.py: aten operations of one Courant RK3 step of "
                       "the FP64 oracle (oracle.step) on a 12^3 box, per zone",
            "_units": "operations per zone per full RK3 step (three right-hand sides, the "
                      "Courant step and the updates)"}
    for wl in ("turbulence", "ideal"):
        res, unknown = count(wl)
        if unknown:
            raise SystemExit("uncounted operations: %s" % unknown)
        data[wl] = {k: round(v, 3) for k, v in res.items()}
    with open(OUT, "w") as fh:
        json.dump(data, fh, indent=1)
        fh.write("\n")
    print(json.dumps(data, indent=1))


if __name__ == "__main__":
    main()
