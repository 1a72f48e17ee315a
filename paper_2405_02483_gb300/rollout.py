"""Differentiable multi-step rollout: torch.autograd.Function over the
library's fixed-dt step and its adjoint, with checkpoints every k steps and
recomputation in between (the reverse sweep holds at most k + 1 states)."""
from __future__ import annotations

import torch


class StaggerRollout(torch.autograd.Function):
    """y = step^n(x) for 8 FP32 CUDA deviation fields x.

    apply(sim, dts, k, *state) with dts a list of per-step time steps (> 0,
    frozen: the adjoint does not differentiate the Courant condition) and k
    the checkpoint interval.  Returns the 8 output fields."""

    @staticmethod
    def forward(ctx, sim, dts, k, *state):
        k = max(1, int(k))
        cur = [t.detach().clone().contiguous() for t in state]
        ckpts = []
        for i, dt in enumerate(dts):
            if i % k == 0:
                ckpts.append([t.clone() for t in cur])
            sim.step(cur, float(dt))
        ctx.sim = sim
        ctx.dts = [float(d) for d in dts]
        ctx.k = k
        ctx.ckpts = ckpts
        return tuple(cur)

    @staticmethod
    def backward(ctx, *grads):
        sim, dts, k = ctx.sim, ctx.dts, ctx.k
        lam = [(g if g is not None else torch.zeros_like(c)).contiguous().float()
               for g, c in zip(grads, ctx.ckpts[0])]
        nseg = len(ctx.ckpts)
        for s in range(nseg - 1, -1, -1):
            i0 = s * k
            i1 = min(i0 + k, len(dts))
            states = [[t.clone() for t in ctx.ckpts[s]]]
            for i in range(i0, i1 - 1):
                nxt = [t.clone() for t in states[-1]]
                sim.step(nxt, dts[i])
                states.append(nxt)
            for i in range(i1 - 1, i0 - 1, -1):
                lam = sim.step_adjoint(states[i - i0], dts[i], lam)
        return (None, None, None, *lam)


def rollout(sim, state, dts, k=8):
    """Differentiable rollout (see StaggerRollout)."""
    return StaggerRollout.apply(sim, list(dts), k, *state)
