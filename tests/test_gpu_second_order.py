"""GPU parity of the second-order switch of the viscous stress (Sect.
Equations, do_2nddiv with d2lnr_lim), reading R18: against the FP64 oracle on
states where about half the cells are flagged.

The flag is an integer decided from floating point (|D2 ln rho|, |D2 ln e|
against the limit).  The limit is set in the middle of the widest gap between
the oracle's values near their median, so that FP32 and FP64 take the same
decision in every cell (the gap is far wider than FP32 rounding)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import stagger as OS
import workloads as inputs

from test_gpu_parity import (VISC_KW, err_group, err_max, err_scale, make, oracle_params,
                             ragged_state)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    return S


def sharp_state(shape, seed=7):
    """A ragged random state whose ln rho and ln e carry short-wavelength
    bumps, so that |D2 ln rho| and |D2 ln e| spread over 0 .. 0.7."""
    w = ragged_state(shape, seed)
    nx, ny, nz = shape
    f = [np.array(a) for a in w.fields]
    bump_x = np.exp(0.8 * np.sin(2 * np.pi * 3 * np.arange(nx) / nx)).reshape(1, 1, nx)
    bump_y = np.exp(0.5 * np.cos(2 * np.pi * 2 * np.arange(ny) / ny)).reshape(1, ny, 1)
    f[0] = f[0] * bump_x
    f[4] = f[4] * bump_x * bump_y
    return inputs.Workload("sharp", shape, w.spacing, f)


def gap_limit(fields):
    """Middle of the widest gap between the oracle's max(|D2 ln rho|, |D2 ln e|)
    values (all axes) within 400 values of their median, and that gap."""
    r, E = torch.tensor(fields[0]), torch.tensor(fields[4])
    lr, le = torch.log(r), torch.log(E / r)
    vals = []
    for ax in "xyz":
        d2r = OS._s(lr, ax, 1) - 2.0 * lr + OS._s(lr, ax, -1)
        d2e = OS._s(le, ax, 1) - 2.0 * le + OS._s(le, ax, -1)
        vals.append(torch.maximum(d2r.abs(), d2e.abs()).flatten())
    v = np.sort(torch.cat(vals).numpy())
    i0 = max(len(v) // 2 - 200, 0)
    seg = v[i0:i0 + 400]
    j = int(np.argmax(np.diff(seg)))
    return 0.5 * (seg[j] + seg[j + 1]), seg[j + 1] - seg[j]


SHAPES = [(20, 12, 9), (21, 10, 7)]     # four-cell threads; one-cell threads (nx % 4 != 0)


def _setup(shape, **extra):
    w = sharp_state(shape)
    lim, gap = gap_limit(w.fields)
    assert gap > 1e-5, gap
    kw = dict(VISC_KW, c1=-1.0 / 3.0, do_2nddiv=1, d2lnr_lim=float(lim), **extra)
    return w, kw


@pytest.mark.parametrize("shape", SHAPES)
def test_second_order_switch_rhs(S, shape):
    w, kw = _setup(shape)
    g = oracle.Grid(*w.shape, *w.spacing)
    f64 = [torch.tensor(a) for a in w.fields]
    P = OS.rhs_parts(f64, g, oracle_params(kw))
    frac = float(sum(P["d2flags"][a].double().mean() for a in "xyz") / 3)
    assert 0.2 < frac < 0.8, frac
    Fo = [P[k].numpy() for k in ("d_r", "d_px", "d_py", "d_pz", "d_E", "d_Bx", "d_By", "d_Bz")]
    # The switch changes the answer far beyond the tolerance.
    Foff = [t.numpy() for t in oracle.rhs(f64, g, oracle_params(dict(kw, do_2nddiv=0)))]
    assert max(err_scale(Foff, Fo)) > 1e-2
    for sc in (0, 1):
        sim, refs, dev = make(S, w, dict(kw, scalar_cells=sc))
        F = sim.rhs(dev)
        Fu = sim.rhs_unfused(dev)
        d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
        F64 = sim.rhs_unfused_f64(d64)
        torch.cuda.synchronize()
        e = err_scale([t.double().cpu().numpy() for t in F], Fo)
        eu = err_scale([t.double().cpu().numpy() for t in Fu], Fo)
        e64 = err_scale([t.cpu().numpy() for t in F64], Fo)
        assert max(e) < 2e-4, (shape, sc, e)
        assert max(eu) < 2e-4, (shape, sc, eu)
        assert max(e64) < 1e-10, (shape, sc, e64)
        sim.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_second_order_switch_steps(S, shape):
    w, kw = _setup(shape)
    sim, refs, dev = make(S, w, kw)
    g = oracle.Grid(*w.shape, *w.spacing)
    po = oracle_params(kw)
    fo = [torch.tensor(a) for a in w.fields]
    for _ in range(3):
        dt = sim.step(dev, None, want_dt=True)
        fo, dto = oracle.step(fo, g, po, dt=dt)
        assert abs(dt / dto - 1) < 1e-4, (dt, dto)
    e = err_group(S.join_state(dev, refs), [t.numpy() for t in fo])
    assert max(e) < 3e-5, (shape, e)
    sim.close()


def test_second_order_switch_adjoint_fp64(S):
    w, kw = _setup((13, 11, 9))
    sim, refs, dev = make(S, w, kw)
    g = oracle.Grid(*w.shape, *w.spacing)
    f64 = [torch.tensor(a) for a in w.fields]
    dt = 2e-4
    gen = torch.Generator().manual_seed(1)
    lam = [torch.randn(t.shape, generator=gen, dtype=torch.float64) for t in f64]
    ref = [t.numpy() for t in oracle.step_adjoint(f64, dt, lam, g, oracle_params(kw))]
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
    out64 = sim.step_adjoint_f64(d64, dt, [l.cuda() for l in lam])
    torch.cuda.synchronize()
    e64 = err_max([t.cpu().numpy() for t in out64], ref)
    assert max(e64) < 1e-10, e64
    sim.close()
