"""Rigid z walls (Sect. "Boundary Conditions", "Rigid"; reading R25) on the
GPU against the FP64 oracle.

The GPU keeps STAGGER_ZGHOST_MIN ghost planes at each end of its arrays; the
ghost values of rho, E and B are the caller's and stay as they are, and the
ghost momenta are set from the boundary planes' velocity before every use of
a state.  Right-hand sides are compared on the physical planes with the
tolerance of the other RHS tests (2e-4 of the term scale plus ten FP32
floors) and are zero on the ghost planes; three Courant steps to 5e-5 of each
field group on every plane, the ghost rho, E and B unchanged bit for bit; the
Courant step to 1e-5; the diagnostics to 1e-6; a discretely balanced
isothermal atmosphere stays at rest to FP32 roundoff over 20 steps (2e-6 of
rho c_s).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as inputs
from oracle.stagger import DA, DB, DC
from test_gpu_parity import K_FLOOR, U32, VISC_KW, err_group, oracle_params, scale_of
from test_oracle_rigid import rigid_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    return S


CASES = {
    "ideal_20x12x10": ((20, 12, 10), {}),
    "viscous_quench_gravity_36x9x12": ((36, 9, 12), dict(VISC_KW, g=(0.0, 0.0, -1.0))),
    "const_nu_c1_gravity_13x8x9": ((13, 8, 9), dict(nu_const=0.003, c1=-1 / 3, nuE=0.5, nuB=0.7,
                                                    g=(0.1, 0.0, -1.0))),
    "lnp_aver_cooling_gravity_24x10x8": ((24, 10, 8), dict(VISC_KW, lnp_aver=1, t_cool=0.05,
                                                          e_cool=0.7, rho_cool=1.02, cool_cut=1,
                                                          g=(0.0, 0.0, -1.0))),
    "second_order_ediffav_16x8x11": ((16, 8, 11), dict(VISC_KW, do_2nddiv=1, d2lnr_lim=-1.0,
                                                      ediffav=1)),
    # the thinnest box allowed: two physical planes between the ghost layers
    "thinnest_viscous_gravity_12x8x1": ((12, 8, 1), dict(VISC_KW, g=(0.0, 0.0, -1.0))),
}
RHS_PARAMS = [(name, fuse) for name in CASES for fuse in (0, 1)
              if not (fuse and CASES[name][1].get("lnp_aver"))]


def _state(S, shape, seed=5):
    nx, ny, nphys = shape
    f, g, lb, ub = rigid_state(nx, ny, nphys, seed=seed, G=S.ZGHOST_MIN)
    return [t.numpy() for t in f], g, lb, ub


def _make(S, fields, g, kw):
    refs, dev = S.split_state(fields)
    sim = S.Sim((g.nx, g.ny, g.nz), (g.dx, g.dy, g.dz),
                S.default_params(ref=refs, zwalls=2, zghost=S.ZGHOST_MIN, **kw))
    return sim, refs, dev


def _floor(fields, g, kw, refs, lb, ub):
    po = oracle_params(kw)
    f = [torch.tensor(a) for a in fields]
    F = oracle.rhs_rigid(f, g, po, lb, ub)
    delta = [0.0] * 8
    for seed in (1, 2):
        gen = torch.Generator().manual_seed(seed)
        fp = [a + (a - r) * U32 * (2.0 * torch.rand(a.shape, generator=gen, dtype=a.dtype) - 1.0)
              for a, r in zip(f, refs)]
        Fp = oracle.rhs_rigid(fp, g, po, lb, ub)
        delta = [max(d, float((a - b).abs().max())) for d, a, b in zip(delta, Fp, F)]
    return [t.numpy() for t in F], delta


@pytest.mark.parametrize("name,fuse", RHS_PARAMS)
def test_rigid_rhs_matches_oracle(S, name, fuse):
    shape, kw = CASES[name]
    fields, g, lb, ub = _state(S, shape)
    sim, refs, dev = _make(S, fields, g, dict(kw, fuse_flux_div=fuse))
    F = [t.double().cpu().numpy() for t in sim.rhs(dev)]
    sim.close()
    Fo, delta = _floor(fields, g, kw, refs, lb, ub)
    sc = scale_of(Fo)
    for c in range(8):
        err = float(np.abs(F[c] - Fo[c]).max())     # ghost planes: 0 on both sides
        assert err <= 2e-4 * sc[c] + K_FLOOR * delta[c], (name, c, err / sc[c], delta[c] / sc[c])
        assert not F[c][:lb].any() and not F[c][ub + 1:].any(), (name, c)


@pytest.mark.parametrize("name", ["viscous_quench_gravity_36x9x12", "const_nu_c1_gravity_13x8x9",
                                  "lnp_aver_cooling_gravity_24x10x8"])
def test_rigid_steps_and_frozen_ghosts(S, name):
    shape, kw = CASES[name]
    fields, g, lb, ub = _state(S, shape, seed=8)
    sim, refs, dev = _make(S, fields, g, kw)
    po = oracle_params(kw)
    fo = [torch.tensor(a) for a in fields]
    ghost0 = [t.clone() for t in dev]
    dt_gpu, _ = sim.courant(dev)
    q1 = oracle.rhs_rigid(fo, g, po, lb, ub)
    dt_o, _ = oracle.courant_rigid(fo, q1, g, po, lb, ub)
    assert abs(dt_gpu / dt_o - 1) < 1e-5, (dt_gpu, dt_o)
    for _ in range(3):
        dt = sim.step(dev, None, want_dt=True)
        fo, dto = oracle.step_rigid(fo, g, po, lb, ub, dt=dt)
    got = S.join_state(dev, refs)
    e = err_group(got, [t.numpy() for t in fo])      # every plane, ghosts included
    assert max(e) < 5e-5, (name, e)
    for c in (0, 4, 5, 6, 7):
        assert torch.equal(dev[c][:lb], ghost0[c][:lb]) and torch.equal(dev[c][ub + 1:], ghost0[c][ub + 1:]), c
    sim.close()


def test_rigid_diagnostics(S):
    shape, kw = CASES["viscous_quench_gravity_36x9x12"]
    fields, g, lb, ub = _state(S, shape, seed=4)
    sim, refs, dev = _make(S, fields, g, kw)
    d = sim.diagnostics(dev)
    do = oracle.diagnostics_rigid([torch.tensor(a) for a in fields], g, oracle_params(kw), lb, ub)
    for i in (0, 1, 2, 3, 4, 5, 6):
        assert abs(d[i] - do[i]) <= 1e-6 * max(abs(do[i]), abs(do[0])), (i, d[i], do[i])
    assert abs(d[7] - do[7]) <= 1e-4 * do[7] + 1e-6 and abs(d[8] - do[8]) <= 1e-4 * do[8] + 1e-6
    assert d[9] == 0
    sim.close()


@pytest.mark.parametrize("lnp", [0, 1])
def test_rigid_box_keeps_a_balanced_atmosphere_at_rest(S, lnp):
    """The isothermal atmosphere P = rho = exp(-z/H) with gravity equal to the
    discrete pressure gradient over the density (closed form, the oracle pin
    of the same name; with ln(P/P_aver) the gradient of an exponential is
    exact and the balancing gravity is -1/H): every right-hand side is zero
    in exact arithmetic.  In FP32, over 20 Courant steps with RM viscosity and
    the quench, the momenta stay within 2e-6 of rho c_s and the density within
    1e-6 of itself (measured on GB300: 1.6e-7 and 1.4e-7; 1.3e-7 of rho c_s
    with ln(P/P_aver))."""
    G = S.ZGHOST_MIN
    nx, ny, nphys, H = 8, 6, 24, 1.0
    nz = nphys + 1 + 2 * G
    h = 1.0 / nphys
    lam = -1.0 / H
    s = (2.0 / h) * (DA * math.sinh(lam * h / 2) + DB * math.sinh(3 * lam * h / 2)
                     + DC * math.sinh(5 * lam * h / 2))
    gam = 5.0 / 3.0
    z = ((np.arange(nz) - G + 0.5) * h).reshape(nz, 1, 1) * np.ones((1, ny, nx))
    r = np.exp(-z / H)
    zero = np.zeros_like(r)
    fields = [r, zero, zero, zero, r / (gam - 1.0), zero, zero, zero + 0.2]
    g = oracle.Grid(nx, ny, nz, 1.0 / nx, 1.0 / ny, h)
    kw = dict(VISC_KW, g=(0.0, 0.0, lam if lnp else s), lnp_aver=lnp)
    sim, refs, dev = _make(S, fields, g, kw)
    for _ in range(20):
        sim.step(dev, None)
    got = S.join_state(dev, refs)
    cs = math.sqrt(gam)
    pmax = max(float(np.abs(got[c] / np.maximum(r, 1e-30)).max()) for c in (1, 2, 3))
    rerr = float(np.abs(got[0] / r - 1).max())
    print("rigid atmosphere lnp_aver=%d: max |p|/rho = %.3e c_s, max |drho/rho| = %.3e"
          % (lnp, pmax / cs, rerr))
    assert pmax < 2e-6 * cs and rerr < 1e-6, (pmax / cs, rerr)
    sim.close()


def test_rigid_walls_refuse_the_adjoint(S):
    fields, g, lb, ub = _state(S, (8, 8, 4))
    sim, refs, dev = _make(S, fields, g, {})
    with pytest.raises(S.StaggerError) as ei:
        sim.step_adjoint(dev, 1e-3, [torch.zeros_like(t) for t in dev])
    assert ei.value.status == S.EUNSUPPORTED
    sim.close()


def test_rigid_op_graph_matches_oracle(S):
    """stagger_rhs_unfused(_f64) and stagger_step_unfused_f64 with rigid walls:
    the same ghost fill and zero ghost derivatives around the op graph; FP64
    to 1e-10 of the term scale against the oracle, FP32 to the RHS tolerance."""
    shape, kw = CASES["viscous_quench_gravity_36x9x12"]
    fields, g, lb, ub = _state(S, shape, seed=6)
    sim, refs, dev = _make(S, fields, g, kw)
    po = oracle_params(kw)
    f64 = [torch.tensor(a) for a in fields]
    Fo = [t.numpy() for t in oracle.rhs_rigid(f64, g, po, lb, ub)]
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(fields, refs)]
    F64 = [t.cpu().numpy() for t in sim.rhs_unfused_f64(d64)]
    sc = scale_of(Fo)
    for c in range(8):
        assert float(np.abs(F64[c] - Fo[c]).max()) <= 1e-10 * sc[c], c
        assert not F64[c][:lb].any() and not F64[c][ub + 1:].any(), c
    Fo_, delta = _floor(fields, g, kw, refs, lb, ub)
    F32 = [t.double().cpu().numpy() for t in sim.rhs_unfused(dev)]
    for c in range(8):
        assert float(np.abs(F32[c] - Fo[c]).max()) <= 2e-4 * sc[c] + K_FLOOR * delta[c], c
    dt = 2e-3
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(fields, refs)]
    sim.step_unfused_f64(d64, dt)
    fo, _ = oracle.step_rigid(f64, g, po, lb, ub, dt=dt)
    got = [t.cpu().numpy() + r for t, r in zip(d64, refs)]
    for c in range(8):
        ref = fo[c].numpy()
        assert float(np.abs(got[c] - ref).max()) <= 1e-12 * max(1.0, float(np.abs(ref).max())), c
    sim.close()


def test_stratified_atmosphere_fp32_against_fp64_op_graph(S):
    """The stratified atmosphere of the rigid-wall workload (two scale heights
    here, 24^3 physical cells, velocity noise 1e-3), 20 Courant steps of the
    FP32 fused path and of the FP64 op graph with the same dt, RM viscosity
    and the quench.  The momentum derivative is the small residual of the
    pressure gradient and gravity, each of size rho |g|, so FP32 rounding of
    those terms sets the momentum error: judged on the sound-speed momentum
    scale max(rho) c_s, the density and energy on their ranges, the field on
    its largest magnitude; each within 1e-6."""
    G = S.ZGHOST_MIN
    w = inputs.stratified_atmosphere(24, 24, 24, zghost=G, lengths=(1.0, 1.0, 1.0), H=0.5)
    kw = dict(VISC_KW, g=(0.0, 0.0, -2.0))
    refs, d32 = S.split_state(w.fields)
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, zwalls=2, zghost=G, **kw))
    for _ in range(20):
        dt = sim.step(d32, None, want_dt=True)
        sim.step_unfused_f64(d64, dt)
    sim.close()
    lb, ub = G, G + 23
    a = [d32[c][lb:ub + 1].double().cpu().numpy() + refs[c] for c in range(8)]
    b = [d64[c][lb:ub + 1].cpu().numpy() + refs[c] for c in range(8)]
    rmax = float(b[0].max())
    bmax = max(float(np.abs(b[c]).max()) for c in (5, 6, 7))
    errs = []
    for c in range(8):
        e = float(np.abs(a[c] - b[c]).max())
        sc = (float(b[c].max() - b[c].min()) if c in (0, 4) else rmax * 1.0 if c in (1, 2, 3)
              else bmax)
        errs.append(e / sc)
    print("stratified 24^3 FP32 vs FP64 graph, 20 steps, err/scale:", ["%.2e" % e for e in errs])
    assert max(errs) < 1e-6, errs
