"""Closed z walls (Sect. "Boundary Conditions", "Closed"; reading R22) on the
GPU against the FP64 oracle's closed box (the periodic right-hand side of the
doubled mirror-symmetric state).

The GPU keeps STAGGER_ZGHOST_MIN ghost planes at each end of its arrays,
refills them by reflection before every stage and runs its periodic kernels
over the padded arrays; the oracle never pads.  Right-hand sides are compared
on the physical planes with the tolerance of the other RHS tests (2e-4 of the
term scale plus ten FP32 floors), three Courant steps to 5e-5 of each field
group, the ghost planes bit for bit against the oracle's reflection of the
GPU's own physical planes, the Courant step to 1e-5 and the totals the closed
box conserves to 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as inputs
from test_gpu_parity import K_FLOOR, U32, VISC_KW, err_group, oracle_params, scale_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    return S


def wall_workload(nx, ny, nphys, G, seed=11, grav=False):
    """A smooth state on nx x ny x (nphys + 1 + 2 G) planes, the physical part
    the centre planes G .. G + nphys; solenoidal B (B_x independent of x, B_y
    of y, B_z uniform), so the momentum and div B invariants are exact."""
    nz = nphys + 1 + 2 * G
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) - G + 0.5) / nphys
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")

    def smooth(a):
        ph = rng.uniform(0, 2 * np.pi, 4)
        return a * (np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
                    + 0.5 * np.sin(np.pi * 1.3 * Z + ph[2]) + 0.3 * np.cos(2 * np.pi * (X + Y) + ph[3]))

    r = 1.0 + 0.05 * smooth(1.0)
    if grav:
        r = r * np.exp(-Z / 2.0)
    bx = 0.1 * np.sin(2 * np.pi * Y + 0.3) * np.cos(1.7 * Z) + 0.0 * X
    by = 0.1 * np.cos(2 * np.pi * X + 0.2) * np.sin(2.3 * Z + 0.4) + 0.0 * Y
    f = [r, 0.2 * smooth(1.0), 0.2 * smooth(1.0), 0.2 * smooth(1.0),
         0.9 * r * (1.0 + 0.03 * smooth(1.0)), bx, by, 0.3 + 0.0 * Z]
    lb, ub = G, G + nphys
    f = [t.numpy() for t in oracle.fill_wall_ghosts([torch.tensor(a) for a in f], lb, ub)]
    return inputs.Workload("walls", (nx, ny, nz), (1.0 / nx, 1.1 / ny, 0.9 / nphys), f), lb, ub


CASES = {
    "ideal_20x12x16": ((20, 12, 16), {}, False),
    "viscous_quench_36x9x20": ((36, 9, 20), VISC_KW, False),
    "const_nu_gravity_13x8x12": ((13, 8, 12),
                                 dict(nu_const=0.003, c1=-1 / 3, nuE=0.5, nuB=0.7,
                                      g=(0.1, 0.0, -1.0)), True),
    "viscous_quench_gravity_32x16x6": ((32, 16, 6), dict(VISC_KW, g=(0.0, 0.0, -1.0)), True),
    "second_order_cooling_chromo_24x10x9": (
        (24, 10, 9), dict(VISC_KW, do_2nddiv=1, d2lnr_lim=-1.0, t_cool=0.05, e_cool=0.7,
                          rho_cool=1.02, cool_cut=1, t_chromo=0.2, rho_bot=1.1), True),
    # eq. (pressure) through ln(P/P_aver), on the gravity-stratified state
    "lnp_aver_gravity_20x12x10": ((20, 12, 10), dict(VISC_KW, g=(0.0, 0.0, -1.0), lnp_aver=1), True),
}
# The fused flux-divergence kernel does not take lnp_aver (STAGGER_EINVAL).
RHS_PARAMS = [(name, fuse) for name in CASES for fuse in (0, 1)
              if not (fuse and CASES[name][1].get("lnp_aver"))]


def _make(S, w, kw, G):
    refs = [float(np.mean(w.fields[0])), 0.0, 0.0, 0.0, float(np.mean(w.fields[4])), 0.0, 0.0, 0.3]
    refs, dev = S.split_state(w.fields, refs)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, zwalls=1, zghost=G, **kw))
    return sim, refs, dev


def _floor(w, kw, refs, lb, ub):
    g = oracle.Grid(*w.shape, *w.spacing)
    po = oracle_params(kw)
    f = [torch.tensor(a) for a in w.fields]
    F = oracle.rhs_walls(f, g, po, lb, ub)
    delta = [0.0] * 8
    for seed in (1, 2):
        gen = torch.Generator().manual_seed(seed)
        fp = [a + (a - r) * U32 * (2.0 * torch.rand(a.shape, generator=gen, dtype=a.dtype) - 1.0)
              for a, r in zip(f, refs)]
        Fp = oracle.rhs_walls(fp, g, po, lb, ub)
        delta = [max(d, float((a - b).abs().max())) for d, a, b in zip(delta, Fp, F)]
    return [t.numpy() for t in F], delta


@pytest.mark.parametrize("name,fuse", RHS_PARAMS)
def test_walls_rhs_matches_oracle(S, name, fuse):
    (nx, ny, nphys), kw, grav = CASES[name]
    G = S.ZGHOST_MIN
    w, lb, ub = wall_workload(nx, ny, nphys, G, grav=grav)
    sim, refs, dev = _make(S, w, dict(kw, fuse_flux_div=fuse), G)
    F = [t.double().cpu().numpy() for t in sim.rhs(dev)]
    sim.close()
    Fo, delta = _floor(w, kw, refs, lb, ub)
    sc = scale_of(Fo)
    for c in range(8):
        err = float(np.abs(F[c] - Fo[c]).max())     # ghost planes: 0 on both sides
        assert err <= 2e-4 * sc[c] + K_FLOOR * delta[c], (name, c, err / sc[c], delta[c] / sc[c])


@pytest.mark.parametrize("name", ["viscous_quench_36x9x20", "const_nu_gravity_13x8x12",
                                  "lnp_aver_gravity_20x12x10"])
def test_walls_steps_ghosts_and_courant(S, name):
    (nx, ny, nphys), kw, grav = CASES[name]
    G = S.ZGHOST_MIN
    w, lb, ub = wall_workload(nx, ny, nphys, G, grav=grav)
    sim, refs, dev = _make(S, w, kw, G)
    g = oracle.Grid(*w.shape, *w.spacing)
    po = oracle_params(kw)
    fo = [torch.tensor(a) for a in w.fields]
    # Courant step of the closed box
    dt_gpu, _ = sim.courant(dev)
    q1 = oracle.rhs_walls(fo, g, po, lb, ub)
    dt_o, _ = oracle.courant_walls(fo, q1, g, po, lb, ub)
    assert abs(dt_gpu / dt_o - 1) < 1e-5, (dt_gpu, dt_o)
    for _ in range(3):
        dt = sim.step(dev, None, want_dt=True)
        fo, dto = oracle.step_walls(fo, g, po, lb, ub, dt=dt)
    got = S.join_state(dev, refs)
    phys = [a[lb:ub + 1] for a in got]
    e = err_group(phys, [t[lb:ub + 1].numpy() for t in fo])
    assert max(e) < 5e-5, (name, e)
    # ghost planes: the reflection of the GPU's own physical planes, bit for bit
    dev32 = [t.cpu() for t in dev]
    mirrored = oracle.fill_wall_ghosts([t.double() for t in dev32], lb, ub)
    for c in range(8):
        assert torch.equal(mirrored[c].float(), dev32[c]), c
    sim.close()


def test_walls_conservation_and_diagnostics(S):
    (nx, ny, nphys), kw, grav = CASES["viscous_quench_gravity_32x16x6"]
    G = S.ZGHOST_MIN
    w, lb, ub = wall_workload(nx, ny, 10, G, grav=True, seed=4)
    sim, refs, dev = _make(S, w, kw, G)
    g = oracle.Grid(*w.shape, *w.spacing)
    po = oracle_params(kw)
    d0 = sim.diagnostics(dev)
    do = oracle.diagnostics_walls([torch.tensor(a) for a in w.fields], g, po, lb, ub)
    for i in (0, 1, 2, 3, 4, 5, 6):
        assert abs(d0[i] - do[i]) <= 1e-6 * max(abs(do[i]), abs(do[0])), (i, d0[i], do[i])
    assert abs(d0[8] - do[8]) <= 1e-4 * do[8] + 1e-6 and d0[9] == 0
    for _ in range(20):
        sim.step(dev, None)
    d1 = sim.diagnostics(dev)
    # FP32 deviations: each cell update rounds at ulp(rho') ~ 1e-8 here
    assert abs(d1[0] - d0[0]) < 1e-6 * d0[0], (d1[0], d0[0])
    pscale = float(sum(t[lb:ub + 1].abs().sum() for t in dev[1:3]))
    assert abs(d1[1] - d0[1]) < 1e-5 * pscale and abs(d1[2] - d0[2]) < 1e-5 * pscale
    assert d1[7] < 1e-3 / (0.9 / 10) and d1[9] == 0
    sim.close()


def test_walls_refuse_the_op_graph(S):
    w, lb, ub = wall_workload(8, 8, 4, S.ZGHOST_MIN)
    sim, refs, dev = _make(S, w, {}, S.ZGHOST_MIN)
    with pytest.raises(S.StaggerError) as ei:
        sim.rhs_unfused(dev)
    assert ei.value.status == S.EUNSUPPORTED
    with pytest.raises(S.StaggerError):
        sim.step_adjoint(dev, 1e-3, [torch.zeros_like(t) for t in dev])
    sim.close()
