"""GPU parity on a stretched vertical mesh (Sect. Derivatives; the mesh file of
Sect. Input and output), reading R19, against the FP64 oracle: the right-hand
side (fused FP32 with one- and four-cell threads, unfused FP32, FP64), Courant
steps, the Courant limits, the weighted diagnostics and the FP64 adjoint.

The mesh is z(xi) = hbar (xi + A sin(th xi) / th), th = 2 pi / nz (periodic),
with dz/dk varying by +-45 % (A = 0.45).  Tolerances are those of the uniform
cases (tests/test_gpu_parity.py)."""
import math

import numpy as np
import pytest
import torch

import oracle
from test_gpu_parity import VISC_KW, err_group, err_max, err_scale, oracle_params, ragged_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    return S


def mesh(nz, hbar, A=0.45):
    th = 2 * math.pi / nz
    zc = tuple(hbar * (1 + A * math.cos(th * (k + 0.5))) for k in range(nz))
    zf = tuple(hbar * (1 + A * math.cos(th * k)) for k in range(nz))
    return zc, zf


CASES = {
    # four-cell threads (nx % 4 == 0); RM viscosity with the quench
    "zs20x12x10_visc_quench": ((20, 12, 10), VISC_KW),
    # one-cell threads; Smagorinsky with RM, bulk term, second-order switch off
    "zs21x10x12_smag_c1": ((21, 10, 12), dict(VISC_KW, csmag=0.15, c1=-1.0 / 3.0)),
    # constant viscosity with cooling (high-density cutoff), no log interpolation
    "zs16x8x9_const_nu_cooling": ((16, 8, 9), dict(nu_const=0.002, nuE=0.5, nuB=0.7, t_cool=0.1,
                                                   e_cool=0.8, rho_cool=0.98, cool_cut=2,
                                                   log_interp=0)),
    # eq. (pressure) through ln(P/P_aver): dddn_z ln P_aver on the stretched faces
    "zs20x12x8_visc_lnp_aver": ((20, 12, 8), dict(VISC_KW, lnp_aver=1)),
}


def setup(S, name, **extra):
    shape, kw = CASES[name]
    w = ragged_state(shape)
    zc, zf = mesh(shape[2], w.spacing[2])
    g = oracle.Grid(*shape, *w.spacing, zc=zc, zf=zf)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, zc=zc, zf=zf, **kw, **extra))
    return w, kw, g, sim, refs, dev


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_rhs(S, name):
    w, kw, g, sim, refs, dev = setup(S, name)
    f64 = [torch.tensor(a) for a in w.fields]
    Fo = [t.numpy() for t in oracle.rhs(f64, g, oracle_params(kw))]
    # The mesh changes the answer far beyond the tolerance.
    gu = oracle.Grid(*w.shape, *w.spacing)
    Fu = [t.numpy() for t in oracle.rhs(f64, gu, oracle_params(kw))]
    assert max(err_scale(Fu, Fo)) > 1e-2
    F = [t.double().cpu().numpy() for t in sim.rhs(dev)]
    Fun = [t.double().cpu().numpy() for t in sim.rhs_unfused(dev)]
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
    F64 = [t.cpu().numpy() for t in sim.rhs_unfused_f64(d64)]
    sim.close()
    assert max(err_scale(F, Fo)) < 2e-4, err_scale(F, Fo)
    assert max(err_scale(Fun, Fo)) < 2e-4, err_scale(Fun, Fo)
    assert max(err_scale(F64, Fo)) < 1e-10, err_scale(F64, Fo)
    if w.shape[0] % 4 == 0:
        _, _, _, sim1, _, dev1 = setup(S, name, scalar_cells=1)
        F1 = [t.double().cpu().numpy() for t in sim1.rhs(dev1)]
        sim1.close()
        assert max(err_scale(F1, F)) < 2e-5


@pytest.mark.parametrize("name", list(CASES))
def test_stretched_courant_diagnostics_and_steps(S, name):
    w, kw, g, sim, refs, dev = setup(S, name)
    po = oracle_params(kw)
    f64 = [torch.tensor(a) for a in w.fields]
    dt, lim = sim.courant(dev)
    dto, limo = oracle.courant_dt(f64, oracle.rhs(f64, g, po), g, po)
    assert dt == pytest.approx(dto, rel=1e-5)
    for a, b in zip(lim, limo):
        assert a == pytest.approx(b, rel=1e-4)
    d = sim.diagnostics(dev)
    do = oracle.diagnostics(f64, g, po)
    for i in (0, 4, 5, 6):
        assert d[i] == pytest.approx(do[i], rel=1e-6), (i, d[i], do[i])
    for i in (1, 2, 3):
        assert abs(d[i] - do[i]) < 1e-6 * float(np.abs(w.fields[i]).sum()), (i, d[i], do[i])
    assert d[7] == pytest.approx(do[7], rel=1e-3) and d[8] == pytest.approx(do[8], rel=1e-3)
    fo = f64
    for _ in range(3):
        dt = sim.step(dev, None, want_dt=True)
        fo, dto = oracle.step(fo, g, po, dt=dt)
    e = err_group(S.join_state(dev, refs), [t.numpy() for t in fo])
    assert max(e) < 3e-5, (name, e)
    sim.close()


def test_stretched_adjoint_fp64(S):
    w, kw, g, sim, refs, dev = setup(S, "zs20x12x10_visc_quench")
    f64 = [torch.tensor(a) for a in w.fields]
    dt = 2e-4
    gen = torch.Generator().manual_seed(2)
    lam = [torch.randn(t.shape, generator=gen, dtype=torch.float64) for t in f64]
    ref = [t.numpy() for t in oracle.step_adjoint(f64, dt, lam, g, oracle_params(kw))]
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
    out64 = sim.step_adjoint_f64(d64, dt, [l.cuda() for l in lam])
    torch.cuda.synchronize()
    e64 = err_max([t.cpu().numpy() for t in out64], ref)
    sim.close()
    assert max(e64) < 1e-10, e64


def test_all_options_together(S):
    """Stretched z, second-order switch, Smagorinsky with RM and the quench,
    Newtonian, chromospheric and coronal cooling, gravity and the bulk term in
    one parameter set, on four-cell threads: RHS (FP32, FP64) and three steps
    against the oracle."""
    import test_gpu_second_order as T2
    shape = (20, 12, 10)
    w = T2.sharp_state(shape)
    lim, gap = T2.gap_limit(w.fields)
    assert gap > 1e-5
    zc, zf = mesh(shape[2], w.spacing[2])
    kw = dict(VISC_KW, csmag=0.12, c1=-1.0 / 3.0, do_2nddiv=1, d2lnr_lim=float(lim),
              t_cool=0.2, e_cool=0.8, rho_cool=1.1, cool_cut=1, t_chromo=0.08, rho_bot=0.9,
              cor_L0=1.0, cor_Tunit=8e3, g=(0.0, 0.0, -0.5))
    g = oracle.Grid(*shape, *w.spacing, zc=zc, zf=zf)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, zc=zc, zf=zf, **kw))
    f64 = [torch.tensor(a) for a in w.fields]
    po = oracle_params(kw)
    Fo = [t.numpy() for t in oracle.rhs(f64, g, po)]
    F = [t.double().cpu().numpy() for t in sim.rhs(dev)]
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
    F64 = [t.cpu().numpy() for t in sim.rhs_unfused_f64(d64)]
    assert max(err_scale(F, Fo)) < 2e-4, err_scale(F, Fo)
    assert max(err_scale(F64, Fo)) < 1e-10, err_scale(F64, Fo)
    fo = f64
    for _ in range(3):
        dt = sim.step(dev, None, want_dt=True)
        fo, dto = oracle.step(fo, g, po, dt=dt)
        assert abs(dt / dto - 1) < 1e-4, (dt, dto)
    e = err_group(S.join_state(dev, refs), [t.numpy() for t in fo])
    sim.close()
    assert max(e) < 3e-5, e
