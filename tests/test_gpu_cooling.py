"""GPU parity of the chromospheric cooling (eq. ChromoCool, horizontal-plane
mean of e, reading R20) and the coronal thin cooling (eq. CoronaCool, reading
R21) against the FP64 oracle: right-hand side (fused FP32 with one- and
four-cell threads, unfused FP32, FP64), three Courant steps, and the FP64
adjoint, whose reverse sweep takes the transpose of the plane mean."""
import pytest
import torch

import oracle
from test_gpu_parity import VISC_KW, err_group, err_max, err_scale, make, oracle_params, ragged_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    return S


CHROMO = dict(t_chromo=0.05, rho_bot=0.9)
CORONA = dict(cor_L0=0.3, cor_Tunit=8e3)
CASES = {
    "cool20x12x9_chromo_corona_visc": ((20, 12, 9), dict(VISC_KW, **CHROMO, **CORONA)),
    "cool21x10x7_chromo": ((21, 10, 7), dict(CHROMO)),
    # a stronger coronal loss next to the Newtonian relaxation
    "cool16x8x10_corona_newton": ((16, 8, 10), dict(cor_L0=5.0, cor_Tunit=8e3, t_cool=0.1,
                                                     e_cool=0.8)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_cooling_rhs(S, name):
    shape, kw = CASES[name]
    w = ragged_state(shape)
    g = oracle.Grid(*shape, *w.spacing)
    f64 = [torch.tensor(a) for a in w.fields]
    Fo = [t.numpy() for t in oracle.rhs(f64, g, oracle_params(kw))]
    base = {k: v for k, v in kw.items() if k not in CHROMO and k not in CORONA}
    Fb = [t.numpy() for t in oracle.rhs(f64, g, oracle_params(base))]
    assert err_scale(Fb, Fo)[4] > 1e-2          # the cooling matters
    for sc in (0, 1):
        sim, refs, dev = make(S, w, dict(kw, scalar_cells=sc))
        F = [t.double().cpu().numpy() for t in sim.rhs(dev)]
        Fu = [t.double().cpu().numpy() for t in sim.rhs_unfused(dev)]
        d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
        F64 = [t.cpu().numpy() for t in sim.rhs_unfused_f64(d64)]
        sim.close()
        assert max(err_scale(F, Fo)) < 2e-4, (name, sc, err_scale(F, Fo))
        assert max(err_scale(Fu, Fo)) < 2e-4, (name, sc, err_scale(Fu, Fo))
        assert max(err_scale(F64, Fo)) < 1e-10, (name, sc, err_scale(F64, Fo))


@pytest.mark.parametrize("name", list(CASES))
def test_cooling_steps(S, name):
    shape, kw = CASES[name]
    w = ragged_state(shape)
    sim, refs, dev = make(S, w, kw)
    g = oracle.Grid(*shape, *w.spacing)
    po = oracle_params(kw)
    fo = [torch.tensor(a) for a in w.fields]
    for _ in range(3):
        dt = sim.step(dev, None, want_dt=True)
        fo, dto = oracle.step(fo, g, po, dt=dt)
        assert abs(dt / dto - 1) < 1e-4, (dt, dto)
    e = err_group(S.join_state(dev, refs), [t.numpy() for t in fo])
    sim.close()
    assert max(e) < 3e-5, (name, e)


def test_cooling_adjoint_fp64(S):
    shape, kw = CASES["cool20x12x9_chromo_corona_visc"]
    w = ragged_state((13, 11, 9))
    sim, refs, dev = make(S, w, kw)
    g = oracle.Grid(*w.shape, *w.spacing)
    f64 = [torch.tensor(a) for a in w.fields]
    dt = 2e-4
    gen = torch.Generator().manual_seed(3)
    lam = [torch.randn(t.shape, generator=gen, dtype=torch.float64) for t in f64]
    ref = [t.numpy() for t in oracle.step_adjoint(f64, dt, lam, g, oracle_params(kw))]
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
    out64 = sim.step_adjoint_f64(d64, dt, [l.cuda() for l in lam])
    torch.cuda.synchronize()
    e64 = err_max([t.cpu().numpy() for t in out64], ref)
    sim.close()
    assert max(e64) < 1e-10, e64
