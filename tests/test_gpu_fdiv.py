"""The fused flux-divergence stage kernel (k_fdiv: every flux formed on chip,
the divergences and the RK update in one z-marching launch) against the FP64
oracle and against the split kernels (fluxes stored by one set of launches
and differentiated by another, the default layout; the fused one is
stagger_params.fuse_flux_div = 1).

The shapes put the kernel's tiling on its edges: several z chunks of 64 planes
with a ragged last one (nz = 131, 70, 66), x tiles of 32 and y tiles of 8
cells that are partly outside the grid (37, 29, 45, 9 ...), a single cell
along x or y (the tile's halo then wraps onto the same cells), and grids with
fewer planes than the kernel's 3-plane z halo.  Tolerances are those of the
other RHS and step parity tests: 2e-4 of each equation's term scale for one
right-hand side, 2e-5 between the two kernel layouts (the same FP32
operations in another order), each plus ten times the equation's FP32 floor
at the state (the change of the oracle's right-hand side when the stored
deviations are rounded to FP32, which the quench ratio of eq. (quench)
amplifies where a stress is small); 5e-5 of each field group after three
Courant steps."""
import numpy as np
import pytest
import torch

import oracle
import workloads as inputs
from test_gpu_parity import (K_FLOOR, VISC_KW, err_group, err_scale, fp32_floor, make,
                             oracle_params, ragged_state, scale_of)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    return S


CASES = {
    "visc_quench_37x29x131": ((37, 29, 131), VISC_KW),
    "ideal_gravity_33x9x70": ((33, 9, 70), dict(g=(0.3, -0.2, -1.0))),
    "const_nu_c1_nolog_45x1x70": (
        (45, 1, 70), dict(nu_const=0.002, c1=-1.0 / 3.0, nuE=0.5, nuB=0.7, log_interp=0)),
    "visc_cooling_all_1x17x9": (
        (1, 17, 9), dict(VISC_KW, t_cool=0.05, e_cool=0.7, rho_cool=1.02, cool_cut=1,
                         t_chromo=0.2, rho_bot=1.1, cor_L0=0.01, cor_Tunit=1e4)),
    "smagorinsky_rm_ediffav_64x8x66": ((64, 8, 66), dict(VISC_KW, csmag=0.15, ediffav=1)),
    "ideal_2planes_40x24x2": ((40, 24, 2), {}),
}


def _state(shape):
    nx, ny, nz = shape
    if min(shape) < 2:
        # ragged_state needs a spectral band along every axis: take a slab of
        # a larger state and keep it periodic by construction of the oracle.
        big = ragged_state((max(nx, 8), max(ny, 8), max(nz, 8)))
        f = [a[:nz, :ny, :nx].copy() for a in big.fields]
        return inputs.Workload("slab", shape, (1.0 / nx, 1.1 / ny, 0.9 / nz), f)
    return ragged_state(shape)


@pytest.mark.parametrize("name", list(CASES))
def test_fused_stage_rhs_matches_oracle_and_split_kernels(S, name):
    shape, kw = CASES[name]
    w = _state(shape)
    got = {}
    for fuse in (1, 0):
        sim, refs, dev = make(S, w, dict(kw, fuse_flux_div=fuse))
        got[fuse] = [t.double().cpu().numpy() for t in sim.rhs(dev)]
        sim.close()
    Fo, delta = fp32_floor(w, kw, refs)
    sc = scale_of(Fo)
    for c in range(8):
        for tag, fuse in (("fused", 1), ("split", 0)):
            err = float(np.abs(got[fuse][c] - Fo[c]).max())
            assert err <= 2e-4 * sc[c] + K_FLOOR * delta[c], (name, tag, c, err / sc[c],
                                                               delta[c] / sc[c])
        d = float(np.abs(got[1][c] - got[0][c]).max())
        assert d <= 2e-5 * sc[c] + K_FLOOR * delta[c], (name, c, d / sc[c], delta[c] / sc[c])


@pytest.mark.parametrize("name", ["visc_quench_37x29x131", "ideal_gravity_33x9x70",
                                  "visc_cooling_all_1x17x9"])
def test_fused_stage_courant_steps(S, name):
    """Three Courant steps (stage 1 writes the derivative and takes the rate
    limit in the kernel; stages 2 and 3 apply the update) against the oracle."""
    shape, kw = CASES[name]
    w = _state(shape)
    sim, refs, dev = make(S, w, dict(kw, fuse_flux_div=1))
    g = oracle.Grid(*w.shape, *w.spacing)
    po = oracle_params(kw)
    fo = [torch.tensor(a) for a in w.fields]
    for _ in range(3):
        dt = sim.step(dev, None, want_dt=True)
        fo, dto = oracle.step(fo, g, po, dt=dt)
        assert abs(dt / dto - 1) < 1e-4, (dt, dto)
    e = err_group(S.join_state(dev, refs), [t.numpy() for t in fo])
    assert max(e) < 5e-5, (name, e)
    sim.close()


def test_fused_stage_layout_switch(S):
    """fuse_flux_div = 1 launches k_fdiv (and no flux or divergence kernel);
    the default launches k_flux, k_flux_e and k_div."""
    w = ragged_state((37, 29, 11))
    sim, refs, dev = make(S, w, dict(VISC_KW, fuse_flux_div=1))
    sim.timing(True)
    sim.step(dev, None)
    kt = sim.kernel_times()
    sim.close()
    assert "k_fdiv" in kt and kt["k_fdiv"][1] == 3
    assert not ({"k_flux", "k_flux_e", "k_div"} & set(kt)), kt
    sim, refs, dev = make(S, w, VISC_KW)
    sim.timing(True)
    sim.step(dev, None)
    kt = sim.kernel_times()
    sim.close()
    assert "k_fdiv" not in kt and {"k_flux", "k_flux_e", "k_div"} <= set(kt), kt
