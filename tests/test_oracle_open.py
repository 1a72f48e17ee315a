"""Pins of the stellar-atmosphere z boundaries of the FP64 oracle (Sect.
"Boundary Conditions", "Stellar Atmosphere"; reading R26).

- The fill continues an exponential atmosphere (ln rho linear, e uniform)
  exactly into both ends' ghost planes; the top limits clamp the ghost
  density to its plane-mean multiples and e to its range about the boundary
  value; the bottom momenta are symmetric about the boundary point, the top
  ghost velocity is the boundary velocity clipped to top_umax; B is
  extrapolated and, at the bottom, blended fully toward B_bdry in inflows and
  left alone in outflows.
- Bottom derivatives: E relaxes to bdry_E on bdry_t in every column; in an
  inflow rho relaxes to bdry_rho; in an outflow the added density change
  keeps d/dt ln(P rho^-gamma) what the plain right-hand side gives (eqs.
  constS to addderiv, the ideal gas).
- Top, eq. (rbdrylo): with a uniform mass flux the vertical divergence is
  zero and the correction is the flux over the pressure scale height.
- A discretely balanced isothermal atmosphere at rest, with the bottom
  targets at its bottom values, is steady to roundoff.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle.stagger import DT, DA, DB, DC, Grid, Params

G = 14
VISC = dict(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=True)


def atmosphere(nx, ny, nphys, H=0.5, gam=5.0 / 3.0):
    """rho = P = exp(-z/H) at rest, B = (0, 0, 0.2), on nphys + 1 physical
    centre planes with G ghost planes at each end."""
    nz = nphys + 1 + 2 * G
    h = 1.0 / nphys
    z = ((torch.arange(nz, dtype=DT) - G + 0.5) * h).reshape(nz, 1, 1).expand(nz, ny, nx)
    r = torch.exp(-z / H)
    zero = torch.zeros_like(r)
    f = [r.clone(), zero.clone(), zero.clone(), zero.clone(), r / (gam - 1.0), zero.clone(),
         zero.clone(), zero + 0.2]
    return f, Grid(nx, ny, nz, 1.0 / nx, 1.0 / ny, h), G, G + nphys


def random_state(nx, ny, nphys, seed=3):
    """The atmosphere with smooth random perturbations: a few per cent in rho
    and E, momenta and field of 0.05 (sinusoids with random phases; grid-scale
    noise would make the linear extrapolation over 14 ghost planes run away)."""
    f, g, lb, ub = atmosphere(nx, ny, nphys)
    rng = np.random.default_rng(seed)
    nz = g.nz
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) - lb + 0.5) / (ub - lb)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")

    def smooth():
        ph = rng.uniform(0, 2 * np.pi, 4)
        return torch.tensor(np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
                            + 0.5 * np.sin(np.pi * 1.3 * Z + ph[2])
                            + 0.3 * np.cos(2 * np.pi * (X + Y) + ph[3]), dtype=DT)
    for c in range(8):
        if c in (0, 4):
            f[c] = f[c] * (1.0 + 0.02 * smooth())
        else:
            f[c] = f[c] + 0.05 * smooth()
    return f, g, lb, ub


@pytest.mark.parametrize("gz", [-1.0, 1.0])
def test_open_fill_continues_an_exponential_atmosphere(gz):
    f, g, lb, ub = atmosphere(5, 4, 10)
    p = Params(g=(0.0, 0.0, gz))
    fo = oracle.fill_open_ghosts(f, p, lb, ub)
    for c in (0, 4, 7):
        err = float(((fo[c] - f[c]) / f[c]).abs().max())
        assert err <= 1e-13, (c, err)
    for c in (1, 2, 3, 5, 6):
        assert float(fo[c].abs().max()) == 0.0


def test_open_top_limits_clamp_density_and_energy():
    f, g, lb, ub = atmosphere(6, 5, 10)
    p = Params(g=(0.0, 0.0, -1.0), top_rho_lo=0.8, top_rho_hi=1.25, top_e_fac=1.1)
    # a steep horizontal pattern in the top two planes: the extrapolation runs away
    xs = torch.linspace(-1.0, 1.0, 6, dtype=DT).reshape(1, 1, 6).expand(1, 5, 6)
    f[0][ub] = f[0][ub] * torch.exp(0.5 * xs[0])
    f[4][ub] = f[4][ub] * torch.exp(0.8 * xs[0])
    fo = oracle.fill_open_ghosts(f, p, lb, ub)
    lr = torch.log(f[0])
    e = f[4] / f[0]
    for j in range(1, G + 1):
        k = ub + j
        rx = torch.exp(lr[ub] + j * (lr[ub] - lr[ub - 1]))
        m = float(rx.mean())
        assert float(fo[0][k].min()) >= 0.8 * m * (1 - 1e-14)
        assert float(fo[0][k].max()) <= 1.25 * m * (1 + 1e-14)
        ek = fo[4][k] / fo[0][k]
        assert bool((ek >= e[ub] / 1.1 * (1 - 1e-14)).all()) and bool((ek <= e[ub] * 1.1 * (1 + 1e-14)).all())
    # the limits were active (far planes hit both density bounds)
    k = ub + G
    rx = torch.exp(lr[ub] + G * (lr[ub] - lr[ub - 1]))
    assert abs(float(fo[0][k].max()) - 1.25 * float(rx.mean())) <= 1e-13 * float(rx.mean())
    assert abs(float(fo[0][k].min()) - 0.8 * float(rx.mean())) <= 1e-13 * float(rx.mean())


def test_open_momenta_and_field_in_the_ghost_planes():
    f, g, lb, ub = random_state(6, 5, 12)
    p = Params(g=(0.0, 0.0, -1.0), top_umax=0.03, bdry_u=1e-12, bdry_B=(0.7, -0.4, 0.0))
    fo = oracle.fill_open_ghosts(f, p, lb, ub)
    # bottom (lb): symmetric momenta
    for j in range(1, G + 1):
        for c in (1, 2):
            assert torch.equal(fo[c][lb - j], f[c][lb + j])
    for m in range(lb + 1):
        assert torch.equal(fo[3][m], f[3][2 * lb + 1 - m])
    # top (ub): the boundary velocity, clipped
    rf = oracle.face_densities(fo, p)
    for c, d, src in ((1, 0, ub), (2, 1, ub), (3, 2, ub)):
        ubv = torch.clamp(f[c][src] / rf[d][src], -0.03, 0.03)
        for k in range(ub + 1, g.nz):
            err = float((fo[c][k] / rf[d][k] - ubv).abs().max())
            assert err <= 1e-15, (c, k, err)
    assert float((f[1][ub] / rf[0][ub]).abs().max()) > 0.03     # the clip was active
    # B: linear extrapolation, then at the bottom all or nothing toward B_bdry
    # (U_bdry tiny: f is 1 in inflow columns, 0 in outflow columns)
    uout = -fo[3][lb + 1] / rf[2][lb + 1]
    inflow = uout < 0
    assert bool(inflow.any()) and bool((~inflow).any())
    for j in range(1, G + 1):
        for c, bb in ((5, 0.7), (6, -0.4)):
            lin = f[c][lb] + j * (f[c][lb] - f[c][lb + 1])
            want = torch.where(inflow, torch.full_like(lin, bb), lin)
            assert float((fo[c][lb - j] - want).abs().max()) <= 1e-14
            lin_t = f[c][ub] + j * (f[c][ub] - f[c][ub - 1])
            assert float((fo[c][ub + j] - lin_t).abs().max()) <= 1e-14
    for m in range(lb + 1):
        d = lb + 1 - m
        want = f[7][lb + 1] + d * (f[7][lb + 1] - f[7][lb + 2])
        assert float((fo[7][m] - want).abs().max()) <= 1e-13


def test_open_bottom_relaxation_and_entropy():
    f, g, lb, ub = random_state(6, 5, 12, seed=8)
    p = Params(**VISC, g=(0.0, 0.0, -1.0), bdry_u=1e-12, bdry_t=0.3, bdry_rho=1.3, bdry_E=2.1)
    F = oracle.rhs_open(f, g, p, lb, ub)
    fo = oracle.fill_open_ghosts(f, p, lb, ub)
    F0 = oracle.rhs(fo, g, p)
    r, E = fo[0][lb], fo[4][lb]
    assert float((F[4][lb] - (2.1 - E) / 0.3).abs().max()) <= 1e-13 * float(E.abs().max()) / 0.3
    rf = oracle.face_densities(fo, p)
    inflow = (-fo[3][lb + 1] / rf[2][lb + 1]) < 0
    # inflow: rho relaxes to bdry_rho; the horizontal momenta are damped toward their mean
    a = F[0][lb][inflow]
    assert float((a - (1.3 - r[inflow]) / 0.3).abs().max()) <= 1e-13
    for c in (1, 2):
        want = F0[c][lb] - (fo[c][lb] - fo[c][lb].mean()) / 0.3
        want = torch.where(inflow, want, F0[c][lb])
        assert float((F[c][lb] - want).abs().max()) <= 1e-12
    # outflow: the entropy rate of the plain right-hand side is kept
    gam = p.gamma
    s_new = (F[4][lb] / E - gam * F[0][lb] / r)[~inflow]
    s_old = (F0[4][lb] / E - gam * F0[0][lb] / r)[~inflow]
    assert float((s_new - s_old).abs().max()) <= 1e-12 * float(s_old.abs().max() + 1.0)
    # and the pressure relaxes to (gamma - 1) bdry_E like the inflow's
    assert float((F[4][lb] - F0[4][lb]).abs().max()) > 1e-3
    # ghost planes: zero derivative
    for c in range(8):
        assert float(F[c][:lb].abs().max()) == 0.0 and float(F[c][ub + 1:].abs().max()) == 0.0
    assert float(F[3][lb].abs().max()) == 0.0 and float(F[7][lb].abs().max()) == 0.0


def test_open_top_replaces_the_vertical_mass_flux_divergence():
    """Uniform rho = 1.2, E = 2 and a uniform p_z = P0: the fill keeps p_z
    uniform in every ghost face (symmetric at the bottom, rho_face u_b at the
    top), so the plain d rho/dt is zero everywhere, and the top plane's rate
    is the flux over the pressure scale height, P0 / H_P, H_P = (gamma - 1)
    e / |g_z|; no other plane changes."""
    nx, ny, nphys = 5, 4, 10
    nz = nphys + 1 + 2 * G
    g = Grid(nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nphys)
    one = torch.ones((nz, ny, nx), dtype=DT)
    P0, gz = 0.013, -3.0
    f = [1.2 * one, 0 * one, 0 * one, P0 * one, 2.0 * one, 0 * one, 0 * one, 0.2 * one]
    p = Params(g=(0.0, 0.0, gz), top_umax=10.0)
    lb, ub = G, G + nphys
    F = oracle.rhs_open(f, g, p, lb, ub)
    HP = (p.gamma - 1.0) * (2.0 / 1.2) / abs(gz)
    assert float((F[0][ub] - P0 / HP).abs().max()) <= 1e-13 * P0 / HP
    assert float(F[0][lb + 1:ub].abs().max()) <= 1e-15
    # with gravity the other way the top is lb, where the outward direction is -z
    p2 = Params(g=(0.0, 0.0, -gz), top_umax=10.0)
    F2 = oracle.rhs_open(f, g, p2, lb, ub)
    assert float((F2[0][lb] + P0 / HP).abs().max()) <= 1e-13 * P0 / HP


def test_open_boundaries_hold_a_balanced_atmosphere_at_rest():
    nx, ny, nphys, H = 6, 5, 16, 0.25
    f, g, lb, ub = atmosphere(nx, ny, nphys, H=H)
    h = 1.0 / nphys
    lam = -1.0 / H
    s = (2.0 / h) * (DA * math.sinh(lam * h / 2) + DB * math.sinh(3 * lam * h / 2)
                     + DC * math.sinh(5 * lam * h / 2))
    p = Params(**VISC, g=(0.0, 0.0, s), bdry_rho=float(f[0][lb, 0, 0]),
               bdry_E=float(f[4][lb, 0, 0]), bdry_t=0.1)
    F = oracle.rhs_open(f, g, p, lb, ub)
    scale = float(f[0][lb:ub + 1].max()) * abs(s)
    for c in range(8):
        err = float(F[c].abs().max())
        assert err <= 1e-12 * scale, (c, err / scale)


# ------------------------------------------ top potential field (reading R27) ---

@pytest.mark.parametrize("s", [1, -1])
def test_potential_field_of_a_single_mode_in_closed_form(s):
    """B_z = cos(kx x + ky y) on the plane: the potential field decaying in the
    outward direction s has B_x = s (kx/|k|) sin(kx x + ky y) and
    B_y = s (ky/|k|) sin(kx x + ky y), each at its own face position (B = -grad
    Phi, Phi ~ cos(.) exp(-|k| zeta); div B = 0 and curl B = 0)."""
    nx, ny = 12, 10
    g = Grid(nx, ny, 40, 1.0 / nx, 1.3 / ny, 0.1)
    mx, my = 2, 1
    kx, ky = 2 * math.pi * mx / 1.0, 2 * math.pi * my / 1.3
    kk = math.hypot(kx, ky)
    xc = (torch.arange(nx, dtype=DT) + 0.5) / nx
    yc = (torch.arange(ny, dtype=DT) + 0.5) * 1.3 / ny
    xf = torch.arange(nx, dtype=DT) / nx
    yf = torch.arange(ny, dtype=DT) * 1.3 / ny
    Y, X = torch.meshgrid(yc, xc, indexing="ij")
    bz = torch.cos(kx * X + ky * Y)
    bx, by = oracle.potential_horizontal(bz, g, s)
    Yx, Xx = torch.meshgrid(yc, xf, indexing="ij")
    Yy, Xy = torch.meshgrid(yf, xc, indexing="ij")
    wx = s * kx / kk * torch.sin(kx * Xx + ky * Yx)
    wy = s * ky / kk * torch.sin(kx * Xy + ky * Yy)
    assert float((bx - wx).abs().max()) <= 1e-13
    assert float((by - wy).abs().max()) <= 1e-13
    # a uniform normal field has no horizontal potential part
    bx0, by0 = oracle.potential_horizontal(torch.full((ny, nx), 0.3, dtype=DT), g, s)
    assert float(bx0.abs().max()) <= 1e-15 and float(by0.abs().max()) <= 1e-15


def test_top_relaxes_toward_the_potential_field_and_leaves_it_alone():
    """With top_tpot, the top plane's horizontal field gains (B_pot - (B_h -
    <B_h>)) / top_tpot: zero when the plane already holds the potential field
    of its normal field plus any uniform part, B_pot / top_tpot when its
    horizontal field is uniform; no other plane changes."""
    f, g, lb, ub = random_state(8, 6, 16, seed=4)
    p0 = Params(g=(0.0, 0.0, -1.0), top_umax=10.0)
    pt = Params(**{**p0.__dict__, "top_tpot": 0.05})
    fo = oracle.fill_open_ghosts(f, p0, lb, ub)
    bxp, byp = oracle.potential_horizontal(fo[7][ub], g, 1)
    # top plane: the potential field plus a uniform part
    f = [a.clone() for a in f]
    f[5][ub] = bxp + 0.07
    f[6][ub] = byp - 0.02
    d = [a - b for a, b in zip(oracle.rhs_open(f, g, pt, lb, ub), oracle.rhs_open(f, g, p0, lb, ub))]
    for c in range(8):
        assert float(d[c].abs().max()) <= 1e-12, c
    # uniform horizontal field on the top plane: the rate is B_pot / top_tpot
    f[5][ub] = 0.0 * bxp + 0.07
    f[6][ub] = 0.0 * byp - 0.02
    fo = oracle.fill_open_ghosts(f, p0, lb, ub)
    bxp, byp = oracle.potential_horizontal(fo[7][ub], g, 1)
    d = [a - b for a, b in zip(oracle.rhs_open(f, g, pt, lb, ub), oracle.rhs_open(f, g, p0, lb, ub))]
    assert float((d[5][ub] - bxp / 0.05).abs().max()) <= 1e-11
    assert float((d[6][ub] - byp / 0.05).abs().max()) <= 1e-11
    assert float(bxp.abs().max()) > 1e-3
    for c in range(8):
        rest = torch.cat([d[c][:ub], d[c][ub + 1:]])
        assert float(rest.abs().max()) == 0.0, c
