"""Pins of the rigid z walls of the FP64 oracle (Sect. "Boundary Conditions",
"Rigid"; reading R25: the ghost velocity is the velocity of the boundary
plane, the time derivatives of the ghost values are zero).

- The fill: after it, the velocity p_d / rho_d of every ghost point equals
  the boundary plane's at the same (x, y), and a state built with that
  property is left unchanged by it.
- The reach: the right-hand side of the physical planes does not change when
  six further ghost planes of arbitrary values are put beyond the 14.
- A discretely balanced isothermal atmosphere (gravity equal to the discrete
  pressure gradient over the density, in closed form) is an exact steady
  state of the box with rigid walls, viscosity and the quench on; with
  ln(P/P_aver) (eq. pressure) the balancing gravity is the continuum one.
- A step leaves rho, E and B of the ghost planes unchanged bit for bit.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle.stagger import DT, DA, DB, DC, Grid, Params

G = 14   # ghost planes at each end

VISC = Params(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=True)


def rigid_state(nx, ny, nphys, seed=5, G=G):
    """A smooth random state on nx x ny x (nphys + 1 + 2 G) planes whose
    physical part is the planes G .. G + nphys; the ghost planes hold the
    same smooth functions (any values would do)."""
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

    r = (1.0 + 0.05 * smooth(1.0)) * np.exp(-Z / 2.0)
    f = [r, 0.2 * smooth(1.0), 0.2 * smooth(1.0), 0.2 * smooth(1.0),
         0.9 * r * (1.0 + 0.03 * smooth(1.0)), 0.1 * smooth(1.0), 0.1 * smooth(1.0),
         0.3 + 0.05 * smooth(1.0)]
    g = Grid(nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nphys)
    return [torch.tensor(a, dtype=DT) for a in f], g, G, G + nphys


@pytest.mark.parametrize("log_interp", [True, False])
def test_rigid_fill_gives_ghost_points_the_boundary_velocity(log_interp):
    f, g, lb, ub = rigid_state(9, 7, 8)
    p = Params(log_interp=log_interp)
    fr = oracle.fill_rigid_ghosts(f, p, lb, ub)
    for c in (0, 4, 5, 6, 7):
        assert torch.equal(fr[c], f[c])
    for c in (1, 2, 3):
        assert torch.equal(fr[c][lb:ub + 1], f[c][lb:ub + 1])
    # the velocities the right-hand side forms from the filled state
    parts = oracle.rhs_parts(fr, g, p)
    for key in ("ux", "uy", "uz"):
        u = parts[key]
        for k in list(range(lb)) + list(range(ub + 1, g.nz)):
            b = lb if k < lb else ub
            err = float((u[k] - u[b]).abs().max())
            assert err <= 1e-14 * float(u[b].abs().max()), (key, k, err)


def test_rigid_fill_leaves_a_state_with_that_velocity_unchanged():
    """Momenta built as rho_d (U_d(x, y) + V_d(x, y, z) W(k)), W = 0 on the
    boundary and ghost planes of every field: already the fill's result."""
    f, g, lb, ub = rigid_state(8, 6, 10, seed=9)
    p = Params()
    rf = oracle.face_densities(f, p)
    rng = np.random.default_rng(2)
    k = np.arange(g.nz)
    W = np.where((k > lb) & (k < ub), np.sin(np.pi * (k - lb) / (ub - lb)) ** 2, 0.0)
    W = torch.tensor(W, dtype=DT).reshape(-1, 1, 1)
    g2 = [torch.tensor(rng.standard_normal((1, g.ny, g.nx)), dtype=DT) for _ in range(6)]
    f = list(f)
    for d in range(3):
        f[1 + d] = rf[d] * (0.3 * g2[d] + 0.2 * g2[3 + d] * W)
    fr = oracle.fill_rigid_ghosts(f, p, lb, ub)
    for c in range(8):
        err = float((fr[c] - f[c]).abs().max())
        assert err <= 1e-15 * max(1.0, float(f[c].abs().max())), (c, err)


@pytest.mark.parametrize("p", [Params(), VISC, Params(nu_const=0.003, c1=-1 / 3, g=(0.1, 0, -1.0)),
                               Params(**{**VISC.__dict__, "lnp_aver": True, "g": (0.0, 0.0, -1.0)})],
                         ids=["ideal", "viscous_quench", "const_nu_gravity", "lnp_aver_gravity"])
def test_rigid_rhs_does_not_reach_past_fourteen_ghost_planes(p):
    f, g, lb, ub = rigid_state(8, 6, 9, G=G)
    F = oracle.rhs_rigid(f, g, p, lb, ub)
    # six more ghost planes at each end, holding other values
    extra = 6
    rng = np.random.default_rng(11)
    fe = []
    for c, a in enumerate(f):
        lo = a[:1].expand(extra, -1, -1) * (1 + 0.1 * torch.tensor(rng.random((extra, g.ny, g.nx))))
        hi = a[-1:].expand(extra, -1, -1) * (1 + 0.1 * torch.tensor(rng.random((extra, g.ny, g.nx))))
        fe.append(torch.cat([lo, a, hi]))
    ge = Grid(g.nx, g.ny, g.nz + 2 * extra, g.dx, g.dy, g.dz)
    Fe = oracle.rhs_rigid(fe, ge, p, lb + extra, ub + extra)
    for c in range(8):
        a = F[c][lb:ub + 1]
        b = Fe[c][lb + extra:ub + extra + 1]
        err = float((a - b).abs().max())
        assert err <= 1e-13 * max(1e-12, float(a.abs().max())), (c, err)
        assert float(F[c][:lb].abs().max()) == 0.0 and float(F[c][ub + 1:].abs().max()) == 0.0


@pytest.mark.parametrize("lnp", [False, True])
def test_rigid_box_holds_a_discretely_balanced_isothermal_atmosphere(lnp):
    """P = rho = exp(-z/H) (c^2 = 1) at rest.  ln rho is linear, so the face
    density exp(dn ln rho) is exact, and the staggered derivative of an
    exponential is exact up to its symbol: dddn P = P_face s, s = (2/h) (a
    sinh(lh/2) + b sinh(3lh/2) + c sinh(5lh/2)), l = -1/H.  With g_z = s the
    momentum equation balances face by face; the velocity, the stresses and
    the energy diffusion (e uniform) vanish.  The rigid box, whose ghost
    planes keep the atmosphere, is then steady to roundoff on every physical
    plane, while the closed box (reflection) is not.  With ln(P/P_aver)
    (eq. pressure) the gradient of the exponential is exact, -P_face / H, and
    the balancing gravity is -1/H itself."""
    nx, ny, nphys, H = 6, 5, 16, 0.25
    nz = nphys + 1 + 2 * G
    h = 1.0 / nphys
    lam = -1.0 / H
    s = (2.0 / h) * (DA * math.sinh(lam * h / 2) + DB * math.sinh(3 * lam * h / 2)
                     + DC * math.sinh(5 * lam * h / 2))
    gam = 5.0 / 3.0
    z = ((torch.arange(nz, dtype=DT) - G + 0.5) * h).reshape(nz, 1, 1).expand(nz, ny, nx)
    r = torch.exp(-z / H)
    zero = torch.zeros_like(r)
    f = [r, zero.clone(), zero.clone(), zero.clone(), r / (gam - 1.0), zero.clone(),
         zero.clone(), zero + 0.2]
    g = Grid(nx, ny, nz, 1.0 / nx, 1.0 / ny, h)
    p = Params(**{**VISC.__dict__, "g": (0.0, 0.0, lam if lnp else s), "lnp_aver": lnp})
    lb, ub = G, G + nphys
    F = oracle.rhs_rigid(f, g, p, lb, ub)
    scale = float(r[lb:ub + 1].max()) * abs(s)
    for c in range(8):
        err = float(F[c].abs().max())
        assert err <= 1e-12 * scale, (c, err / scale)
    # the closed box reflects rho about the wall: not in balance there
    Fc = oracle.rhs_walls(f, g, p, lb, ub)
    assert float(Fc[3].abs().max()) > 1e-2 * scale


def test_rigid_step_freezes_the_ghost_density_energy_and_field():
    f, g, lb, ub = rigid_state(8, 6, 7, seed=13)
    out, dt = oracle.step_rigid(f, g, VISC, lb, ub)
    assert dt > 0
    for c in (0, 4, 5, 6, 7):
        assert torch.equal(out[c][:lb], f[c][:lb]) and torch.equal(out[c][ub + 1:], f[c][ub + 1:])
        assert float((out[c][lb:ub + 1] - f[c][lb:ub + 1]).abs().max()) > 0
    # the ghost momenta are the fill of the result
    fr = oracle.fill_rigid_ghosts(out, VISC, lb, ub)
    for c in (1, 2, 3):
        assert torch.equal(fr[c], out[c])
