"""Pins of the closed z walls of the FP64 oracle (Sect. "Boundary Conditions",
"Closed"; reading R22: every field continued across a boundary point by
reflection with its parity).

- The construction: the right-hand side of the closed box (the periodic
  right-hand side of the doubled mirror-symmetric state) equals the periodic
  right-hand side of the arrays with 14 ghost planes filled by reflection, on
  the physical planes: the reach of the right-hand side is 14 cells, so the
  wrap of the padded arrays never reaches a physical plane.
- A standing sound wave between the walls oscillates at the closed-form
  frequency c_s D(theta)/h of the staggered operators.
- Mass and the parallel momenta are conserved to roundoff (half weight on the
  boundary planes), div B stays at roundoff, and the odd fields' derivatives
  vanish on the boundary points.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle.stagger import DT, Grid, Params

G = 14   # ghost planes at each end


def wall_state(nx, ny, nphys, seed=3, grav=False):
    """A smooth random state on nx x ny x (nphys + 1 + 2 G) planes whose
    physical part is the centre planes G .. G + nphys."""
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
    # B solenoidal in the discrete sense: B_x independent of x, B_y of y, B_z
    # uniform, so each term of div B vanishes exactly.
    bx = 0.1 * np.sin(2 * np.pi * Y + 0.3) * np.cos(1.7 * Z) + 0.0 * X
    by = 0.1 * np.cos(2 * np.pi * X + 0.2) * np.sin(2.3 * Z + 0.4) + 0.0 * Y
    f = [r, 0.2 * smooth(1.0), 0.2 * smooth(1.0), 0.2 * smooth(1.0),
         0.9 * r * (1.0 + 0.03 * smooth(1.0)), bx, by, 0.3 + 0.0 * Z]
    g = Grid(nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nphys)
    return [torch.tensor(a, dtype=DT) for a in f], g, G, G + nphys


VISC = Params(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=True)


@pytest.mark.parametrize("p", [Params(), VISC, Params(nu_const=0.003, c1=-1 / 3, g=(0.1, 0, -1.0))],
                         ids=["ideal", "viscous_quench", "const_nu_gravity"])
def test_padded_ghosts_equal_doubled_box(p):
    f, g, lb, ub = wall_state(8, 6, 12)
    F = oracle.rhs_walls(f, g, p, lb, ub)
    fp = oracle.fill_wall_ghosts(f, lb, ub)
    # periodic right-hand side of the padded arrays (z gravity only on the
    # physical faces, as it is odd under the reflection)
    pz0 = Params(**{**p.__dict__, "g": (p.g[0], p.g[1], 0.0)})
    parts = oracle.rhs_parts(fp, g, pz0)
    Fp = [parts[k] for k in ("d_r", "d_px", "d_py", "d_pz", "d_E", "d_Bx", "d_By", "d_Bz")]
    Fp[3] = Fp[3] + parts["rz"] * p.g[2]
    for c in range(8):
        lo = lb + 1 if oracle.Z_FACE[c] else lb
        a, b = F[c][lo:ub + 1], Fp[c][lo:ub + 1]
        sc = float(b.abs().max()) + 1e-30
        # roundoff, amplified where the quench ratio is ill-conditioned
        assert float((a - b).abs().max()) <= 1e-10 * sc, (c, float((a - b).abs().max()) / sc)
        assert float(F[c][:lo].abs().max()) == 0.0 and float(F[c][ub + 1:].abs().max()) == 0.0


def test_standing_sound_wave_frequency():
    """rho = 1 + A cos(k zeta), p = 0, E adiabatic, zeta measured from the
    lower boundary point, k = pi m / (L h): an eigenmode of the closed box,
    with omega = c_s D(k h) / h, D(theta) = 2 [a sin(theta/2) + b sin(3 theta/2)
    + c sin(5 theta/2)] (the symbol of eq. (deriv)); c_s = 1."""
    nphys, m, A = 24, 8, 1e-6
    nz = nphys + 1 + 2 * G
    h = 1.0 / nphys
    gam = 5.0 / 3.0
    zeta = (np.arange(nz) - G) * h
    k = math.pi * m / (nphys * h)
    rho = 1.0 + A * np.cos(k * zeta)
    P = 1.0 / gam + A * np.cos(k * zeta)           # c_s^2 = gamma P / rho = 1
    z0 = np.zeros(nz)
    f = [torch.tensor(v.reshape(nz, 1, 1), dtype=DT) for v in
         (rho, z0, z0, z0, P / (gam - 1.0), z0, z0, z0)]
    g = Grid(1, 1, nz, 1.0, 1.0, h)
    lb, ub = G, G + nphys
    a, b, c = 225.0 / 192.0, -25.0 / 384.0, 3.0 / 640.0
    th = k * h
    omega = 2 * (a * math.sin(th / 2) + b * math.sin(3 * th / 2) + c * math.sin(5 * th / 2)) / h
    dt, t = 0.02 * h, 0.0
    for _ in range(48):
        f, _ = oracle.step_walls(f, g, Params(), lb, ub, dt=dt)
        t += dt
    got = (f[0][lb:ub + 1, 0, 0].numpy() - 1.0) / A
    want = np.cos(k * zeta[lb:ub + 1]) * math.cos(omega * t)
    assert np.abs(got - want).max() < 1e-5, np.abs(got - want).max()
    # the continuum frequency c_s k (0.07% higher at k h = pi/3) would be off
    assert np.abs(np.cos(k * zeta[lb:ub + 1]) * (math.cos(k * t) - math.cos(omega * t))).max() > 1e-4


@pytest.mark.parametrize("p", [VISC, Params(nu_const=0.003, g=(0.0, 0.0, -1.0))],
                         ids=["viscous_quench", "const_nu_gravity"])
def test_conservation_between_walls(p):
    f, g, lb, ub = wall_state(8, 6, 12, grav=True, seed=5)
    f = oracle.fill_wall_ghosts(f, lb, ub)
    d0 = oracle.diagnostics_walls(f, g, p, lb, ub)
    for _ in range(4):
        f, _ = oracle.step_walls(f, g, p, lb, ub)
    d1 = oracle.diagnostics_walls(f, g, p, lb, ub)
    assert abs(d1[0] - d0[0]) <= 1e-13 * abs(d0[0])            # mass
    pscale = max(float(f[1].abs().sum()), float(f[2].abs().sum()))
    assert abs(d1[1] - d0[1]) <= 1e-13 * pscale and abs(d1[2] - d0[2]) <= 1e-13 * pscale
    assert abs(d1[3] - d0[3]) > 1e-8 * pscale                   # the walls push on p_z
    assert d1[7] <= 1e3 * max(d0[7], 1e-16)                     # div B stays at roundoff
    # the odd fields are zero on the boundary points, and so is their rate
    F = oracle.rhs_walls(f, g, p, lb, ub)
    for c in (5, 6):
        assert float(f[c][lb].abs().max()) == 0.0 and float(f[c][ub].abs().max()) == 0.0
        assert float(F[c][lb].abs().max()) <= 1e-12 * float(F[c].abs().max())
        assert float(F[c][ub].abs().max()) <= 1e-12 * float(F[c].abs().max())


def test_ghost_fill_is_the_reflection():
    """Reflection about each boundary point, repeated where the box is thinner
    than the ghost layers (6 physical spacings, 14 ghost planes)."""
    f, g, lb, ub = wall_state(4, 3, 6)
    fp = oracle.fill_wall_ghosts(f, lb, ub)
    for c in range(8):
        s = oracle.WALL_PARITY[c]
        for d in range(1, 4):
            if oracle.Z_FACE[c]:
                assert torch.equal(fp[c][lb + 1 - d], s * fp[c][lb + d])
                assert torch.equal(fp[c][ub + d], s * fp[c][ub + 1 - d])
            else:
                assert torch.equal(fp[c][lb - d], s * fp[c][lb + d])
                assert torch.equal(fp[c][ub + d], s * fp[c][ub - d])
        # every plane: reflection about lb of the reflection about ub, i.e. the
        # shift by the doubled period 2 (ub - lb)
        P = 2 * (ub - lb)
        for k in range(P, fp[c].shape[0]):
            assert torch.equal(fp[c][k], fp[c][k - P])
