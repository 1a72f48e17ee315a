"""Plain FP64 restatement of the Stagger Code MHD right-hand side and step.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never
imports this module.

Every operator is a separate whole-array pass with periodic wrap
(``torch.roll``), in the order the equations are written, with no fusion and
no reordering.  Fields are float64 tensors of shape (nz, ny, nx), x fastest.

Staggering (Sect. "Centering"): rho, E (= rho e) and P at cell centres (C);
momenta, velocities and B on the lower cell faces (Fx = (i-1/2, j, k), ...);
electric field and current on cell edges (Ex = (i, j-1/2, k-1/2),
Ey = (i-1/2, j, k-1/2), Ez = (i-1/2, j-1/2, k)).

Readings taken where the paper is silent or garbled (all shared with the CUDA
path by specification only, never by code):
  R1  product centrings as in the formulas below;
  R2  the viscous stress enters with the dissipative sign (+div tau);
  R3  Richtmyer-Morton nu = nu1|u| + nu3 (c_s + c_A) + nu2 dl_min max(0, -div u);
  R4  log interpolation of rho to faces and edges (do_loginterp);
  R5  max over 3 cells then a 3-cell mean, along x, y, z in turn;
  R6  energy diffusion flux nuE * dn(rho nu_ii) * dd_dn(e);
  R23 eq. (ediffav), with ediffav: the flux nuE * dn(rho nu_ii) * dn(e) *
      dd_dn(ln e - ln <e>_h), <e>_h the mean of e = E/rho over the horizontal
      plane (constant z) of the cell, of the state the RHS is evaluated on;
  R24 eq. (pressure), with lnp_aver: the pressure leaves the diagonal momentum
      flux and its gradient along d at the d face becomes
      exp(dn_d(ln P_aver) + dn_d(ln(P/P_aver))) *
      (dddn_d(ln(P/P_aver)) + dddn_d(ln P_aver)), P_aver the horizontal-plane
      mean of P (the second derivative term vanishes for d = x, y);
  R7  resistivity eta on an edge = nuB * nu of that edge;
  R8  quench: one quenched value per stress / eta J component, the factor
      taken over the directions in which that component is differentiated;
      the ratio's denominator holds the point value |T| of the paper plus
      quench_eps times the 3-cell max of |T| along the direction, which
      only matters where |T| is at roundoff (quench_max3: the 3-cell max of
      |T| alone, an alternative reading);
  R9  Courant step from the stage-1 right-hand side, held for all stages;
  R10 RK constants exactly as printed;
  R13 axes with n = 1 are skipped in dl_min, dl_max, and take dl_min as their
      diffusion length;
  R16 Newtonian cooling enters the energy-per-volume equation as
      -rho (e - e_cool)/t_cool (e relaxes to e_cool on t_cool);
  R17 Smagorinsky: dl_min * Csmag [2 (S_ii^2 - (div u)^2/3 + S_ij^2, i != j)]^1/2
      joins the Richtmyer-Morton nu before the max and the mean;
  R18 the second-order switch of the viscous stress (Sect. "Equations",
      do_2nddiv): the flag of axis a at index (i, j, k) is set where
      |D2_a ln rho| or |D2_a ln e| of the cell with that index exceeds
      d2lnr_lim (D2_a f = f(+1) - 2 f + f(-1) along a); every derivative along
      a in the strain of eq. (itv), in its c1 div u term and in the viscous
      heating built from that strain is then the two-point difference
      (f(i+1) - f(i))/h or (f(i) - f(i-1))/h instead of eq. (deriv);
  R20 chromospheric cooling, eq. (ChromoCool): <e> is the mean of e over the
      horizontal plane (constant z, the vertical axis here) of the cell, of
      the state the right-hand side is evaluated on; rho_bot a parameter;
  R21 coronal thin cooling, eq. (CoronaCool): an energy loss with
      T = Tunit (gamma - 1) e (the paper's T ~ (gamma - 1) e, scaled to kelvin)
      and a prefactor L0 in code units supplied by the caller;
  R19 a stretched vertical mesh (Sect. "Derivatives", the mesh file of
      Sect. "Input and output"): z-derivatives are the index-space stencils
      divided by dz/dk at the centre of the derivative (the cell centre after
      ddup, the lower face after dddn); interpolations stay in index space;
      the diffusion length of z is the local spacing (faces for the Ex, Ey
      edges); dl_min in eq. (RMnu), eq. (nusmag) and the Courant limits is
      the local smallest cell size, and the limits are minima over cells;
      dl_min and dl_max of the anisotropy factor are those of the mesh.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

DT = torch.float64

# Interpolation weights, eq. (interpcoef): a = 1/2 - b - c, b = -25/256, c = 3/256.
IA, IB, IC = 150.0 / 256.0, -25.0 / 256.0, 3.0 / 256.0
# Derivative weights, eq. (derivcoef): c = 3/640, b = -25/384, a = 1 - 3b - 5c.
DA, DB, DC = 225.0 / 192.0, -25.0 / 384.0, 3.0 / 640.0

# Low-storage RK3 constants, eq. (tconst), as printed.
ALPHA = (0.0, -0.641874, -1.31021)
BETA = (0.46173, 0.924087, 0.390614)

_AX = {"x": 2, "y": 1, "z": 0}
NU_FLOOR = 1e-30     # floor under <nu> before its logarithm (ln 0 is not usable)
Q_EPS = 1e-30        # keeps the quench ratio finite where T = 0 and d2T = 0


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    # Stretched vertical mesh (reading R19): dz/dk at the cell centres k and at
    # the lower faces k-1/2 (nz values each), or None for a uniform z.
    zc: tuple = None
    zf: tuple = None

    def n(self, ax):
        return {"x": self.nx, "y": self.ny, "z": self.nz}[ax]

    def h(self, ax):
        return {"x": self.dx, "y": self.dy, "z": self.dz}[ax]

    @property
    def stretched(self):
        return self.zc is not None

    def _zt(self, v):
        return torch.tensor(v, dtype=DT).reshape(self.nz, 1, 1)

    def hc(self, ax):
        """Spacing at cell centres along ax: the divisor of a derivative whose
        output sits at a centre along ax (ddup of a face quantity)."""
        return self._zt(self.zc) if ax == "z" and self.stretched else self.h(ax)

    def hf(self, ax):
        """Spacing at the lower faces along ax: the divisor of a derivative
        whose output sits on a face along ax (dddn of a centred quantity)."""
        return self._zt(self.zf) if ax == "z" and self.stretched else self.h(ax)

    def active(self):
        return [a for a in "xyz" if self.n(a) > 1] or ["x", "y", "z"]

    def _cell_sizes(self, ax):
        return list(self.zc) if ax == "z" and self.stretched else [self.h(ax)]

    @property
    def dl_min(self):
        return min(min(self._cell_sizes(a)) for a in self.active())

    @property
    def dl_max(self):
        return max(max(self._cell_sizes(a)) for a in self.active())

    def dlmin_c(self):
        """Local dl_min at the cell centres: the smallest active cell size
        (a tensor over z on a stretched mesh)."""
        out = None
        for a in self.active():
            out = self.hc(a) if out is None else _vmin(out, self.hc(a))
        return out

    def spacing(self, ax):
        """Diffusion length scale of an axis (R13) on a uniform mesh."""
        return self.h(ax) if self.n(ax) > 1 else self.dl_min

    def spacing_c(self, ax):
        """Diffusion length of an axis at cell centres (R13, R19)."""
        return self.hc(ax) if self.n(ax) > 1 else self.dl_min

    def spacing_f(self, ax):
        """Diffusion length of an axis on its lower faces (R13, R19)."""
        return self.hf(ax) if self.n(ax) > 1 else self.dl_min

    def weights(self):
        """Volume weights of centred and z-face cells for the sums of the
        diagnostics: spacing over mean spacing along a stretched z, else 1."""
        if not self.stretched:
            return 1.0, 1.0
        hbar = sum(self.zc) / self.nz
        return self._zt(self.zc) / hbar, self._zt(self.zf) / hbar


def _vmax(a, b):
    """Maximum of two lengths, each a number or a tensor over z."""
    if torch.is_tensor(a) or torch.is_tensor(b):
        return torch.maximum(torch.as_tensor(a, dtype=DT), torch.as_tensor(b, dtype=DT))
    return max(a, b)


def _vmin(a, b):
    """Minimum of two lengths, each a number or a tensor over z."""
    if torch.is_tensor(a) or torch.is_tensor(b):
        return torch.minimum(torch.as_tensor(a, dtype=DT), torch.as_tensor(b, dtype=DT))
    return min(a, b)


@dataclass
class Params:
    """Physics parameters; defaults follow the paper's namelists (&pde, &run,
    &quench).  All viscosity coefficients zero means ideal MHD."""
    gamma: float = 5.0 / 3.0
    nu1: float = 0.0
    nu2: float = 0.0
    nu3: float = 0.0
    nu_const: float = 0.0    # >0: constant viscosity nu_ij = nu_const (Sect. "Viscosity")
    nuE: float = 1.0
    nuB: float = 1.0
    c1: float = 0.0
    do_quench: bool = False
    qmax: float = 8.0
    qlim: float = 2.0
    log_interp: bool = True
    Cdt: float = 0.4
    Cdtr: float = 0.1
    Cdtd: float = 0.7
    g: tuple = (0.0, 0.0, 0.0)
    t_cool: float = 0.0      # Newtonian cooling time (0: off), Sect. "Newtonian Cooling"
    e_cool: float = 0.0
    rho_cool: float = 1.0
    cool_cut: int = 0        # 0 none, 1 low-density cutoff, 2 high-density cutoff
    csmag: float = 0.0       # Smagorinsky constant, eq. (nusmag) (0: off)
    do_2nddiv: bool = False  # second-order stress derivatives where ln rho, ln e kink (R18)
    d2lnr_lim: float = 0.3
    quench_max3: bool = False   # R8: the 3-cell max of |T| in the quench ratio instead of |T|
    quench_eps: float = 1e-4    # R8: weight of the 3-cell max of |T| added to |T|
    ediffav: bool = False    # energy diffusion of the fluctuations about <e>_h, eq. (ediffav), R23
    lnp_aver: bool = False   # pressure gradient through ln(P/P_aver), eq. (pressure), R24
    t_chromo: float = 0.0    # chromospheric cooling time, eq. (ChromoCool) (0: off), R20
    rho_bot: float = 1.0
    cor_L0: float = 0.0      # coronal thin cooling prefactor in code units (0: off), R21
    cor_Tunit: float = 1.0   # kelvin per code unit of (gamma - 1) e
    # Stellar-atmosphere z boundaries, Sect. "Stellar Atmosphere", reading R26
    bdry_t: float = 1.0      # relaxation time t_bdry of eq. (rein)
    bdry_rho: float = 1.0    # density the bottom inflow relaxes to, eq. (rein)
    bdry_E: float = 1.0      # internal energy per volume the bottom relaxes to
    bdry_u: float = 1.0      # U_bdry of eq. (smooth)
    bdry_B: tuple = (0.0, 0.0, 0.0)   # B_bdry of eq. (bin) (horizontal components used)
    top_rho_lo: float = 0.5  # top ghost density limits, multiples of its plane mean
    top_rho_hi: float = 2.0
    top_e_fac: float = 2.0   # top ghost e within [e_b / fac, e_b * fac]
    top_umax: float = 1.0    # top ghost |u| limit
    top_tpot: float = 0.0    # relaxation time of the top horizontal field toward the
                             # potential field, R27 (0: off)

    def visc_on(self):
        return (self.nu_const > 0 or self.nu1 > 0 or self.nu2 > 0 or self.nu3 > 0
                or self.csmag > 0)


# --------------------------------------------------------------------------
# Staggered operators, eqs. (deriv) and (interp), periodic (Sect. "Derivatives")
# --------------------------------------------------------------------------

def _s(f, ax, k):
    """Value at index i+k along axis ax (periodic)."""
    return torch.roll(f, shifts=-k, dims=_AX[ax])


def up(f, ax):
    """5th-order interpolation to i+1/2, eq. (interp)."""
    return (IA * (f + _s(f, ax, 1)) + IB * (_s(f, ax, -1) + _s(f, ax, 2))
            + IC * (_s(f, ax, -2) + _s(f, ax, 3)))


def dn(f, ax):
    """5th-order interpolation to i-1/2 (the downward variant of eq. (interp))."""
    return (IA * (_s(f, ax, -1) + f) + IB * (_s(f, ax, -2) + _s(f, ax, 1))
            + IC * (_s(f, ax, -3) + _s(f, ax, 2)))


class Spacing:
    """The spacings of one axis at its cell centres (c) and lower faces (f),
    each a number or a tensor over z (R19).  ddup divides by c, dddn by f: in
    this code ddup always takes a face quantity to the centres and dddn a
    centred one to the faces, and the paper's Jacobian is the inverse spacing
    at the centre of the derivative (Sect. "Derivatives")."""

    def __init__(self, c, f):
        self.c, self.f = c, f


def _hc(h):
    return h.c if isinstance(h, Spacing) else h


def _hf(h):
    return h.f if isinstance(h, Spacing) else h


def ddup(f, ax, h):
    """6th-order derivative at i+1/2, eq. (deriv): the index-space stencil
    over the spacing h (a number, a tensor over z, or a Spacing)."""
    return (DA * (_s(f, ax, 1) - f) + DB * (_s(f, ax, 2) - _s(f, ax, -1))
            + DC * (_s(f, ax, 3) - _s(f, ax, -2))) / _hc(h)


def dddn(f, ax, h):
    """6th-order derivative at i-1/2 (downward variant of eq. (deriv))."""
    return (DA * (f - _s(f, ax, -1)) + DB * (_s(f, ax, 1) - _s(f, ax, -2))
            + DC * (_s(f, ax, 2) - _s(f, ax, -3))) / _hf(h)


def ddup2(f, ax, h):
    """Second-order derivative at i+1/2: the two-point difference (R18)."""
    return (_s(f, ax, 1) - f) / _hc(h)


def dddn2(f, ax, h):
    """Second-order derivative at i-1/2: the two-point difference (R18)."""
    return (f - _s(f, ax, -1)) / _hf(h)


def d2_flags(r, E, lim):
    """Second-order switch of the viscous stress (Sect. "Equations",
    do_2nddiv with d2lnr_lim), reading R18: per axis, True where the second
    difference of ln rho or of ln e (e = E/rho) along that axis exceeds lim in
    magnitude, at the cell with the same index."""
    lr, le = torch.log(r), torch.log(E / r)
    flags = {}
    for ax in "xyz":
        d2r = _s(lr, ax, 1) - 2.0 * lr + _s(lr, ax, -1)
        d2e = _s(le, ax, 1) - 2.0 * le + _s(le, ax, -1)
        flags[ax] = (torch.abs(d2r) > lim) | (torch.abs(d2e) > lim)
    return flags


def max3(f, ax):
    """Maximum over the cell and its two neighbours along ax (Sect. "Richtmyer & Morton")."""
    return torch.maximum(torch.maximum(_s(f, ax, -1), f), _s(f, ax, 1))


def smooth3(f, ax):
    """Mean over the cell and its two neighbours along ax."""
    return (_s(f, ax, -1) + f + _s(f, ax, 1)) / 3.0


def quench(T, dirs, p: Params):
    """Quenching of a stress-like component, eq. (quench), reading R8:
    q = |d2 T| / (M + |d2 T|/qmax), T <- T * min(max_d max3_d(q_d), qlim),
    with d2 the second difference along each axis d the component is
    differentiated along.  M is the paper's point value |T| plus quench_eps
    times the 3-cell max of |T| along d: the added term only matters where
    |T| is at roundoff, where the literal ratio is 0/0 (T vanishing by
    symmetry on a grid point) and would carry roundoff to the neighbours
    through the 3-cell max of q.  With quench_max3, M is that 3-cell max
    alone."""
    fac = None
    for ax in dirs:
        d2 = _s(T, ax, 1) - 2.0 * T + _s(T, ax, -1)
        a2 = torch.abs(d2)
        aT = torch.abs(T)
        M = max3(aT, ax) if p.quench_max3 else aT + p.quench_eps * max3(aT, ax)
        q = a2 / (M + a2 / p.qmax + Q_EPS)
        m = max3(q, ax)
        fac = m if fac is None else torch.maximum(fac, m)
    return T * torch.clamp(fac, max=p.qlim)


# --------------------------------------------------------------------------
# Right-hand side F(f): eqs. (mass), (mom), (itv), (ien), (vdiss), (indu), (ohm)
# --------------------------------------------------------------------------

def rhs_parts(f, g: Grid, p: Params):
    """Right-hand side of the eight prognostic equations and the intermediate
    fields it is built from.  Returns a dict; keys d_r ... d_Bz hold F(f)."""
    r, px, py, pz, E, Bx, By, Bz = f
    hx, hy, hz = (Spacing(g.hc(a), g.hf(a)) for a in "xyz")
    out = {}

    # Pointwise primitives (Sect. "Centering"); faces by log interpolation (R4).
    if p.log_interp:
        lr = torch.log(r)
        rx, ry, rz = torch.exp(dn(lr, "x")), torch.exp(dn(lr, "y")), torch.exp(dn(lr, "z"))
    else:
        lr = None
        rx, ry, rz = dn(r, "x"), dn(r, "y"), dn(r, "z")
    ux, uy, uz = px / rx, py / ry, pz / rz
    P = (p.gamma - 1.0) * E
    e = E / r
    divu = ddup(ux, "x", hx) + ddup(uy, "y", hy) + ddup(uz, "z", hz)
    out.update(rx=rx, ry=ry, rz=rz, ux=ux, uy=uy, uz=uz, divu=divu)

    # Current J = curl B on edges (mu = 1).
    Jx = dddn(Bz, "y", hy) - dddn(By, "z", hz)
    Jy = dddn(Bx, "z", hz) - dddn(Bz, "x", hx)
    Jz = dddn(By, "x", hx) - dddn(Bx, "y", hy)
    out.update(Jx=Jx, Jy=Jy, Jz=Jz)

    # Ideal electric field E = -u x B on edges, eq. (ohm).
    Ex = -(dn(uy, "z") * dn(Bz, "y") - dn(uz, "y") * dn(By, "z"))
    Ey = -(dn(uz, "x") * dn(Bx, "z") - dn(ux, "z") * dn(Bz, "x"))
    Ez = -(dn(ux, "y") * dn(By, "x") - dn(uy, "x") * dn(Bx, "y"))

    zero = torch.zeros_like(r)
    Q = zero
    txx = tyy = tzz = txy = tyz = tzx = zero
    ediff = [zero, zero, zero]
    if p.visc_on():
        # Diffusion lengths (R13) at the centres and, for the edges on z faces,
        # at the faces (a stretched z, R19).
        Sx, Sy, Sz = g.spacing_c("x"), g.spacing_c("y"), g.spacing_c("z")
        Sfx, Sfy, Sfz = g.spacing_f("x"), g.spacing_f("y"), g.spacing_f("z")
        dlc = g.dlmin_c()
        if p.nu_const > 0:
            nuc = torch.zeros_like(r) + p.nu_const / dlc
            nxx = nyy = nzz = torch.full_like(r, p.nu_const)
            nxy = nyz = nzx = torch.full_like(r, p.nu_const)
        else:
            # eq. (RMnu) with reading R3; centred speeds.
            uc2 = up(ux, "x") ** 2 + up(uy, "y") ** 2 + up(uz, "z") ** 2
            B2 = up(Bx, "x") ** 2 + up(By, "y") ** 2 + up(Bz, "z") ** 2
            cs = torch.sqrt(p.gamma * P / r)
            ca = torch.sqrt(B2 / r)
            nu = (p.nu1 * torch.sqrt(uc2) + p.nu3 * (cs + ca)
                  + p.nu2 * dlc * torch.clamp(-divu, min=0.0))
            if p.csmag > 0:
                # eq. (nusmag), reading R17: the rate |S| times dl_min joins the
                # velocity-like nu, with Sum_ij over i != j and the off-diagonal
                # squares centred from the edges.
                sxx, syy, szz = ddup(ux, "x", hx), ddup(uy, "y", hy), ddup(uz, "z", hz)
                sxy = 0.5 * (dddn(ux, "y", hy) + dddn(uy, "x", hx))
                syz = 0.5 * (dddn(uy, "z", hz) + dddn(uz, "y", hy))
                szx = 0.5 * (dddn(uz, "x", hx) + dddn(ux, "z", hz))
                s2 = (sxx * sxx + syy * syy + szz * szz - divu * divu / 3.0
                      + 2.0 * (up(up(sxy * sxy, "x"), "y") + up(up(syz * syz, "y"), "z")
                               + up(up(szx * szx, "z"), "x")))
                nu = nu + p.csmag * dlc * torch.sqrt(2.0 * torch.clamp(s2, min=0.0))
            out["nu_raw"] = nu
            # <nu>_{max smooth} (R5).
            for ax in "xyz":
                nu = max3(nu, ax)
            out["nu_max"] = nu
            for ax in "xyz":
                nu = smooth3(nu, ax)
            nuc = nu
            # eq. (nuij): diagonal on centres, off-diagonal by log interpolation.
            lnu = torch.log(torch.clamp(nuc, min=NU_FLOOR))
            nxx, nyy, nzz = Sx * nuc, Sy * nuc, Sz * nuc
            nxy = _vmax(Sx, Sy) * torch.exp(dn(dn(lnu, "x"), "y"))      # Ez edge: z centre
            nyz = _vmax(Sfy, Sfz) * torch.exp(dn(dn(lnu, "y"), "z"))    # Ex edge: z face
            nzx = _vmax(Sfz, Sfx) * torch.exp(dn(dn(lnu, "z"), "x"))    # Ey edge: z face
        out["nu"] = nuc
        # Edge densities (R4).
        if p.log_interp:
            rxy = torch.exp(dn(dn(lr, "x"), "y"))
            ryz = torch.exp(dn(dn(lr, "y"), "z"))
            rzx = torch.exp(dn(dn(lr, "z"), "x"))
        else:
            rxy, ryz, rzx = dn(dn(r, "x"), "y"), dn(dn(r, "y"), "z"), dn(dn(r, "z"), "x")
        # Strain, eq. (itv); with the second-order switch (R18) each derivative
        # along an axis takes the two-point difference where that axis is flagged.
        if p.do_2nddiv:
            fl = d2_flags(r, E, p.d2lnr_lim)
            out["d2flags"] = fl
            h = {"x": hx, "y": hy, "z": hz}

            def dup(f, ax):
                return torch.where(fl[ax], ddup2(f, ax, h[ax]), ddup(f, ax, h[ax]))

            def ddn(f, ax):
                return torch.where(fl[ax], dddn2(f, ax, h[ax]), dddn(f, ax, h[ax]))
        else:
            def dup(f, ax):
                return ddup(f, ax, {"x": hx, "y": hy, "z": hz}[ax])

            def ddn(f, ax):
                return dddn(f, ax, {"x": hx, "y": hy, "z": hz}[ax])
        Sxx, Syy, Szz = dup(ux, "x"), dup(uy, "y"), dup(uz, "z")
        Sxy = 0.5 * (ddn(ux, "y") + ddn(uy, "x"))
        Syz = 0.5 * (ddn(uy, "z") + ddn(uz, "y"))
        Szx = 0.5 * (ddn(uz, "x") + ddn(ux, "z"))
        divs = Sxx + Syy + Szz if p.do_2nddiv else divu
        txx = r * nxx * (Sxx + p.c1 * divs)
        tyy = r * nyy * (Syy + p.c1 * divs)
        tzz = r * nzz * (Szz + p.c1 * divs)
        txy = rxy * nxy * Sxy
        tyz = ryz * nyz * Syz
        tzx = rzx * nzx * Szx
        # Resistive part of E (R7).
        Rx, Ry, Rz = p.nuB * nyz * Jx, p.nuB * nzx * Jy, p.nuB * nxy * Jz
        if p.do_quench:
            txx = quench(txx, "x", p)
            tyy = quench(tyy, "y", p)
            tzz = quench(tzz, "z", p)
            txy = quench(txy, "xy", p)
            tyz = quench(tyz, "yz", p)
            tzx = quench(tzx, "zx", p)
            Rx = quench(Rx, "yz", p)
            Ry = quench(Ry, "zx", p)
            Rz = quench(Rz, "xy", p)
        Ex = Ex + Rx
        Ey = Ey + Ry
        Ez = Ez + Rz
        # Viscous dissipation, eq. (vdiss), and Joule heating, eq. (ien).
        Qv = (txx * Sxx + tyy * Syy + tzz * Szz
              + 2.0 * (up(up(txy * Sxy, "x"), "y") + up(up(tyz * Syz, "y"), "z")
                       + up(up(tzx * Szx, "z"), "x")))
        Qj = up(up(Rx * Jx, "y"), "z") + up(up(Ry * Jy, "z"), "x") + up(up(Rz * Jz, "x"), "y")
        Q = Qv + Qj
        out.update(Qv=Qv, Qj=Qj)
        # Energy diffusion, eq. (ediffuse) with reading R6.
        if p.ediffav:
            # eq. (ediffav), reading R23: only the fluctuations about the
            # horizontal-plane mean of e diffuse.
            le = torch.log(e) - torch.log(e.mean(dim=(1, 2), keepdim=True))
            ediff = [p.nuE * ddup(dn(r * nxx, "x") * dn(e, "x") * dddn(le, "x", hx), "x", hx),
                     p.nuE * ddup(dn(r * nyy, "y") * dn(e, "y") * dddn(le, "y", hy), "y", hy),
                     p.nuE * ddup(dn(r * nzz, "z") * dn(e, "z") * dddn(le, "z", hz), "z", hz)]
        else:
            ediff = [p.nuE * ddup(dn(r * nxx, "x") * dddn(e, "x", hx), "x", hx),
                     p.nuE * ddup(dn(r * nyy, "y") * dddn(e, "y", hy), "y", hy),
                     p.nuE * ddup(dn(r * nzz, "z") * dddn(e, "z", hz), "z", hz)]
        out["ediff"] = ediff
    out.update(txx=txx, tyy=tyy, tzz=tzz, txy=txy, tyz=tyz, tzx=tzx, Ex=Ex, Ey=Ey, Ez=Ez)

    # eq. (mass)
    d_r = -(ddup(px, "x", hx) + ddup(py, "y", hy) + ddup(pz, "z", hz))

    # eq. (mom): -div(rho u u) - grad P + J x B + div tau + rho g (R2).
    if p.lnp_aver:
        # eq. (pressure), reading R24: the gradient through ln(P/P_aver).
        lpa = torch.log(P.mean(dim=(1, 2), keepdim=True)).expand_as(P)
        lq = torch.log(P) - lpa
        gradP = [torch.exp(dn(lpa, "x") + dn(lq, "x")) * dddn(lq, "x", hx),
                 torch.exp(dn(lpa, "y") + dn(lq, "y")) * dddn(lq, "y", hy),
                 torch.exp(dn(lpa, "z") + dn(lq, "z")) * (dddn(lq, "z", hz) + dddn(lpa, "z", hz))]
        out["gradP"] = gradP
        Pf = torch.zeros_like(P)
    else:
        gradP = [0.0, 0.0, 0.0]
        Pf = P
    d_px = (-dddn(up(px, "x") * up(ux, "x") + Pf - txx, "x", hx)
            - ddup(dn(px, "y") * dn(uy, "x") - txy, "y", hy)
            - ddup(dn(px, "z") * dn(uz, "x") - tzx, "z", hz)
            + up(Jy * dn(Bz, "x"), "z") - up(Jz * dn(By, "x"), "y")
            + rx * p.g[0])
    d_py = (-ddup(dn(py, "x") * dn(ux, "y") - txy, "x", hx)
            - dddn(up(py, "y") * up(uy, "y") + Pf - tyy, "y", hy)
            - ddup(dn(py, "z") * dn(uz, "y") - tyz, "z", hz)
            + up(Jz * dn(Bx, "y"), "x") - up(Jx * dn(Bz, "y"), "z")
            + ry * p.g[1])
    d_pz = (-ddup(dn(pz, "x") * dn(ux, "z") - tzx, "x", hx)
            - ddup(dn(pz, "y") * dn(uy, "z") - tyz, "y", hy)
            - dddn(up(pz, "z") * up(uz, "z") + Pf - tzz, "z", hz)
            + up(Jx * dn(By, "z"), "y") - up(Jy * dn(Bx, "z"), "x")
            + rz * p.g[2])
    if p.lnp_aver:
        d_px, d_py, d_pz = d_px - gradP[0], d_py - gradP[1], d_pz - gradP[2]

    # eq. (ien): -div(rho e u) - P div u + Q_visc + eta J^2 (+ energy diffusion).
    d_E = (-(ddup(px * dn(e, "x"), "x", hx) + ddup(py * dn(e, "y"), "y", hy)
             + ddup(pz * dn(e, "z"), "z", hz))
           - P * divu + Q + ediff[0] + ediff[1] + ediff[2])
    if p.t_cool > 0:
        # eq. (NewtonCool), per unit volume (reading R16): -rho (e - e_cool)/t_cool,
        # times the density cutoff of eq. (rhocool).
        qn = -(E - r * p.e_cool) / p.t_cool
        if p.cool_cut:
            x2 = (r / p.rho_cool) ** 2
            qn = qn * ((x2 if p.cool_cut == 1 else 1.0) / (1.0 + x2))
        d_E = d_E + qn
    if p.t_chromo > 0:
        # eq. (ChromoCool), reading R20: -rho (rho/rho_bot)^(5/3) (e - <e>)/t_cool,
        # <e> the mean of e over the horizontal plane (constant z) of the cell.
        emean = e.mean(dim=(1, 2), keepdim=True)
        d_E = d_E - r * (r / p.rho_bot) ** (5.0 / 3.0) * (e - emean) / p.t_chromo
    if p.cor_L0 > 0:
        # eq. (CoronaCool), reading R21: the loss L0 T^(-1/2) rho^2 exp(-(T/10^4 K)^2)
        # with T = Tunit (gamma - 1) e in kelvin; L0 carries the paper's constant,
        # the atomic mass and the code units.
        T = p.cor_Tunit * (p.gamma - 1.0) * e
        d_E = d_E - p.cor_L0 * r * r * torch.exp(-(T / 1e4) ** 2) / torch.sqrt(T)

    # eq. (indu): dB/dt = -curl E.
    d_Bx = -(ddup(Ez, "y", hy) - ddup(Ey, "z", hz))
    d_By = -(ddup(Ex, "z", hz) - ddup(Ez, "x", hx))
    d_Bz = -(ddup(Ey, "x", hx) - ddup(Ex, "y", hy))

    out.update(d_r=d_r, d_px=d_px, d_py=d_py, d_pz=d_pz, d_E=d_E,
               d_Bx=d_Bx, d_By=d_By, d_Bz=d_Bz)
    return out


_DKEYS = ("d_r", "d_px", "d_py", "d_pz", "d_E", "d_Bx", "d_By", "d_Bz")


def rhs(f, g: Grid, p: Params):
    """F(f): the eight time derivatives (r, px, py, pz, E, Bx, By, Bz)."""
    o = rhs_parts(f, g, p)
    return [o[k] for k in _DKEYS]


# --------------------------------------------------------------------------
# Time step: eqs. (dfdt), (ddt), (tupdate), (tconst); Courant eq. (courantcond)
# --------------------------------------------------------------------------

def rk3_step(f, dt, F):
    """One low-storage 3-stage step with derivative function F:
    dfdt <- alpha_i dfdt + F(f); f <- f + beta_i dt dfdt, i = 1..3."""
    f = list(f)
    q = None
    for a, b in zip(ALPHA, BETA):
        Ff = F(f)
        q = Ff if q is None else [a * qi + Fi for qi, Fi in zip(q, Ff)]
        f = [fi + b * dt * qi for fi, qi in zip(f, q)]
    return f


def courant_fields(f, q1, g: Grid, p: Params, nu=None):
    """Per-cell quantities of eq. (courantcond), reading R9: the fastest
    signal speed w = c_s + c_A + |u_perp| at the centre, the relative rate of
    change max(|d rho/dt| / rho, |dE/dt| / E) from the stage-1 derivative q1,
    and the cell-centred viscosity nu (None when no viscosity is on).  The
    limits are reductions of these over the cells (courant_limits)."""
    r, px, py, pz, E, Bx, By, Bz = f
    if p.log_interp:
        lr = torch.log(r)
        rx, ry, rz = torch.exp(dn(lr, "x")), torch.exp(dn(lr, "y")), torch.exp(dn(lr, "z"))
    else:
        rx, ry, rz = dn(r, "x"), dn(r, "y"), dn(r, "z")
    ucx, ucy, ucz = up(px / rx, "x"), up(py / ry, "y"), up(pz / rz, "z")
    bcx, bcy, bcz = up(Bx, "x"), up(By, "y"), up(Bz, "z")
    P = (p.gamma - 1.0) * E
    cs = torch.sqrt(p.gamma * P / r)
    B2 = bcx ** 2 + bcy ** 2 + bcz ** 2
    ca = torch.sqrt(B2 / r)
    u2 = ucx ** 2 + ucy ** 2 + ucz ** 2
    ub = ucx * bcx + ucy * bcy + ucz * bcz
    uperp2 = torch.where(B2 > 0, u2 - ub * ub / torch.where(B2 > 0, B2, 1.0), u2)
    uperp = torch.sqrt(torch.clamp(uperp2, min=0.0))
    w = cs + ca + uperp
    rate = torch.maximum(torch.abs(q1[0]) / r, torch.abs(q1[4]) / E)
    if p.visc_on():
        if nu is None:
            nu = rhs_parts(f, g, p)["nu"]
    else:
        nu = None
    return w, rate, nu


def courant_limits(w, rate, nu, g: Grid, p: Params, dlc=None):
    """eq. (courantcond), reading R9: the wave-speed, rate-of-change and
    diffusion limits from the per-cell fields of courant_fields, taken over
    any set of cells (the maxima are all that matter on a uniform mesh).
    With a stretched z (R19) the limits are minima over the cells of their
    local values, dl the cell's smallest active size (dlc, per cell, default
    the whole grid's).  Returns (dt, (t_wave, t_rate, t_diff))."""
    inf = math.inf
    if g.stretched and dlc is None:
        dlc = g.dlmin_c()
    if g.stretched:
        wr = float(torch.max(w / dlc))
        t_wave = p.Cdt / wr if wr > 0 else inf
    else:
        wmax = float(torch.max(w))
        t_wave = p.Cdt * g.dl_min / wmax if wmax > 0 else inf
    rmax = float(torch.max(rate))
    t_rate = p.Cdtr / rmax if rmax > 0 else inf
    t_diff = inf
    if nu is not None:
        dfac = max(1.0, p.nuE, p.nuB * g.dl_max / g.dl_min)
        if g.stretched:
            dr = float(torch.max(nu / dlc)) * dfac
            t_diff = p.Cdtd / dr if dr > 0 else inf
        else:
            dmax = float(torch.max(nu)) * dfac
            t_diff = p.Cdtd * g.dl_min / dmax if dmax > 0 else inf
    return min(t_wave, t_rate, t_diff), (t_wave, t_rate, t_diff)


def courant_dt(f, q1, g: Grid, p: Params, nu=None):
    """eq. (courantcond), reading R9: the smallest of the wave-speed,
    rate-of-change and diffusion limits, from the state and its stage-1
    derivative.  Returns (dt, (t_wave, t_rate, t_diff))."""
    w, rate, nu = courant_fields(f, q1, g, p, nu)
    return courant_limits(w, rate, nu, g, p)


def step(f, g: Grid, p: Params, dt=None):
    """One full time step.  With dt None the step comes from the Courant
    condition evaluated on the stage-1 derivative (R9).  Returns (f_new, dt)."""
    f = [fi.to(DT) for fi in f]
    if dt is None:
        parts = rhs_parts(f, g, p)
        q1 = [parts[k] for k in _DKEYS]
        dt, _ = courant_dt(f, q1, g, p, nu=parts.get("nu"))
    return rk3_step(f, dt, lambda s: rhs(s, g, p)), dt


def step_adjoint(f, dt, lam, g: Grid, p: Params):
    """Vector-Jacobian product of one fixed-dt step: returns the cotangent of
    the input state given the cotangent ``lam`` of the output state.  The
    reverse sweep is taken by torch.autograd through the forward above."""
    x = [fi.detach().to(DT).clone().requires_grad_(True) for fi in f]
    y = rk3_step(x, dt, lambda s: rhs(s, g, p))
    grads = torch.autograd.grad(y, x, grad_outputs=[l.to(DT) for l in lam])
    return [gr.detach() for gr in grads]


# --------------------------------------------------------------------------
# Diagnostics (FP64 sums; discrete div B at cell centres)
# --------------------------------------------------------------------------

def diagnostics(f, g: Grid, p: Params):
    """[sum r, sum px, sum py, sum pz, sum E, kinetic, magnetic, max|divB|,
    rms divB, non-finite count] with kinetic = sum 1/2 p.u over faces and
    magnetic = sum 1/2 B^2 over faces: plain sums over cells, each term
    weighted by its cell's z size over the mean one on a stretched z (R19),
    z-face quantities by the face spacing; these are the totals the discrete
    equations conserve."""
    r, px, py, pz, E, Bx, By, Bz = [fi.to(DT) for fi in f]
    if p.log_interp:
        lr = torch.log(r)
        rx, ry, rz = torch.exp(dn(lr, "x")), torch.exp(dn(lr, "y")), torch.exp(dn(lr, "z"))
    else:
        rx, ry, rz = dn(r, "x"), dn(r, "y"), dn(r, "z")
    wc, wf = g.weights()
    kin = 0.5 * ((px * px / rx + py * py / ry) * wc + pz * pz / rz * wf).sum()
    mag = 0.5 * ((Bx * Bx + By * By) * wc + Bz * Bz * wf).sum()
    divb = ddup(Bx, "x", g.hc("x")) + ddup(By, "y", g.hc("y")) + ddup(Bz, "z", g.hc("z"))
    nonfinite = sum(int((~torch.isfinite(fi)).sum()) for fi in (r, px, py, pz, E, Bx, By, Bz))
    return [float((r * wc).sum()), float((px * wc).sum()), float((py * wc).sum()),
            float((pz * wf).sum()), float((E * wc).sum()),
            float(kin), float(mag), float(divb.abs().max()), float(divb.pow(2).mean().sqrt()),
            float(nonfinite)]


# --------------------------------------------------------------------------
# Closed walls along z, Sect. "Boundary Conditions" ("Closed"), reading R22
# --------------------------------------------------------------------------
#
# The box is periodic in x and y and closed at two boundary points in z, the
# cell-centre planes lb and ub of the arrays (planes outside [lb, ub] are
# ghost planes).  Every field is continued across a boundary point by
# reflection about it, with the parity of the field: rho, E (so e), the
# parallel momenta and B_z even; the normal momentum p_z and the parallel
# field components B_x, B_y odd (the paper's symmetric parallel velocity,
# anti-symmetric normal velocity and anti-symmetric parallel field; B_z even
# keeps div B = 0 across the wall).  The right-hand side of the closed box is
# then the periodic right-hand side of the mirror-symmetric state on the box
# doubled about one wall, restricted to the physical planes: centres lb..ub,
# z faces lb+1..ub.  Gravity along z is odd under the reflection, so it acts
# with its own sign on the physical faces only.

WALL_PARITY = (1.0, 1.0, 1.0, -1.0, 1.0, -1.0, -1.0, 1.0)   # r px py pz E Bx By Bz
Z_FACE = (False, False, False, True, False, False, False, True)


def mirror_extend(f, lb, ub):
    """The doubled periodic state (period P = 2 (ub - lb) planes along z) of
    the physical planes of a closed box: doubled centre plane m holds
    physical centre lb + m for 0 <= m <= ub - lb and the reflection about ub
    (times the parity) beyond; doubled face plane m (the face below doubled
    centre m) holds physical face lb + m for 1 <= m <= ub - lb and the
    reflection beyond.  Odd centred fields vanish on the boundary points."""
    L = ub - lb
    P = 2 * L
    out = []
    for c, a in enumerate(f):
        s = WALL_PARITY[c]
        d = torch.empty((P,) + tuple(a.shape[1:]), dtype=a.dtype)
        for m in range(P):
            if Z_FACE[c]:
                if 1 <= m <= L:
                    d[m] = a[lb + m]
                else:
                    mm = m if m > L else P
                    d[m] = s * a[2 * ub - lb - mm + 1]
            else:
                if m <= L:
                    d[m] = a[lb + m] if (s > 0 or (m != 0 and m != L)) else 0.0 * a[lb + m]
                else:
                    d[m] = s * a[2 * ub - lb - m]
        out.append(d)
    return out


def fill_wall_ghosts(f, lb, ub):
    """The state with its ghost planes set to the doubled periodic extension
    of its physical planes (reading R22): plane k of a centred field is plane
    m = (k - lb) mod P of the doubled state (P = 2 (ub - lb)), and likewise for
    the z faces; the odd centred fields are zeroed on the boundary points.
    This is the continuation the right-hand side of the closed box implies,
    written into the arrays' own ghost planes (repeated reflections when the
    box is thinner than the ghost layers)."""
    nz = f[0].shape[0]
    L = ub - lb
    P = 2 * L
    d = mirror_extend(f, lb, ub)
    out = [a.clone() for a in f]
    for c in range(8):
        for k in range(nz):
            m = (k - lb) % P
            out[c][k] = d[c][m]
    return out


def _doubled_grid(g: Grid, P):
    return Grid(g.nx, g.ny, P, g.dx, g.dy, g.dz)


def rhs_walls(f, g: Grid, p: Params, lb, ub):
    """F(f) of the closed box (reading R22): the periodic right-hand side of
    the doubled mirror-symmetric state, restricted to the physical planes, with
    gravity along z on the physical z faces.  Ghost planes of the result are
    zero."""
    d = mirror_extend([fi.to(DT) for fi in f], lb, ub)
    L = ub - lb
    pd = Params(**{**p.__dict__, "g": (p.g[0], p.g[1], 0.0)})
    parts = rhs_parts(d, _doubled_grid(g, 2 * L), pd)
    Fd = [parts[k] for k in _DKEYS]
    out = [torch.zeros_like(fi, dtype=DT) for fi in f]
    for c in range(8):
        if Z_FACE[c]:
            out[c][lb + 1:ub + 1] = Fd[c][1:L + 1]
        else:
            out[c][lb:ub + 1] = Fd[c][0:L + 1]
    if p.g[2] != 0.0:
        out[3][lb + 1:ub + 1] += parts["rz"][1:L + 1] * p.g[2]
    return out


def courant_walls(f, q1, g: Grid, p: Params, lb, ub):
    """eq. (courantcond) of the closed box: the limits over the physical planes,
    taken on the doubled state (whose other half repeats them)."""
    L = ub - lb
    d = mirror_extend([fi.to(DT) for fi in f], lb, ub)
    qd = mirror_extend([qi.to(DT) for qi in q1], lb, ub)
    gd = _doubled_grid(g, 2 * L)
    return courant_dt(d, qd, gd, Params(**{**p.__dict__, "g": (p.g[0], p.g[1], 0.0)}))


def step_walls(f, g: Grid, p: Params, lb, ub, dt=None):
    """One full time step of the closed box (R9 for the Courant step); the
    ghost planes of the result hold the reflection of its physical planes."""
    f = fill_wall_ghosts([fi.to(DT) for fi in f], lb, ub)
    if dt is None:
        q1 = rhs_walls(f, g, p, lb, ub)
        dt, _ = courant_walls(f, q1, g, p, lb, ub)
    out = rk3_step(f, dt, lambda s: rhs_walls(s, g, p, lb, ub))
    return fill_wall_ghosts(out, lb, ub), dt


def diagnostics_walls(f, g: Grid, p: Params, lb, ub):
    """The totals of the closed box: half the plain sums over the doubled
    state (centre planes lb, ub count one half, faces lb+1..ub once) -- the
    totals the closed box conserves -- except the sum of p_z, which is odd and
    sums to zero over the doubled state, taken as the plain sum over the
    physical faces lb+1..ub; max |div B| and rms div B over the doubled
    centres; the non-finite count of the physical planes."""
    L = ub - lb
    d = mirror_extend([fi.to(DT) for fi in f], lb, ub)
    out = diagnostics(d, _doubled_grid(g, 2 * L), p)
    for i in range(7):
        out[i] = 0.5 * out[i]
    out[3] = float(f[3][lb + 1:ub + 1].to(DT).sum())
    out[9] = float(sum(int((~torch.isfinite(fi[lb:ub + 1])).sum()) for fi in f))
    return out


# --------------------------------------------------------------------------
# Rigid walls along z, Sect. "Boundary Conditions" ("Rigid"), reading R25
# --------------------------------------------------------------------------
#
# The arrays hold ghost planes below the boundary plane lb and above the
# boundary plane ub; a ghost plane is one whose index lies outside lb..ub,
# for every field whatever its staggering (so the z faces lb and ub are
# physical).  The ghost values of rho, E and B are the caller's and never
# change: their time derivatives are zero.  The ghost momenta are set, before
# every evaluation of the right-hand side, so that the velocity of each ghost
# point is the velocity of the boundary plane at the same (x, y):
# p_d(k) = rho_d(k) u_d(b), u_d = p_d / rho_d, rho_d the density at the
# position of p_d (the same face density as the right-hand side's), b = lb
# below and ub above.  The right-hand side of the physical planes is then the
# right-hand side of the padded arrays, whose ghost layers cover the reach of
# the operators (at least 14 planes), so that the periodic wrap of the padded
# arrays never reaches a physical plane.


def face_densities(f, p: Params):
    """rho at the x, y and z faces as the right-hand side forms it (R4)."""
    r = f[0].to(DT)
    if p.log_interp:
        lr = torch.log(r)
        return [torch.exp(dn(lr, a)) for a in "xyz"]
    return [dn(r, a) for a in "xyz"]


def fill_rigid_ghosts(f, p: Params, lb, ub):
    """The state with the momenta of its ghost planes (indices outside lb..ub)
    set to the face density there times the velocity of the boundary plane
    (lb below, ub above) at the same (x, y), reading R25; rho, E and B are
    returned unchanged."""
    out = [fi.to(DT).clone() for fi in f]
    rf = face_densities(out, p)
    for d in range(3):
        c = 1 + d
        u = out[c] / rf[d]
        out[c][:lb] = rf[d][:lb] * u[lb]
        out[c][ub + 1:] = rf[d][ub + 1:] * u[ub]
    return out


def rhs_rigid(f, g: Grid, p: Params, lb, ub):
    """F(f) of the box with rigid z walls (reading R25): the right-hand side of
    the state with its ghost momenta filled, on the physical planes lb..ub of
    every field; zero on the ghost planes."""
    fr = fill_rigid_ghosts(f, p, lb, ub)
    F = rhs(fr, g, p)
    for c in range(8):
        F[c][:lb] = 0.0
        F[c][ub + 1:] = 0.0
    return F


def courant_rigid(f, q1, g: Grid, p: Params, lb, ub):
    """eq. (courantcond) of the box with rigid z walls: the limits over the
    physical centre planes lb..ub of the filled state."""
    fr = fill_rigid_ghosts(f, p, lb, ub)
    w, rate, nu = courant_fields(fr, q1, g, p)
    sl = slice(lb, ub + 1)
    return courant_limits(w[sl], rate[sl], None if nu is None else nu[sl], g, p)


def step_rigid(f, g: Grid, p: Params, lb, ub, dt=None):
    """One full time step with rigid z walls (R9 for the Courant step); the
    ghost momenta of the result are filled from its own boundary planes."""
    f = fill_rigid_ghosts(f, p, lb, ub)
    if dt is None:
        q1 = rhs_rigid(f, g, p, lb, ub)
        dt, _ = courant_rigid(f, q1, g, p, lb, ub)
    out = rk3_step(f, dt, lambda s: rhs_rigid(s, g, p, lb, ub))
    return fill_rigid_ghosts(out, p, lb, ub), dt


def diagnostics_rigid(f, g: Grid, p: Params, lb, ub):
    """The totals of the physical planes lb..ub (every field, centres and z
    faces alike) of the filled state: plain sums, kinetic and magnetic energy,
    max |div B| and rms div B over the centres lb..ub, the non-finite count of
    the physical planes."""
    fr = fill_rigid_ghosts(f, p, lb, ub)
    r, px, py, pz, E, Bx, By, Bz = fr
    rx, ry, rz = face_densities(fr, p)
    sl = slice(lb, ub + 1)
    kin = 0.5 * (px * px / rx + py * py / ry + pz * pz / rz)[sl].sum()
    mag = 0.5 * (Bx * Bx + By * By + Bz * Bz)[sl].sum()
    divb = (ddup(Bx, "x", g.hc("x")) + ddup(By, "y", g.hc("y")) + ddup(Bz, "z", g.hc("z")))[sl]
    nonfinite = sum(int((~torch.isfinite(fi[sl])).sum()) for fi in f)
    return [float(r[sl].sum()), float(px[sl].sum()), float(py[sl].sum()), float(pz[sl].sum()),
            float(E[sl].sum()), float(kin), float(mag), float(divb.abs().max()),
            float(divb.pow(2).mean().sqrt()), float(nonfinite)]


# --------------------------------------------------------------------------
# Stellar-atmosphere z boundaries, Sect. "Boundary Conditions" ("Stellar
# Atmosphere"), reading R26
# --------------------------------------------------------------------------
#
# The arrays carry ghost planes beyond the boundary planes lb and ub as for
# the closed walls: physical centres lb..ub and z faces lb+1..ub, every other
# plane a ghost plane whose time derivative is zero.  The bottom boundary
# (the interior one, inside the convection zone) is the end gravity points to:
# lb when g_z < 0, ub when g_z > 0; the other end is the top (the exterior
# boundary, in the atmosphere).  s is the outward index direction at an end
# (-1 at lb, +1 at ub); the outward velocity there is U = s u_z, u_z taken on
# the z face nearest the boundary plane inside the box (lb+1 or ub).
#
# Before every evaluation of the right-hand side the ghost planes are filled:
#  - ln rho and e = E/rho: linear extrapolation from the boundary plane b and
#    its inner neighbour, x(b + s j) = x(b) + j (x(b) - x(b - s)); at the top
#    the ghost density is then limited to [lo, hi] times the mean of the
#    extrapolated ghost density over its plane, and e to [e_b/fac, e_b fac]
#    about the boundary value at the same (x, y); E = rho e;
#  - bottom momenta symmetric about the boundary point: p_x, p_y of plane
#    b + s j from plane b - s j, p_z of face m from face 2b + 1 - m;
#  - top momenta p_d = rho_d u_d, the ghost velocity the boundary velocity at
#    the same (x, y) limited to |u| <= top_umax (p_x, p_y from plane b, p_z
#    from the nearest inside face), rho_d the face density of the filled rho;
#  - B: every component extrapolated linearly (B_x, B_y from the plane b and
#    its inner neighbour, B_z from the two nearest inside faces); at the
#    bottom the horizontal components are then blended toward B_bdry, eq.
#    (bin), B_h = (1 - f) B_h + f B_bdry, f = 1 / (1 + exp(U / U_bdry)), eq.
#    (smooth), U the outward velocity of the column (f -> 1 in inflows).
# After the right-hand side F of the filled state:
#  - bottom plane b, per column, with the same f: the inflow part relaxes rho
#    and E (per volume) to bdry_rho, bdry_E on bdry_t, eq. (rein), and damps
#    the horizontal momenta toward their plane mean on bdry_t; the outflow
#    part relaxes E the same way and adds to d rho/dt the change that keeps
#    the entropy, eqs. (constS) to (addderiv) for the ideal gas, where
#    (d ln P/d ln rho)_e = 1 and (d ln P/d e)_rho = 1/e give a = 0 and
#    b = 1/(gamma e): d rho/dt += ((bdry_E - E)/t - dE/dt) / (gamma e);
#    mixed: dE/dt = (bdry_E - E)/t, d rho/dt = f (bdry_rho - rho)/t +
#    (1 - f)(F_rho + ((bdry_E - E)/t - F_E)/(gamma e)), dp_h/dt = F_ph -
#    f (p_h - <p_h>_b)/t;
#  - top plane b, eq. (rbdrylo): the vertical divergence of the mass flux is
#    replaced by the inward mass flux over the pressure scale height,
#    d rho/dt += ddup_z(p_z) + s up_z(p_z) / H_P, H_P = (gamma - 1) e / |g_z|.
# With top_tpot > 0 (reading R27), the horizontal field of the top plane also
# relaxes toward the potential field of its normal field: dB_h/dt +=
# (B_pot,h - (B_h - <B_h>))/top_tpot, B_pot,h the horizontal components, on
# the plane, of the current-free field that decays outward from the normal
# field B_z of the inside face nearest the plane (zero horizontal mean).


def _open_ends(p: Params, lb, ub):
    """(bottom plane, its outward sign), (top plane, its outward sign)."""
    if p.g[2] < 0:
        return (lb, -1), (ub, 1)
    if p.g[2] > 0:
        return (ub, 1), (lb, -1)
    raise ValueError("stellar-atmosphere boundaries need gravity along z")


def _inside_face(b, s):
    """The z face nearest the boundary plane b inside the box."""
    return b + 1 if s < 0 else b


def _outward_u(f, p: Params, b, s):
    """Outward velocity s u_z of each column at the boundary plane b."""
    rz = face_densities(f, p)[2]
    m = _inside_face(b, s)
    return s * f[3][m] / rz[m]


def fill_open_ghosts(f, p: Params, lb, ub):
    """The state with the ghost planes of the stellar-atmosphere boundaries
    filled (reading R26)."""
    out = [fi.to(DT).clone() for fi in f]
    nz = out[0].shape[0]
    G = min(lb, nz - 1 - ub)
    (bb, sb), (bt, st) = _open_ends(p, lb, ub)
    lr = torch.log(out[0])
    e = out[4] / out[0]
    for b, s, top in ((bb, sb, False), (bt, st, True)):
        dl = lr[b] - lr[b - s]
        de = e[b] - e[b - s]
        for j in range(1, G + 1):
            k = b + s * j
            rj = torch.exp(lr[b] + j * dl)
            ej = e[b] + j * de
            if top:
                m = rj.mean()
                rj = torch.clamp(rj, min=p.top_rho_lo * m, max=p.top_rho_hi * m)
                ej = torch.minimum(torch.maximum(ej, e[b] / p.top_e_fac), e[b] * p.top_e_fac)
            out[0][k] = rj
            out[4][k] = rj * ej
    # momenta: symmetric about the bottom boundary point
    for j in range(1, G + 1):
        k = bb + sb * j
        for c in (1, 2):
            out[c][k] = out[c][bb - sb * j]
    for m in range(nz):
        if (sb < 0 and m <= lb) or (sb > 0 and m >= ub + 1):
            out[3][m] = out[3][2 * bb + 1 - m]
    rf = face_densities(out, p)
    mt = _inside_face(bt, st)
    ub_top = [out[1][bt] / rf[0][bt], out[2][bt] / rf[1][bt], out[3][mt] / rf[2][mt]]
    ub_top = [torch.clamp(u, min=-p.top_umax, max=p.top_umax) for u in ub_top]
    for j in range(1, G + 1):
        k = bt + st * j
        out[1][k] = rf[0][k] * ub_top[0]
        out[2][k] = rf[1][k] * ub_top[1]
    for m in range(nz):
        top_ghost = (m <= lb) if st < 0 else (m >= ub + 1)
        if top_ghost:
            out[3][m] = rf[2][m] * ub_top[2]
    # magnetic field: linear extrapolation, then the bottom blending with the
    # outward velocity of the filled state
    f_bot = 1.0 / (1.0 + torch.exp(_outward_u(out, p, bb, sb) / p.bdry_u))
    for b, s, top in ((bb, sb, False), (bt, st, True)):
        mi = _inside_face(b, s)
        for j in range(1, G + 1):
            k = b + s * j
            for c in (5, 6):
                v = out[c][b] + j * (out[c][b] - out[c][b - s])
                if not top:
                    v = (1.0 - f_bot) * v + f_bot * p.bdry_B[c - 5]
                out[c][k] = v
        for m in range(nz):
            d = (mi - m) if s < 0 else (m - mi)     # faces beyond the inside face
            ghost = (m <= lb) if s < 0 else (m >= ub + 1)
            if ghost:
                out[7][m] = out[7][mi] + d * (out[7][mi] - out[7][mi - s])
    return out


def potential_horizontal(bz, g: Grid, s):
    """The horizontal components, at the x faces and the y faces of a plane,
    of the potential (current-free) field above a plane whose normal field is
    bz (cell centres in x and y, shape (ny, nx)), decaying in the outward
    direction s along z (reading R27): per horizontal Fourier mode k,
    B_h = -i s (k_h / |k|) B_z, B = -grad Phi with Phi ~ exp(-|k| zeta).  The
    mean and the Nyquist modes carry no potential part.  The faces sit half a
    cell below the centres along their axis, which is a phase factor."""
    ny, nx = bz.shape
    Lx, Ly = g.nx * g.dx, g.ny * g.dy
    mx = torch.fft.fftfreq(nx, d=1.0 / nx, dtype=DT)          # integer mode numbers
    my = torch.fft.fftfreq(ny, d=1.0 / ny, dtype=DT)
    MY, MX = torch.meshgrid(my, mx, indexing="ij")
    kx, ky = 2 * math.pi * MX / Lx, 2 * math.pi * MY / Ly
    kk = torch.sqrt(kx ** 2 + ky ** 2)
    keep = (kk > 0)
    if nx % 2 == 0:
        keep = keep & (MX != -nx // 2)
    if ny % 2 == 0:
        keep = keep & (MY != -ny // 2)
    bh = torch.fft.fft2(bz.to(DT))
    safe = torch.where(keep, kk, torch.ones_like(kk))
    px = torch.where(keep, -1j * s * (kx / safe) * bh, torch.zeros_like(bh))
    py = torch.where(keep, -1j * s * (ky / safe) * bh, torch.zeros_like(bh))
    px = px * torch.exp(-1j * math.pi * MX / nx)              # x faces: x_c - h/2
    py = py * torch.exp(-1j * math.pi * MY / ny)
    return torch.fft.ifft2(px).real, torch.fft.ifft2(py).real


def rhs_open(f, g: Grid, p: Params, lb, ub):
    """F(f) with the stellar-atmosphere z boundaries (reading R26): the
    right-hand side of the filled state with the bottom and top corrections
    on the boundary planes, zero on the ghost planes."""
    fo = fill_open_ghosts(f, p, lb, ub)
    F = rhs(fo, g, p)
    (bb, sb), (bt, st) = _open_ends(p, lb, ub)
    r, E = fo[0], fo[4]
    t = p.bdry_t
    # bottom, eqs. (rein), (constS) to (addderiv)
    fb = 1.0 / (1.0 + torch.exp(_outward_u(fo, p, bb, sb) / p.bdry_u))
    eb = E[bb] / r[bb]
    dE = (p.bdry_E - E[bb]) / t
    Fr_out = F[0][bb] + (dE - F[4][bb]) / (p.gamma * eb)
    F[0][bb] = fb * (p.bdry_rho - r[bb]) / t + (1.0 - fb) * Fr_out
    F[4][bb] = dE.clone()
    for c in (1, 2):
        F[c][bb] = F[c][bb] - fb * (fo[c][bb] - fo[c][bb].mean()) / t
    # top, eq. (rbdrylo)
    hz = Spacing(g.hc("z"), g.hf("z"))
    HP = (p.gamma - 1.0) * E[bt] / r[bt] / abs(p.g[2])
    F[0][bt] = F[0][bt] + ddup(fo[3], "z", hz)[bt] + st * up(fo[3], "z")[bt] / HP
    if p.top_tpot > 0:
        # R27: the top horizontal field relaxes toward the potential field.
        bxp, byp = potential_horizontal(fo[7][_inside_face(bt, st)], g, st)
        for c, target in ((5, bxp), (6, byp)):
            fluct = fo[c][bt] - fo[c][bt].mean()
            F[c][bt] = F[c][bt] + (target - fluct) / p.top_tpot
    for c in range(8):
        if Z_FACE[c]:
            F[c][:lb + 1] = 0.0
            F[c][ub + 1:] = 0.0
        else:
            F[c][:lb] = 0.0
            F[c][ub + 1:] = 0.0
    return F


def courant_open(f, q1, g: Grid, p: Params, lb, ub):
    """eq. (courantcond) with the stellar-atmosphere boundaries: the limits
    over the physical centre planes lb..ub of the filled state."""
    fo = fill_open_ghosts(f, p, lb, ub)
    w, rate, nu = courant_fields(fo, q1, g, p)
    sl = slice(lb, ub + 1)
    return courant_limits(w[sl], rate[sl], None if nu is None else nu[sl], g, p)


def step_open(f, g: Grid, p: Params, lb, ub, dt=None):
    """One full time step with the stellar-atmosphere boundaries (R9 for the
    Courant step); the ghost planes of the result are filled from it."""
    f = fill_open_ghosts(f, p, lb, ub)
    if dt is None:
        q1 = rhs_open(f, g, p, lb, ub)
        dt, _ = courant_open(f, q1, g, p, lb, ub)
    out = rk3_step(f, dt, lambda s: rhs_open(s, g, p, lb, ub))
    return fill_open_ghosts(out, p, lb, ub), dt


def diagnostics_open(f, g: Grid, p: Params, lb, ub):
    """The totals of the physical planes (centres lb..ub, z faces lb+1..ub) of
    the filled state: plain sums, kinetic and magnetic energy, max |div B| and
    rms div B over the centres lb..ub, the non-finite count of the physical
    planes."""
    fo = fill_open_ghosts(f, p, lb, ub)
    r, px, py, pz, E, Bx, By, Bz = fo
    rx, ry, rz = face_densities(fo, p)
    c = slice(lb, ub + 1)
    fz = slice(lb + 1, ub + 1)
    kin = 0.5 * ((px * px / rx + py * py / ry)[c].sum() + (pz * pz / rz)[fz].sum())
    mag = 0.5 * ((Bx * Bx + By * By)[c].sum() + (Bz * Bz)[fz].sum())
    divb = (ddup(Bx, "x", g.hc("x")) + ddup(By, "y", g.hc("y")) + ddup(Bz, "z", g.hc("z")))[c]
    nonfinite = sum(int((~torch.isfinite(fi[c])).sum()) for fi in f)
    return [float(r[c].sum()), float(px[c].sum()), float(py[c].sum()), float(pz[fz].sum()),
            float(E[c].sum()), float(kin), float(mag), float(divb.abs().max()),
            float(divb.pow(2).mean().sqrt()), float(nonfinite)]
