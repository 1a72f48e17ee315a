"""Seeded synthetic initial states for the staggered MHD workloads.

This module only evaluates analytic initial conditions at the staggered
positions of the mesh (cell centres for rho and E, lower cell faces for the
momenta and the magnetic field).  It contains none of the method's discrete
arithmetic: no staggered derivative or interpolation, no right-hand side and
no time step.  Both the FP64 oracle and the CUDA path take their inputs from
here.

Layout: every field is a float64 array of shape (nz, ny, nx), x fastest.
Positions (box [0, L) per axis, spacing h = L/n):
    centre  x_i = (i + 1/2) h        (rho, E)
    face    x_i = i h                (px, Bx along x; py, By along y; ...)
The eight prognostic fields are returned in the order
    r, px, py, pz, E, Bx, By, Bz
with E the internal energy per unit volume (rho * e).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FIELD_NAMES = ("r", "px", "py", "pz", "E", "Bx", "By", "Bz")


@dataclass
class Workload:
    """A seeded initial state plus the grid and the physics it is run with."""
    name: str
    shape: tuple            # (nx, ny, nz)
    spacing: tuple          # (dx, dy, dz)
    fields: list            # 8 float64 arrays, shape (nz, ny, nx)
    physics: dict = field(default_factory=dict)


def _coords(n: int, L: float, face: bool) -> np.ndarray:
    h = L / n
    i = np.arange(n, dtype=np.float64)
    return i * h if face else (i + 0.5) * h


def _mesh(shape, lengths, face_axis):
    """3D coordinate arrays (z, y, x order) with one axis on faces (or none)."""
    nx, ny, nz = shape
    Lx, Ly, Lz = lengths
    x = _coords(nx, Lx, face_axis == 0)
    y = _coords(ny, Ly, face_axis == 1)
    z = _coords(nz, Lz, face_axis == 2)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def linear_waves(n: int = 32, seed: int = 1, amp: float = 1e-3,
                 gamma: float = 5.0 / 3.0, b0: float = 0.5) -> Workload:
    """Uniform state rho=1, P=1/gamma (c_s = 1), B=(0,0,b0), plus one
    travelling sound wave and one travelling shear Alfven wave of amplitude
    ``amp``, each with a wave vector 2*pi*m, m drawn from {-2..2}^3 \\ {0}
    (for the Alfven wave m_z != 0) by ``numpy.random.default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    cand = [(a, b, c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)
            if (a, b, c) != (0, 0, 0)]
    ms = np.array(cand[rng.integers(len(cand))], dtype=np.float64)
    cand_a = [m for m in cand if m[2] != 0]
    ma = np.array(cand_a[rng.integers(len(cand_a))], dtype=np.float64)
    phs, pha = rng.uniform(0.0, 2 * math.pi, size=2)

    shape = (n, n, n)
    L = (1.0, 1.0, 1.0)
    h = 1.0 / n
    rho0, P0 = 1.0, 1.0 / gamma
    cs = math.sqrt(gamma * P0 / rho0)
    ks = 2 * math.pi * ms
    khat = ks / np.linalg.norm(ks)
    ka = 2 * math.pi * ma
    ez = np.array([0.0, 0.0, 1.0])
    ea = np.cross(ka, ez)
    if np.linalg.norm(ea) == 0.0:
        ea = np.array([1.0, 0.0, 0.0])
    ea = ea / np.linalg.norm(ea)
    sgn = 1.0 if ka[2] > 0 else -1.0

    def rho_at(X, Y, Z):
        return rho0 + amp * np.sin(ks[0] * X + ks[1] * Y + ks[2] * Z + phs)

    def u_at(d, X, Y, Z):
        snd = amp * cs * khat[d] * np.sin(ks[0] * X + ks[1] * Y + ks[2] * Z + phs)
        alf = amp * ea[d] * np.sin(ka[0] * X + ka[1] * Y + ka[2] * Z + pha)
        return snd + alf

    def b_at(d, X, Y, Z):
        base = b0 if d == 2 else 0.0
        return base - sgn * math.sqrt(rho0) * amp * ea[d] * np.sin(
            ka[0] * X + ka[1] * Y + ka[2] * Z + pha)

    Xc, Yc, Zc = _mesh(shape, L, None)
    r = rho_at(Xc, Yc, Zc)
    E = (P0 + cs * cs * (r - rho0)) / (gamma - 1.0)
    mom, mag = [], []
    for d in range(3):
        X, Y, Z = _mesh(shape, L, d)
        mom.append(rho_at(X, Y, Z) * u_at(d, X, Y, Z))
        mag.append(b_at(d, X, Y, Z))
    fields = [r, mom[0], mom[1], mom[2], E, mag[0], mag[1], mag[2]]
    return Workload("linear_waves", shape, (h, h, h), fields,
                    dict(gamma=gamma, m_sound=ms.tolist(), m_alfven=ma.tolist()))


def orszag_tang(nx: int = 1024, ny: int = 1024, nz: int = 1,
                gamma: float = 5.0 / 3.0) -> Workload:
    """Orszag-Tang vortex in the unit square (uniform in z):
    rho = 25/(36 pi), P = 5/(12 pi), u = (-sin 2 pi y, sin 2 pi x, 0),
    B = B0 (-sin 2 pi y, sin 4 pi x, 0), B0 = 1/sqrt(4 pi)."""
    shape = (nx, ny, nz)
    L = (1.0, 1.0, 1.0)
    rho0 = 25.0 / (36.0 * math.pi)
    P0 = 5.0 / (12.0 * math.pi)
    B0 = 1.0 / math.sqrt(4.0 * math.pi)
    Xc, Yc, Zc = _mesh(shape, L, None)
    r = np.full(Xc.shape, rho0)
    E = np.full(Xc.shape, P0 / (gamma - 1.0))
    X, Y, Z = _mesh(shape, L, 0)
    px = rho0 * -np.sin(2 * math.pi * Y)
    Bx = B0 * -np.sin(2 * math.pi * Y)
    X, Y, Z = _mesh(shape, L, 1)
    py = rho0 * np.sin(2 * math.pi * X)
    By = B0 * np.sin(4 * math.pi * X)
    pz = np.zeros(Xc.shape)
    Bz = np.zeros(Xc.shape)
    fields = [r, px, py, pz, E, Bx, By, Bz]
    return Workload("orszag_tang", shape, (1.0 / nx, 1.0 / ny, 1.0 / nz), fields,
                    dict(gamma=gamma))


def solenoidal_velocity(shape, seed: int, urms: float, kmin: float = 1.0,
                        kmax: float = 4.0, slope: float = -2.0, device: str = "cpu",
                        solenoidal: bool = True):
    """Gaussian random velocity in a periodic unit box with energy spectrum
    E(k) ~ k^slope for kmin <= |m| <= kmax (m the integer wave vector),
    projected onto its divergence-free part unless ``solenoidal`` is False,
    sampled at the three face positions and scaled to the given rms speed.
    Returns three float64 numpy arrays (ux, uy, uz)."""
    import torch

    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    K = int(math.ceil(kmax))
    m1 = np.arange(-K, K + 1)
    MZ, MY, MX = np.meshgrid(m1, m1, m1, indexing="ij")
    kk = np.sqrt(MX ** 2 + MY ** 2 + MZ ** 2)
    band = (kk >= kmin) & (kk <= kmax)
    # Each component of every mode a complex Gaussian; amplitude chosen so the
    # shell energy follows k^slope (shell area ~ k^2).
    coef = (rng.standard_normal((3,) + MX.shape) + 1j * rng.standard_normal((3,) + MX.shape))
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(band, kk ** ((slope - 2.0) / 2.0), 0.0)
    coef = coef * amp
    # Make the field real: c(-m) = conj(c(m)).
    coef = 0.5 * (coef + np.conj(coef[:, ::-1, ::-1, ::-1]))
    # Solenoidal projection c <- c - m (m.c)/|m|^2.
    if solenoidal:
        with np.errstate(divide="ignore", invalid="ignore"):
            mdotc = (MX * coef[0] + MY * coef[1] + MZ * coef[2]) / np.where(kk > 0, kk ** 2, 1.0)
        coef = coef - np.stack([MX, MY, MZ]) * mdotc

    comps = []
    for d, (n_d) in enumerate((nx, ny, nz)):
        spec = torch.zeros((nz, ny, nx // 2 + 1), dtype=torch.complex128, device=device)
        # Fill the rfft half-spectrum directly (mx >= 0).
        sel = band & (MX >= 0)
        vals = coef[d][sel]
        mxv, myv, mzv = MX[sel], MY[sel], MZ[sel]
        # The FFT grid point i sits at i*h, the lower face; along the axes
        # where this component lives at the centre (i+1/2)h add a half-cell phase.
        shift = np.zeros(len(vals))
        for ax, mv, n_ax in ((0, mxv, nx), (1, myv, ny), (2, mzv, nz)):
            if ax != d:
                shift = shift + mv * (0.5 / n_ax)
        phase = np.exp(2j * math.pi * shift)
        v = vals * phase
        # irfftn supplies the mx<0 half as the conjugate mirror; the mx=0
        # plane is Hermitian in (my, mz) by construction, so it is kept as is.
        zi = torch.as_tensor(np.mod(mzv, nz), device=device)
        yi = torch.as_tensor(np.mod(myv, ny), device=device)
        xi = torch.as_tensor(mxv, device=device)
        spec.index_put_((zi, yi, xi), torch.as_tensor(v, device=device), accumulate=True)
        u = torch.fft.irfftn(spec, s=(nz, ny, nx)) * (nx * ny * nz)
        comps.append(u.cpu().numpy())
    rms = math.sqrt(sum(float((c ** 2).mean()) for c in comps))
    s = urms / rms
    return [c * s for c in comps]


def turbulence(n: int = 512, seed: int = 3, urms: float = 0.5, b0: float = 0.3,
               gamma: float = 5.0 / 3.0, device: str = "cpu") -> Workload:
    """Driven-free compressible MHD turbulence start: rho=1, P=1/gamma
    (c_s = 1), B=(0,0,b0), Gaussian random solenoidal velocity with
    E(k) ~ k^-2 for 1 <= |m| <= 4 and rms speed ``urms`` (Mach 0.5)."""
    shape = (n, n, n)
    h = 1.0 / n
    ux, uy, uz = solenoidal_velocity(shape, seed, urms, device=device)
    r = np.ones((n, n, n))
    E = np.full((n, n, n), (1.0 / gamma) / (gamma - 1.0))
    z = np.zeros((n, n, n))
    Bz = np.full((n, n, n), b0)
    fields = [r, ux, uy, uz, E, z, z.copy(), Bz]
    return Workload("turbulence", shape, (h, h, h), fields, dict(gamma=gamma))


def orszag_tang_3d(n: int = 128, seed: int = 4, pert: float = 1e-3,
                   gamma: float = 5.0 / 3.0) -> Workload:
    """Orszag-Tang fields on an n^3 box (uniform in z) plus a seeded random
    velocity perturbation of rms ``pert`` (with a compressive part, so that
    div u is not zero and every axis matters)."""
    w = orszag_tang(n, n, n, gamma)
    du = solenoidal_velocity((n, n, n), seed, pert, solenoidal=False)
    rho0 = w.fields[0][0, 0, 0]
    for d in range(3):
        w.fields[1 + d] = w.fields[1 + d] + rho0 * du[d]
    w.name = "orszag_tang_3d"
    return w


def stratified_atmosphere(nx: int = 768, ny: int = 768, nz: int = 384, zghost: int = 14,
                          lengths=(2.0, 2.0, 1.0), H: float = 0.125, noise: float = 1e-3,
                          seed: int = 5, b0: float = 0.1, gamma: float = 5.0 / 3.0) -> Workload:
    """Isothermal hydrostatic atmosphere for a box walled in z: P = rho (c_iso =
    1), rho = exp(-z/H), which gravity g = 1/H along -z holds in balance,
    E = P/(gamma - 1), B = (0, 0, b0), and Gaussian velocity noise of rms
    ``noise`` per component (``numpy.random.default_rng(seed)``, independent
    at every point).  The arrays hold the nz physical centre planes
    z = (k + 1/2) h, k = 0..nz-1, and ``zghost`` planes beyond each end that
    continue the atmosphere (at rest), so that the walls sit on the first and
    last physical planes (indices zghost and zghost + nz - 1).  Each momentum
    is rho at its own position times the velocity there.  ``physics`` carries
    the gravity and the wall planes."""
    Lx, Ly, Lz = lengths
    h = (Lx / nx, Ly / ny, Lz / nz)
    nzt = nz + 2 * zghost
    kc = np.arange(nzt, dtype=np.float64) - zghost
    zc = ((kc + 0.5) * h[2]).reshape(nzt, 1, 1)     # centres
    zf = (kc * h[2]).reshape(nzt, 1, 1)              # lower z faces
    ones = np.ones((nzt, ny, nx))
    rc = np.exp(-zc / H) * ones
    rf = np.exp(-zf / H) * ones
    rng = np.random.default_rng(seed)
    phys = ((kc >= 0) & (kc < nz)).reshape(nzt, 1, 1)
    u = [noise * rng.standard_normal((nzt, ny, nx)) * phys for _ in range(3)]
    fields = [rc, rc * u[0], rc * u[1], rf * u[2], rc / (gamma - 1.0),
              np.zeros((nzt, ny, nx)), np.zeros((nzt, ny, nx)), np.full((nzt, ny, nx), b0)]
    return Workload("stratified_atmosphere", (nx, ny, nzt), h, fields,
                    dict(gamma=gamma, g=(0.0, 0.0, -1.0 / H), zghost=zghost))


def brio_wu(n: int = 500, L: float = 2.0, gamma: float = 2.0, bn: float = 0.75,
            axis: int = 0) -> Workload:
    """The Brio-Wu MHD shock tube (Sect. "Brio-Wu MHD Shock Tube", Table 2):
    left state rho = 1, P = 1, transverse B = 1; right state rho = 0.125,
    P = 0.1, transverse B = -1; gamma = 2; at rest; the field component along
    the tube ``bn`` (0.75, the usual value for this problem; the paper's table
    does not list it).  On a periodic line of ``n`` cells and length ``L`` along
    ``axis`` (the other two axes one cell), the left state fills the middle
    half [L/4, 3L/4): two mirror-image tubes whose waves do not meet before
    t = 0.15 when L = 2 (each half then matches the paper's 250 cells on a unit
    tube).  The transverse field lies along the next axis."""
    shape = [1, 1, 1]
    shape[axis] = n
    shape = tuple(shape)
    lengths = [1.0, 1.0, 1.0]
    lengths[axis] = L
    h = tuple(lengths[a] / shape[a] for a in range(3))
    tr = (axis + 1) % 3
    nx, ny, nz = shape

    def coord(face_axis):
        X, Y, Z = _mesh(shape, lengths, face_axis)
        return (X, Y, Z)[axis]

    def left(s):
        return (s >= 0.25 * L) & (s < 0.75 * L)

    sc = coord(None)
    r = np.where(left(sc), 1.0, 0.125)
    P = np.where(left(sc), 1.0, 0.1)
    zero = np.zeros((nz, ny, nx))
    B = [zero.copy(), zero.copy(), zero.copy()]
    B[axis] = np.full((nz, ny, nx), bn)
    B[tr] = np.where(left(coord(tr)), 1.0, -1.0)
    fields = [r, zero.copy(), zero.copy(), zero.copy(), P / (gamma - 1.0), B[0], B[1], B[2]]
    return Workload("brio_wu", shape, h, fields, dict(gamma=gamma))


def advection(n: int = 64, sharp: bool = False, u0: float = 1.0, P0: float = 0.01,
              amp: float = 0.5, gamma: float = 5.0 / 3.0) -> Workload:
    """The density advection test (Sect. "Advection"): a density profile
    1 + amp g(x) in a uniform flow u0 along x at uniform pressure P0, on a
    periodic unit line of ``n`` cells; g is a Gaussian of width 6 cells
    (smooth) or a hat 16 cells wide (sharp), centred at x = 1/4.  The exact
    solution is the profile carried at u0; the momentum is the density at the
    x faces times u0."""
    h = 1.0 / n

    def rho(x):
        d = ((x - 0.25 + 0.5) % 1.0) - 0.5
        if sharp:
            return 1.0 + amp * (np.abs(d) < 8 * h)
        return 1.0 + amp * np.exp(-(d / (6 * h)) ** 2)

    xc = ((np.arange(n) + 0.5) * h).reshape(1, 1, n)
    xf = (np.arange(n) * h).reshape(1, 1, n)
    zero = np.zeros((1, 1, n))
    fields = [rho(xc), rho(xf) * u0, zero.copy(), zero.copy(),
              np.full((1, 1, n), P0 / (gamma - 1.0)), zero.copy(), zero.copy(), zero.copy()]
    return Workload("advection", (n, 1, 1), (h, 1.0, 1.0), fields,
                    dict(gamma=gamma, u0=u0, exact=rho))
