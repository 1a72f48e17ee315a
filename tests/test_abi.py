"""The C-ABI library loads and exports every function include/stagger.h
declares; argument validation rejects bad input before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "stagger.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(stagger_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def S():
    import paper_2405_02483_gb300 as S
    return S


def test_every_declared_symbol_is_exported(S):
    names = _declared()
    assert len(names) >= 15
    lib = ctypes.CDLL(S.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    bound = {n for n, _, _ in S.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_params_default_matches_namelists(S):
    p = S.default_params()
    assert p.gamma == pytest.approx(5 / 3)
    assert (p.Cdt, p.Cdtr, p.Cdtd) == (0.4, 0.1, 0.7)
    assert (p.qmax, p.qlim, p.log_interp) == (8.0, 2.0, 1)
    assert (p.nu1, p.nu2, p.nu3, p.nu_const) == (0.0, 0.0, 0.0, 0.0)
    assert S.lib.stagger_params_default(None) == S.EINVAL


def test_create_rejects_bad_arguments_without_gpu(S):
    h = ctypes.c_void_p()
    p = S.default_params()
    bad_grids = [S.Grid(0, 8, 8, 1, 1, 1), S.Grid(8, 8, 8, 0, 1, 1), S.Grid(8, -1, 8, 1, 1, 1),
                 S.Grid(2048, 2048, 1024, 1, 1, 1), S.Grid(4, 65536, 1, 1, 1, 1),
                 S.Grid(4, 1, 65536, 1, 1, 1)]
    for g in bad_grids:
        assert S.lib.stagger_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h)) == S.EINVAL
    g = S.Grid(8, 8, 8, 0.1, 0.1, 0.1)
    for field, val in [("gamma", 1.0), ("nu1", -1.0), ("Cdt", 0.0)]:
        q = S.default_params(**{field: val})
        assert S.lib.stagger_create(ctypes.byref(g), ctypes.byref(q), ctypes.byref(h)) == S.EINVAL
    q = S.default_params(do_quench=1, qmax=0.0)
    assert S.lib.stagger_create(ctypes.byref(g), ctypes.byref(q), ctypes.byref(h)) == S.EINVAL
    assert S.lib.stagger_create(None, ctypes.byref(p), ctypes.byref(h)) == S.EINVAL
    assert S.lib.stagger_create(ctypes.byref(g), ctypes.byref(p), None) == S.EINVAL


def test_mesh_and_switch_parameters_are_validated_without_gpu(S):
    h = ctypes.c_void_p()
    g = S.Grid(8, 8, 6, 0.1, 0.1, 0.1)
    good = [0.1] * 6
    cases = [dict(zc=good),                                  # zf missing
             dict(zc=good, zf=good[:5] + [0.0]),             # a non-positive spacing
             dict(zc=good[:5] + [float("nan")], zf=good),    # not finite
             dict(do_2nddiv=2), dict(do_2nddiv=1, d2lnr_lim=float("inf")),
             dict(scalar_cells=2), dict(ediffav=2), dict(lnp_aver=2), dict(lnp_aver=-1),
             dict(lnp_aver=1, fuse_flux_div=1)]   # k_fdiv does not take ln(P/P_aver)
    for kw in cases:
        q = S.default_params(**kw)
        assert S.lib.stagger_create(ctypes.byref(g), ctypes.byref(q), ctypes.byref(h)) == S.EINVAL, kw
    g1 = S.Grid(8, 8, 1, 0.1, 0.1, 0.1)                      # a stretched z needs nz > 1
    q = S.default_params(zc=[0.1], zf=[0.1])
    assert S.lib.stagger_create(ctypes.byref(g1), ctypes.byref(q), ctypes.byref(h)) == S.EINVAL
    # The allocation-free diagnostics cannot hold a mesh on the device.  The
    # rejection comes before any launch; where a GPU is present the state
    # still points at real device arrays of the grid's size, so that no
    # reordering of the checks could make a kernel read outside them.
    q = S.default_params(zc=good, zf=good)
    keep = None
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except ImportError:
        has_gpu = False
    if has_gpu:
        keep = [torch.zeros(6, 8, 8, device="cuda") for _ in range(8)]
        state = S._dev(keep)
    else:
        state = S.P8F(*[ctypes.cast(ctypes.c_void_p(16 * (i + 1)), ctypes.POINTER(ctypes.c_float))
                        for i in range(8)])
    out = (ctypes.c_double * 10)()
    assert S.lib.stagger_diagnostics_noalloc(ctypes.byref(g), ctypes.byref(q), state, out,
                                             None) == S.EUNSUPPORTED
    # Invalid grids and parameters take the same checks as stagger_create.
    for gg, qq in [(S.Grid(8, 8, 0, 0.1, 0.1, 0.1), S.default_params()),
                   (S.Grid(4, 65536, 1, 0.1, 0.1, 0.1), S.default_params()),
                   (g, S.default_params(gamma=1.0))]:
        assert S.lib.stagger_diagnostics_noalloc(ctypes.byref(gg), ctypes.byref(qq), state, out,
                                                 None) == S.EINVAL
    del keep


def test_null_context_calls_are_rejected(S):
    nul = S.P8F()
    assert S.lib.stagger_rhs(None, nul, nul, None) == S.EINVAL
    assert S.lib.stagger_step(None, nul, 0.1, None, None) == S.EINVAL
    assert S.lib.stagger_step_adjoint(None, nul, 0.1, nul, nul, None) == S.EINVAL
    assert S.lib.stagger_destroy(None) == S.OK
    assert S.lib.stagger_cells(None) == 0
    assert S.lib.stagger_strerror(S.ENONFINITE).decode() == "non-finite value in the state"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "stagger_copy", os.path.join(ROOT, "paper_2405_02483_gb300", "__init__.py"),
        submodule_search_locations=[])
    mod = importlib.util.module_from_spec(spec)
    monkeypatch.setattr(os.path, "exists", lambda p: False if p.endswith("libstagger.so") else True)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def _build_c_user(tmp_path):
    """Compile and link the plain C user of the library (tests/c_abi_step.c)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pkg = os.path.join(ROOT, "paper_2405_02483_gb300")
    exe = str(tmp_path / "c_abi_step")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_step.c"), "-o", exe, "-L", pkg, "-lstagger",
           "-Wl,-rpath," + pkg, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_plain_c_program_compiles_and_links(tmp_path):
    """The header is plain C99 and the library links without Python."""
    _build_c_user(tmp_path)


@pytest.mark.gpu
def test_plain_c_program_matches_the_binding(tmp_path):
    import subprocess
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    exe = _build_c_user(tmp_path)
    out = str(tmp_path / "state.bin")
    r = subprocess.run([exe, out], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.stdout, r.stderr)
    got = np.fromfile(out, dtype=np.float32).reshape(8, 16, 16, 16)
    # The same state and steps through the Python binding.
    n, tau = 16, 2 * np.pi
    x = ((np.arange(n) + 0.5) / n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = [0.02 * np.sin(tau * X) * np.cos(tau * Z), 0.1 * np.sin(tau * Y), 0.1 * np.sin(tau * Z),
         0.1 * np.sin(tau * X), 0.01 * np.cos(tau * Y), 0.05 * np.cos(tau * Z),
         0.05 * np.cos(tau * X), 0 * X]
    host = [torch.tensor(a.astype(np.float32)).contiguous() for a in f]
    ref = [1.0, 0, 0, 0, 0.9, 0, 0, 0.3]
    p = S.default_params(ref=ref, nu1=0.04, nu2=1.0, nu3=0.04, do_quench=1)
    sim = S.Sim((n, n, n), (1.0 / n,) * 3, p)
    sim.step_host(host, 2, 1e-3)
    sim.close()
    for c in range(8):
        assert np.array_equal(got[c], host[c].numpy()), c


def test_dt_entry_rejects_bad_arguments_without_gpu(S):
    nul = S.P8F()
    out = (ctypes.c_double * 4)()
    assert S.lib.stagger_dt(None, nul, ctypes.cast(out, ctypes.c_void_p), 0, None) == S.EINVAL


@pytest.mark.gpu
def test_dt_on_device_and_host_equal_courant():
    """stagger_dt with a device output (asynchronous, stream-ordered) and with
    a host output give the step and limits of stagger_courant bit for bit, and
    the device copy is the value of the call, not of a later one."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2405_02483_gb300 as S
    from test_gpu_parity import VISC_KW, make, ragged_state
    w = ragged_state((20, 12, 10))
    sim, refs, dev = make(S, w, VISC_KW)
    dt, lim = sim.courant(dev)
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    sim.dt(dev, out=out)
    sim.step(dev, None)                  # rewrites the library's own dt scratch
    got = out.cpu().tolist()
    assert got == [dt, *lim]
    dt2, lim2 = sim.dt(dev)
    dt3, lim3 = sim.courant(dev)
    assert (dt2, lim2) == (dt3, lim3) and dt2 != dt
    sim.close()


def test_wall_parameters_are_validated_without_gpu(S):
    h = ctypes.c_void_p()
    ok_nz = 2 * S.ZGHOST_MIN + 2
    cases = [(S.Grid(8, 8, ok_nz, 0.1, 0.1, 0.1), dict(zwalls=3, zghost=S.ZGHOST_MIN)),
             (S.Grid(8, 8, ok_nz, 0.1, 0.1, 0.1), dict(zwalls=2, zghost=S.ZGHOST_MIN - 1)),
             (S.Grid(8, 8, ok_nz - 1, 0.1, 0.1, 0.1), dict(zwalls=2, zghost=S.ZGHOST_MIN)),
             (S.Grid(8, 8, ok_nz, 0.1, 0.1, 0.1), dict(zwalls=2, zghost=S.ZGHOST_MIN, csmag=0.1)),
             # stellar-atmosphere boundaries
             (S.Grid(8, 8, 3 * S.ZGHOST_MIN + 2, 0.1, 0.1, 0.1),
              dict(zwalls=3, zghost=S.ZGHOST_MIN)),                      # no gravity
             (S.Grid(8, 8, 3 * S.ZGHOST_MIN + 1, 0.1, 0.1, 0.1),
              dict(zwalls=3, zghost=S.ZGHOST_MIN, g=(0, 0, -1.0))),      # too thin
             (S.Grid(8, 8, 3 * S.ZGHOST_MIN + 2, 0.1, 0.1, 0.1),
              dict(zwalls=3, zghost=S.ZGHOST_MIN, g=(0, 0, -1.0), bdry_t=0.0)),
             (S.Grid(8, 8, 3 * S.ZGHOST_MIN + 2, 0.1, 0.1, 0.1),
              dict(zwalls=3, zghost=S.ZGHOST_MIN, g=(0, 0, -1.0), top_rho_lo=1.5)),
             (S.Grid(8, 8, 3 * S.ZGHOST_MIN + 2, 0.1, 0.1, 0.1),
              dict(zwalls=3, zghost=S.ZGHOST_MIN, g=(0, 0, -1.0), fuse_flux_div=1)),
             (S.Grid(8, 8, 3 * S.ZGHOST_MIN + 2, 0.1, 0.1, 0.1),
              dict(zwalls=3, zghost=S.ZGHOST_MIN, g=(0, 0, -1.0), bdry_B=(float("nan"), 0, 0))),
             (S.Grid(8, 8, 3 * S.ZGHOST_MIN + 2, 0.1, 0.1, 0.1),
              dict(zwalls=3, zghost=S.ZGHOST_MIN, g=(0, 0, -1.0), top_tpot=-1.0)),
             (S.Grid(8, 8, ok_nz, 0.1, 0.1, 0.1), dict(zwalls=1, zghost=S.ZGHOST_MIN - 1)),
             (S.Grid(8, 8, ok_nz - 1, 0.1, 0.1, 0.1), dict(zwalls=1, zghost=S.ZGHOST_MIN)),
             (S.Grid(8, 8, ok_nz, 0.1, 0.1, 0.1), dict(zwalls=1, zghost=S.ZGHOST_MIN, csmag=0.1)),
             (S.Grid(8, 8, ok_nz, 0.1, 0.1, 0.1),
              dict(zwalls=1, zghost=S.ZGHOST_MIN, zc=[0.1] * ok_nz, zf=[0.1] * ok_nz)),
             (S.Grid(8, 8, ok_nz, 0.1, 0.1, 0.1),
              dict(zwalls=1, zghost=S.ZGHOST_MIN, ref=[1, 0, 0, 0, 1, 0.2, 0, 0.3]))]
    for g, kw in cases:
        q = S.default_params(**kw)
        assert S.lib.stagger_create(ctypes.byref(g), ctypes.byref(q), ctypes.byref(h)) == S.EINVAL, kw
