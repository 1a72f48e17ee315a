"""Python binding of libstagger (include/stagger.h): the staggered-mesh MHD
right-hand side and low-storage RK3 step of the Stagger Code on sm_103a.

This module only marshals arguments: every step of the method runs in the
library's CUDA kernels.  Device arrays are torch CUDA tensors (torch is used
for device memory and streams only).  If libstagger.so has not been built,
importing the binding raises ImportError; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# STAGGER_LIB selects another build of the library (e.g. an A/B variant).
LIB_PATH = os.environ.get("STAGGER_LIB") or os.path.join(PKG, "libstagger.so")

OK, EINVAL, ECUDA, ENONFINITE, EOOM, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
FIELDS = ("r", "px", "py", "pz", "E", "Bx", "By", "Bz")


class StaggerError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, _strerror(status), status))


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double),
                ("nu1", ctypes.c_double), ("nu2", ctypes.c_double), ("nu3", ctypes.c_double),
                ("nu_const", ctypes.c_double), ("nuE", ctypes.c_double),
                ("nuB", ctypes.c_double), ("c1", ctypes.c_double),
                ("do_quench", ctypes.c_int), ("qmax", ctypes.c_double),
                ("qlim", ctypes.c_double), ("log_interp", ctypes.c_int),
                ("Cdt", ctypes.c_double), ("Cdtr", ctypes.c_double), ("Cdtd", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("ref", ctypes.c_double * 8),
                ("t_cool", ctypes.c_double), ("e_cool", ctypes.c_double),
                ("rho_cool", ctypes.c_double), ("cool_cut", ctypes.c_int),
                ("csmag", ctypes.c_double), ("scalar_cells", ctypes.c_int),
                ("do_2nddiv", ctypes.c_int), ("d2lnr_lim", ctypes.c_double),
                ("zc", ctypes.POINTER(ctypes.c_double)), ("zf", ctypes.POINTER(ctypes.c_double)),
                ("t_chromo", ctypes.c_double), ("rho_bot", ctypes.c_double),
                ("cor_L0", ctypes.c_double), ("cor_Tunit", ctypes.c_double),
                ("fuse_flux_div", ctypes.c_int),
                ("quench_max3", ctypes.c_int), ("quench_eps", ctypes.c_double),
                ("zwalls", ctypes.c_int), ("zghost", ctypes.c_int),
                ("ediffav", ctypes.c_int),
                ("lnp_aver", ctypes.c_int),
                ("bdry_t", ctypes.c_double), ("bdry_rho", ctypes.c_double),
                ("bdry_E", ctypes.c_double), ("bdry_u", ctypes.c_double),
                ("bdry_B", ctypes.c_double * 3),
                ("top_rho_lo", ctypes.c_double), ("top_rho_hi", ctypes.c_double),
                ("top_e_fac", ctypes.c_double), ("top_umax", ctypes.c_double),
                ("top_tpot", ctypes.c_double)]

ZGHOST_MIN = 14   # STAGGER_ZGHOST_MIN of include/stagger.h


P8F = ctypes.POINTER(ctypes.c_float) * 8
P8D = ctypes.POINTER(ctypes.c_double) * 8
VP = ctypes.c_void_p

# (name, restype, argtypes) of every exported function.
SIGNATURES = [
    ("stagger_params_default", ctypes.c_int, [ctypes.POINTER(Params)]),
    ("stagger_create", ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Params), ctypes.POINTER(VP)]),
    ("stagger_destroy", ctypes.c_int, [VP]),
    ("stagger_rhs", ctypes.c_int, [VP, P8F, P8F, VP]),
    ("stagger_step", ctypes.c_int, [VP, P8F, ctypes.c_double, ctypes.POINTER(ctypes.c_double), VP]),
    ("stagger_run", ctypes.c_int, [VP, P8F, ctypes.c_int, ctypes.c_double, VP]),
    ("stagger_courant", ctypes.c_int, [VP, P8F, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), VP]),
    ("stagger_dt", ctypes.c_int, [VP, P8F, ctypes.c_void_p, ctypes.c_int, VP]),
    ("stagger_diagnostics", ctypes.c_int, [VP, P8F, ctypes.POINTER(ctypes.c_double), VP]),
    ("stagger_step_adjoint", ctypes.c_int, [VP, P8F, ctypes.c_double, P8F, P8F, VP]),
    ("stagger_rhs_unfused", ctypes.c_int, [VP, P8F, P8F, VP]),
    ("stagger_rhs_unfused_f64", ctypes.c_int, [VP, P8D, P8D, VP]),
    ("stagger_step_unfused_f64", ctypes.c_int, [VP, P8D, ctypes.c_double, VP]),
    ("stagger_step_adjoint_f64", ctypes.c_int, [VP, P8D, ctypes.c_double, P8D, P8D, VP]),
    ("stagger_step_host", ctypes.c_int, [VP, P8F, ctypes.c_int, ctypes.c_double, VP]),
    ("stagger_timing", ctypes.c_int, [VP, ctypes.c_int]),
    ("stagger_kernel_times", ctypes.c_int, [VP, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_longlong), VP]),
    ("stagger_diagnostics_noalloc", ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Params),
                                                   P8F, ctypes.POINTER(ctypes.c_double), VP]),
    ("stagger_cells", ctypes.c_size_t, [VP]),
    ("stagger_launch_count", ctypes.c_longlong, [VP]),
    ("stagger_strerror", ctypes.c_char_p, [ctypes.c_int]),
]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libstagger.so is not built (expected at %s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` or "
                          "`python -m paper_2405_02483_gb300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _strerror(status):
    return lib.stagger_strerror(status).decode()


def _check(status, where):
    if status != OK:
        raise StaggerError(status, where)


def default_params(**kw) -> Params:
    p = Params()
    _check(lib.stagger_params_default(ctypes.byref(p)), "stagger_params_default")
    for k, v in kw.items():
        if k == "g":
            p.g = (ctypes.c_double * 3)(*v)
        elif k == "ref":
            p.ref = (ctypes.c_double * 8)(*v)
        elif k == "bdry_B":
            p.bdry_B = (ctypes.c_double * 3)(*v)
        elif k in ("zc", "zf"):
            # Stretched z mesh: dz/dk at centres / lower faces (nz values each);
            # the array lives as long as the Params object.
            arr = (ctypes.c_double * len(v))(*[float(x) for x in v])
            setattr(p, k, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)))
            setattr(p, "_" + k, arr)
        else:
            setattr(p, k, v)
    return p


def _ptrs(tensors, kind, dtype_name):
    import torch
    want = torch.float32 if kind is P8F else torch.float64
    if len(tensors) != 8:
        raise ValueError("expected 8 field arrays")
    for t in tensors:
        if t.dtype != want or not t.is_contiguous():
            raise ValueError("fields must be contiguous %s tensors" % dtype_name)
    ct = ctypes.POINTER(ctypes.c_float) if kind is P8F else ctypes.POINTER(ctypes.c_double)
    return kind(*[ctypes.cast(t.data_ptr(), ct) for t in tensors])


def _dev(tensors, kind=P8F):
    for t in tensors:
        if not t.is_cuda:
            raise ValueError("device arrays must be CUDA tensors")
    return _ptrs(tensors, kind, "float32" if kind is P8F else "float64")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Sim:
    """One context: a grid, its physics parameters and the device scratch."""

    def __init__(self, shape, spacing, params: Params | None = None, **kw):
        nx, ny, nz = shape
        self.shape = (nx, ny, nz)
        self.grid = Grid(nx, ny, nz, *spacing)
        self.params = params if params is not None else default_params(**kw)
        h = ctypes.c_void_p()
        _check(lib.stagger_create(ctypes.byref(self.grid), ctypes.byref(self.params),
                                  ctypes.byref(h)), "stagger_create")
        self.ctx = h

    def close(self):
        if self.ctx:
            _check(lib.stagger_destroy(self.ctx), "stagger_destroy")
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def refs(self):
        return [self.params.ref[k] for k in range(8)]

    def empty(self, dtype=None):
        import torch
        nx, ny, nz = self.shape
        return [torch.empty((nz, ny, nx), dtype=dtype or torch.float32, device="cuda")
                for _ in range(8)]

    def rhs(self, state, out=None, stream=None):
        out = out if out is not None else self.empty()
        _check(lib.stagger_rhs(self.ctx, _dev(state), _dev(out), _stream(stream)), "stagger_rhs")
        return out

    def step(self, state, dt=None, want_dt=False, stream=None):
        d = ctypes.c_double(0.0)
        _check(lib.stagger_step(self.ctx, _dev(state), float(dt or 0.0),
                                ctypes.byref(d) if want_dt else None, _stream(stream)),
               "stagger_step")
        return d.value if want_dt else None

    def run(self, state, nsteps, dt=None, stream=None):
        _check(lib.stagger_run(self.ctx, _dev(state), int(nsteps), float(dt or 0.0),
                               _stream(stream)), "stagger_run")

    def courant(self, state, stream=None):
        dt = ctypes.c_double()
        lim = (ctypes.c_double * 3)()
        _check(lib.stagger_courant(self.ctx, _dev(state), ctypes.byref(dt), lim, _stream(stream)),
               "stagger_courant")
        return dt.value, tuple(lim)

    def dt(self, state, out=None, stream=None):
        """Courant step and its three limits.  With out (a CUDA float64 tensor
        of 4 values) the result is written there on the stream, asynchronously;
        without, the call synchronises and returns (dt, (wave, rate, diffusion))."""
        if out is not None:
            import torch
            if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 4):
                raise ValueError("out must be a CUDA float64 tensor of at least 4 values")
            _check(lib.stagger_dt(self.ctx, _dev(state), ctypes.c_void_p(out.data_ptr()), 1,
                                  _stream(stream)), "stagger_dt")
            return out
        h = (ctypes.c_double * 4)()
        _check(lib.stagger_dt(self.ctx, _dev(state), ctypes.cast(h, ctypes.c_void_p), 0,
                              _stream(stream)), "stagger_dt")
        return h[0], (h[1], h[2], h[3])

    def diagnostics(self, state, stream=None, check=True):
        out = (ctypes.c_double * 10)()
        st = lib.stagger_diagnostics(self.ctx, _dev(state), out, _stream(stream))
        if check or st not in (OK, ENONFINITE):
            _check(st, "stagger_diagnostics")
        return list(out)

    def step_adjoint(self, state_n, dt, lam, out=None, stream=None):
        out = out if out is not None else self.empty()
        _check(lib.stagger_step_adjoint(self.ctx, _dev(state_n), float(dt), _dev(lam), _dev(out),
                                        _stream(stream)), "stagger_step_adjoint")
        return out

    def rhs_unfused(self, state, out=None, stream=None):
        out = out if out is not None else self.empty()
        _check(lib.stagger_rhs_unfused(self.ctx, _dev(state), _dev(out), _stream(stream)),
               "stagger_rhs_unfused")
        return out

    def rhs_unfused_f64(self, state, out=None, stream=None):
        import torch
        out = out if out is not None else self.empty(torch.float64)
        _check(lib.stagger_rhs_unfused_f64(self.ctx, _dev(state, P8D), _dev(out, P8D),
                                           _stream(stream)), "stagger_rhs_unfused_f64")
        return out

    def step_unfused_f64(self, state, dt, stream=None):
        _check(lib.stagger_step_unfused_f64(self.ctx, _dev(state, P8D), float(dt), _stream(stream)),
               "stagger_step_unfused_f64")

    def step_adjoint_f64(self, state_n, dt, lam, out=None, stream=None):
        import torch
        out = out if out is not None else self.empty(torch.float64)
        _check(lib.stagger_step_adjoint_f64(self.ctx, _dev(state_n, P8D), float(dt),
                                            _dev(lam, P8D), _dev(out, P8D), _stream(stream)),
               "stagger_step_adjoint_f64")
        return out

    def step_host(self, host_state, nsteps=1, dt=None, stream=None):
        """host_state: 8 contiguous float32 CPU tensors (pinned recommended)."""
        for t in host_state:
            if t.is_cuda:
                raise ValueError("step_host takes host arrays")
        _check(lib.stagger_step_host(self.ctx, _ptrs(host_state, P8F, "float32"), int(nsteps),
                                     float(dt or 0.0), _stream(stream)), "stagger_step_host")

    def timing(self, on=True):
        _check(lib.stagger_timing(self.ctx, 1 if on else 0), "stagger_timing")

    def kernel_times(self, stream=None):
        """{kernel name: (total ms, launches)} of the timed launches."""
        m = 32
        names = (ctypes.c_char_p * m)()
        ms = (ctypes.c_double * m)()
        cnt = (ctypes.c_longlong * m)()
        k = lib.stagger_kernel_times(self.ctx, m, names, ms, cnt, _stream(stream))
        if k < 0:
            _check(k, "stagger_kernel_times")
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(k) if cnt[i] > 0}

    def cells(self):
        return int(lib.stagger_cells(self.ctx))

    def launches(self):
        return int(lib.stagger_launch_count(self.ctx))


def split_state(fields64, refs=None):
    """Full FP64 fields (numpy or torch, shape (nz, ny, nx)) -> (refs, FP32
    CUDA deviations).  refs default to the per-field mean of r, E and each B
    component (zero for the momenta)."""
    import numpy as np
    import torch
    arrs = [np.asarray(f, dtype=np.float64) for f in fields64]
    if refs is None:
        refs = [float(arrs[0].mean()), 0.0, 0.0, 0.0, float(arrs[4].mean()),
                float(arrs[5].mean()), float(arrs[6].mean()), float(arrs[7].mean())]
    dev = [torch.from_numpy(np.ascontiguousarray(a - r)).to(torch.float32).cuda()
           for a, r in zip(arrs, refs)]
    return list(refs), dev


def join_state(dev, refs):
    """FP32 deviations -> full FP64 numpy fields."""
    return [t.double().cpu().numpy() + r for t, r in zip(dev, refs)]


from .rollout import StaggerRollout  # noqa: E402,F401
