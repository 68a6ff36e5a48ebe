"""ctypes binding of the C ABI declared in include/pmg.h.

Argument marshalling only: every numerical step runs in the CUDA library.
Device vectors are torch CUDA tensors (fp64, contiguous); their data_ptr()
and the current torch stream are passed through.  Importing this module does
not load the library; the first call does, and raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpmg.so")

SMOOTHER = {"EA": 0, "FA": 1}
OVERLAP = {"0": 0, "l": 1, "lf": 2}
WEIGHTING = {"unweighted": 0, "arithmetic": 1, "cubic": 3, "quintic": 5}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_tc": 2, "mixed_tf32": 3}

STATUS = {0: "PMG_OK", -1: "PMG_EINVAL", -2: "PMG_ENOMEM", -3: "PMG_ECUDA", -4: "PMG_ENOCONV",
          -5: "PMG_EBREAKDOWN", -6: "PMG_ENAN", -7: "PMG_ETIMEOUT"}

EXPORTS = ["pmg_options_default", "pmg_grid_create", "pmg_grid_destroy", "pmg_grid_coords",
           "pmg_hierarchy_build", "pmg_hierarchy_destroy", "pmg_num_levels", "pmg_level_info",
           "pmg_apply", "pmg_residual", "pmg_rhs", "pmg_smooth", "pmg_restrict", "pmg_prolong",
           "pmg_coarse_solve", "pmg_vcycle", "pmg_solve", "pmg_solve_host", "pmg_status_string",
           "pmg_last_error", "pmg_schwarz_sweep", "pmg_kernel_launches", "pmg_coarse_solve_static",
           "pmg_schwarz_sweep_fma", "pmg_schwarz_sweep_native", "pmg_mlp_forward",
           "pmg_mlp_backward", "pmg_mlp_adam", "pmg_batch_create", "pmg_batch_solve",
           "pmg_batch_destroy", "pmg_batch_last_error", "pmg_hierarchy_autotune", "pmg_tuned_threads",
           "pmg_tc_timeouts", "pmg_device_status", "pmg_test_stall_tc_waits",
           "pmg_fma_probe"]


class PmgOptions(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("overlap", ctypes.c_int), ("weighting", ctypes.c_int),
                ("ns_pre", ctypes.c_int), ("ns_post", ctypes.c_int), ("variable_v", ctypes.c_int),
                ("omega", ctypes.c_double), ("precision", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("omega_level", ctypes.c_double * 8), ("tau_level", ctypes.c_double * 8),
                ("preconditioner", ctypes.c_int), ("outer_apply", ctypes.c_int), ("nrhs", ctypes.c_int)]


class PmgStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("r0", ctypes.c_double), ("rn", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("status", ctypes.c_int),
                ("device_loop", ctypes.c_int)]


class PmgError(RuntimeError):
    def __init__(self, fn, status, detail=""):
        self.status = status
        super().__init__(f"{fn} -> {STATUS.get(status, status)}"
                         + (f": {detail}" if detail else ""))


_lib = None


def load(path: str | None = None):
    """Load libpmg.so (built by paper_1603_02524_gb300.build); raise if missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "pmg_options_default": (None, [ctypes.POINTER(PmgOptions)]),
        "pmg_grid_create": (i, [i, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p),
                                i, d, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(vp)]),
        "pmg_grid_destroy": (None, [vp]),
        "pmg_grid_coords": (i, [vp, i, ctypes.POINTER(ctypes.c_double)]),
        "pmg_hierarchy_build": (i, [vp, ctypes.POINTER(PmgOptions), ctypes.POINTER(vp)]),
        "pmg_hierarchy_destroy": (None, [vp]),
        "pmg_num_levels": (i, [vp]),
        "pmg_level_info": (i, [vp, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]),
        "pmg_apply": (i, [vp, i, vp, vp, vp]),
        "pmg_residual": (i, [vp, i, vp, vp, vp, vp]),
        "pmg_rhs": (i, [vp, vp, vp, vp]),
        "pmg_smooth": (i, [vp, i, vp, vp, i, vp]),
        "pmg_restrict": (i, [vp, i, vp, vp, vp]),
        "pmg_prolong": (i, [vp, i, vp, vp, vp]),
        "pmg_coarse_solve": (i, [vp, vp, vp, vp]),
        "pmg_vcycle": (i, [vp, vp, vp, vp]),
        "pmg_solve": (i, [vp, vp, vp, d, vp, vp]),
        "pmg_solve_host": (i, [vp, vp, vp, d, vp, vp]),
        "pmg_status_string": (ctypes.c_char_p, [i]),
        "pmg_last_error": (ctypes.c_char_p, [vp]),
        "pmg_schwarz_sweep": (i, [vp, i, i, vp, vp, vp]),
        "pmg_kernel_launches": (ctypes.c_ulonglong, []),
        "pmg_tc_timeouts": (i, [ctypes.POINTER(ctypes.c_uint)]),
        "pmg_device_status": (i, [vp, vp, ctypes.POINTER(ctypes.c_int)]),
        "pmg_test_stall_tc_waits": (i, [vp, ctypes.c_uint]),
        "pmg_fma_probe": (i, [i, i, vp, ctypes.POINTER(ctypes.c_double)]),
        "pmg_coarse_solve_static": (i, [vp, vp, vp, vp]),
        "pmg_schwarz_sweep_fma": (i, [vp, i, i, ctypes.POINTER(ctypes.c_double)]),
        "pmg_schwarz_sweep_native": (i, [vp, i, i, vp]),
        "pmg_mlp_forward": (i, [vp, vp, i, vp, vp, vp, vp]),
        "pmg_mlp_backward": (i, [vp, vp, vp, vp, vp, vp, vp, i, vp, vp, vp, vp]),
        "pmg_mlp_adam": (i, [vp, vp, vp, vp, i, i, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, vp]),
        "pmg_batch_create": (i, [i, vp, vp, vp, d, vp]),
        "pmg_batch_solve": (i, [vp, ctypes.POINTER(PmgStats), vp]),
        "pmg_batch_destroy": (None, [vp]),
        "pmg_batch_last_error": (ctypes.c_char_p, [vp]),
        "pmg_hierarchy_autotune": (i, [vp, vp]),
        "pmg_tuned_threads": (i, [vp, i, i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def options(smoother="EA", overlap="l", weighting="quintic", ns=(1, 1), variable_v=False,
            omega=1.0, precision="fp64", max_iter=100, omega_level=None, tau_level=None,
            preconditioner="vcycle", outer_apply="fp64", nrhs=1) -> PmgOptions:
    """omega_level / tau_level: optional per-level sequences (index = level, 0 = default);
    preconditioner "vcycle" (Algorithm 2) or "none" (plain CG); outer_apply "fp64" or "df"
    (the CG's operator apply in double-float on the FP32 pipes)."""
    o = PmgOptions()
    load().pmg_options_default(ctypes.byref(o))
    o.smoother = SMOOTHER[smoother]
    o.overlap = OVERLAP[overlap]
    o.weighting = WEIGHTING[weighting]
    o.ns_pre, o.ns_post = int(ns[0]), int(ns[1])
    o.variable_v = int(bool(variable_v))
    o.omega = float(omega)
    o.precision = PRECISION[precision]
    o.max_iter = int(max_iter)
    for l, v in enumerate(omega_level or []):
        o.omega_level[l] = float(v)
    for l, v in enumerate(tau_level or []):
        o.tau_level[l] = float(v)
    o.preconditioner = {"vcycle": 0, "none": 1}[preconditioner]
    o.outer_apply = {"fp64": 0, "df": 1}[outer_apply]
    o.nrhs = int(nrhs)
    return o


def tc_timeouts() -> int:
    """Blocks of the tcgen05 patch kernel that gave up waiting for their MMAs
    since the last call (reset by the call; synchronises the device)."""
    n = ctypes.c_uint(0)
    _check("pmg_tc_timeouts", load().pmg_tc_timeouts(ctypes.byref(n)))
    return int(n.value)


def _check(fn, st, hier=None):
    if st != 0:
        detail = ""
        if hier:
            detail = (load().pmg_last_error(hier) or b"").decode()
        raise PmgError(fn, st, detail)


class Grid:
    """pmg_grid_create / pmg_grid_destroy / pmg_grid_coords."""

    def __init__(self, dim, P, n_elem, spacing, periodic, mu_star=1.0, beta=0.0):
        lib = load()
        self.dim, self.P = dim, P
        self.n_elem = tuple(int(x) for x in n_elem) + (1,) * (3 - len(n_elem))
        ne = (ctypes.c_int * 3)(*self.n_elem)
        self._sp = [(ctypes.c_double * len(s))(*s) for s in spacing]
        sp = (ctypes.c_void_p * 3)(*([ctypes.cast(a, ctypes.c_void_p) for a in self._sp]
                                     + [None] * (3 - len(self._sp))))
        b = beta if isinstance(beta, (list, tuple)) else [beta] * 3
        bt = (ctypes.c_double * 3)(*(list(b) + [0.0] * (3 - len(b))))
        h = ctypes.c_void_p()
        _check("pmg_grid_create", lib.pmg_grid_create(dim, P, ne, sp, int(bool(periodic)),
                                                       float(mu_star), bt, ctypes.byref(h)))
        self.handle = h

    def coords(self, axis):
        import numpy as np
        n = self.n_elem[axis] * (self.P + 1)
        out = (ctypes.c_double * n)()
        _check("pmg_grid_coords", load().pmg_grid_coords(self.handle, axis, out))
        return np.frombuffer(out, dtype=np.float64).reshape(self.n_elem[axis], self.P + 1).copy()

    def close(self):
        if self.handle:
            load().pmg_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, n):
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"expected a contiguous fp64 CUDA tensor with {n} entries")
    return _ptr(t)


class Hierarchy:
    """pmg_hierarchy_build and the per-level entry points (torch CUDA tensors in and out)."""

    def __init__(self, grid: Grid, **opts):
        lib = load()
        self.grid = grid
        self.opts = options(**opts)
        h = ctypes.c_void_p()
        _check("pmg_hierarchy_build", lib.pmg_hierarchy_build(grid.handle, ctypes.byref(self.opts),
                                                               ctypes.byref(h)))
        self.handle = h
        self.L = lib.pmg_num_levels(h) - 1

    def level_info(self, level):
        P = ctypes.c_int()
        n = ctypes.c_longlong()
        _check("pmg_level_info", load().pmg_level_info(self.handle, level, ctypes.byref(P), ctypes.byref(n)))
        return P.value, n.value

    def ndof(self, level=None):
        return self.level_info(self.L if level is None else level)[1]

    def apply(self, level, u, out, stream=None):
        n = self.ndof(level)
        _check("pmg_apply", load().pmg_apply(self.handle, level, _dev(u, n), _dev(out, n), _stream(stream)), self.handle)

    def residual(self, level, u, f, out, stream=None):
        n = self.ndof(level)
        _check("pmg_residual", load().pmg_residual(self.handle, level, _dev(u, n), _dev(f, n), _dev(out, n),
                                                   _stream(stream)), self.handle)

    def rhs(self, f, out, stream=None):
        n = self.ndof()
        _check("pmg_rhs", load().pmg_rhs(self.handle, _dev(f, n), _dev(out, n), _stream(stream)), self.handle)

    def smooth(self, level, u, f, nsteps=1, stream=None):
        n = self.ndof(level)
        _check("pmg_smooth", load().pmg_smooth(self.handle, level, _dev(u, n), _dev(f, n), nsteps,
                                               _stream(stream)), self.handle)

    def restrict(self, level, rf, fc, stream=None):
        _check("pmg_restrict", load().pmg_restrict(self.handle, level, _dev(rf, self.ndof(level)),
                                                   _dev(fc, self.ndof(level - 1)), _stream(stream)), self.handle)

    def prolong(self, level, uc, uf, stream=None):
        _check("pmg_prolong", load().pmg_prolong(self.handle, level, _dev(uc, self.ndof(level - 1)),
                                                 _dev(uf, self.ndof(level)), _stream(stream)), self.handle)

    def coarse_solve(self, f0, u0, stream=None):
        n = self.ndof(0)
        _check("pmg_coarse_solve", load().pmg_coarse_solve(self.handle, _dev(f0, n), _dev(u0, n),
                                                           _stream(stream)), self.handle)

    def schwarz_sweep_fma(self, level, family):
        out = ctypes.c_double()
        _check("pmg_schwarz_sweep_fma", load().pmg_schwarz_sweep_fma(self.handle, level, family, ctypes.byref(out)))
        return out.value

    def schwarz_sweep(self, level, family, r, u, stream=None):
        n = self.ndof(level)
        _check("pmg_schwarz_sweep", load().pmg_schwarz_sweep(self.handle, level, family, _dev(r, n), _dev(u, n),
                                                             _stream(stream)), self.handle)

    def vcycle(self, f, u, stream=None):
        n = self.ndof()
        _check("pmg_vcycle", load().pmg_vcycle(self.handle, _dev(f, n), _dev(u, n), _stream(stream)), self.handle)

    def solve(self, g, u, rtol=1e-10, stream=None, history=True, check=True):
        """Algorithm 2 on device tensors; returns (status, iterations, residual history).
        A hierarchy with nrhs > 1 (g, u: nrhs vectors back to back) returns
        (status, [iterations per right-hand side], [history per right-hand side])."""
        n = self.ndof()
        k = self.opts.nrhs
        st = (PmgStats * k)()
        hists = []
        for i in range(k):
            hist = (ctypes.c_double * (self.opts.max_iter + 1))() if history else None
            hists.append(hist)
            st[i].history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if history else None
        rc = load().pmg_solve(self.handle, _dev(g, n), _dev(u, n), float(rtol), st, _stream(stream))
        if check and rc not in (0, -4):
            _check("pmg_solve", rc, self.handle)
        self.last_device_loop = bool(st[0].device_loop)
        self.last_stats = [(st[i].status, st[i].iterations, st[i].r0, st[i].rn) for i in range(k)]
        hs = [list(hists[i][: st[i].iterations + 1]) if history else [] for i in range(k)]
        if k == 1:
            return rc, st[0].iterations, hs[0]
        return rc, [st[i].iterations for i in range(k)], hs

    def solve_host(self, g_host, u_host, rtol=1e-10, stream=None):
        """Algorithm 2 on host arrays (numpy or pinned torch CPU tensors, fp64, contiguous)."""
        import numpy as np
        n = self.ndof()

        def hp(a):
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == n
                return ctypes.c_void_p(a.ctypes.data)
            assert a.numel() == n and a.is_contiguous() and not a.is_cuda
            return ctypes.c_void_p(a.data_ptr())
        st = (PmgStats * self.opts.nrhs)()
        rc = load().pmg_solve_host(self.handle, hp(g_host), hp(u_host), float(rtol), st, _stream(stream))
        if rc not in (0, -4):
            _check("pmg_solve_host", rc, self.handle)
        return rc, st[0].iterations

    def device_status(self, stream=None):
        """Read and reset the hierarchy's device status word (pmg_device_status)."""
        v = ctypes.c_int(0)
        _check("pmg_device_status", load().pmg_device_status(self.handle, _stream(stream), ctypes.byref(v)),
               self.handle)
        return v.value

    def test_stall_tc_waits(self, limit_us):
        """Test hook: make the tcgen05 patch kernel's bounded waits run out (pmg_test_stall_tc_waits)."""
        _check("pmg_test_stall_tc_waits", load().pmg_test_stall_tc_waits(self.handle, int(limit_us)),
               self.handle)

    def autotune(self, stream=None):
        """Pick the patch kernel's CTA size per level by timing (pmg_hierarchy_autotune)."""
        _check("pmg_hierarchy_autotune", load().pmg_hierarchy_autotune(self.handle, _stream(stream)),
               self.handle)

    def tuned_threads(self, level, family=-1):
        st = load().pmg_tuned_threads(self.handle, level, family)
        if st < 0:
            _check("pmg_tuned_threads", st, self.handle)
        return st

    def close(self):
        if getattr(self, "handle", None):
            load().pmg_hierarchy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """pmg_batch_create / pmg_batch_solve / pmg_batch_destroy: independent MGCG solves
    (one per distinct hierarchy, with its own g and u device tensors) recorded as one
    CUDA graph and run with one launch."""

    def __init__(self, hiers, gs, us, rtol=1e-10):
        lib = load()
        n = len(hiers)
        if not (n == len(gs) == len(us)) or n == 0:
            raise ValueError("hiers, gs and us must have the same non-zero length")
        self._keep = (list(hiers), list(gs), list(us))
        hs = (ctypes.c_void_p * n)(*[h.handle.value for h in hiers])
        gp = (ctypes.c_void_p * n)(*[_dev(g, h.ndof()).value for g, h in zip(gs, hiers)])
        up = (ctypes.c_void_p * n)(*[_dev(u, h.ndof()).value for u, h in zip(us, hiers)])
        b = ctypes.c_void_p()
        _check("pmg_batch_create", lib.pmg_batch_create(n, hs, gp, up, float(rtol), ctypes.byref(b)))
        self.handle = b
        self.count = n
        self.max_iter = [h.opts.max_iter for h in hiers]
        self.nrhs = [h.opts.nrhs for h in hiers]

    def solve(self, stream=None, history=False, check=True):
        """Run every solve; returns (status, [(status, iterations, r0, rn[, history]) ...]) with
        one entry per right-hand side, solve by solve."""
        total = sum(self.nrhs)
        mx = [m for m, k in zip(self.max_iter, self.nrhs) for _ in range(k)]
        st = (PmgStats * total)()
        hists = []
        for i in range(total):
            if history:
                hist = (ctypes.c_double * (mx[i] + 1))()
                hists.append(hist)
                st[i].history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
            else:
                st[i].history = None
        rc = load().pmg_batch_solve(self.handle, st, _stream(stream))
        if check and rc not in (0, -4):
            detail = (load().pmg_batch_last_error(self.handle) or b"").decode()
            raise PmgError("pmg_batch_solve", rc, detail)
        out = []
        for i in range(total):
            item = (st[i].status, st[i].iterations, st[i].r0, st[i].rn)
            if history:
                item = item + (list(hists[i][: st[i].iterations + 1]),)
            out.append(item)
        return rc, out

    def close(self):
        if getattr(self, "handle", None):
            load().pmg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
