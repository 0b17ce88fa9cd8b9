"""Thin Python binding of the C ABI in include/tmg.h (argument marshalling only).

Every step of the solve runs in the CUDA library ``libtmg.so``; PyTorch only
supplies device memory and the stream.  There is no CPU path: importing this
module on a machine without the built library raises at first use.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build_ext

TMG_OK, TMG_EINVAL, TMG_ENOMEM, TMG_ECUDA, TMG_ENOTCONV, TMG_ENUMERIC, TMG_ETIMEOUT, TMG_EUNSUPPORTED = range(8)
FP64, MIXED = 0, 1
SCHED_AUTO, SCHED_GRID, SCHED_CTA = 0, 1, 2
_PREC = {"fp64": FP64, "mixed": MIXED, FP64: FP64, MIXED: MIXED}


class TmgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().tmg_strerror(status).decode()
        if status == TMG_ECUDA:
            msg += f" (cudaError {_lib().tmg_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")


class _Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_cycles", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("gamma", ctypes.c_int), ("precision", ctypes.c_int),
                ("n_min", ctypes.c_int64), ("use_graph", ctypes.c_int), ("initial_guess", ctypes.c_int),
                ("tail_cap", ctypes.c_int64), ("use_pdl", ctypes.c_int), ("update_residual", ctypes.c_int),
                ("fuse_levels", ctypes.c_int), ("schedule", ctypes.c_int), ("check_fp64", ctypes.c_int)]


_LIB = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)

EXPORTS = ["tmg_opts_default", "tmg_setup", "tmg_solve", "tmg_solve_host", "tmg_solve_direct", "tmg_adjoint", "tmg_cycle",
           "tmg_cycle_down", "tmg_cycle_up", "tmg_residual",
           "tmg_stats", "tmg_error_vs_fp64", "tmg_plan_shape", "tmg_level_constants", "tmg_transfer_matrices", "tmg_plan_info",
           "tmg_plan_launches", "tmg_profile_cycle", "tmg_inspect", "tmg_residual_norm_noalloc", "tmg_destroy", "tmg_strerror",
           "tmg_last_cuda_error", "tmg_setup_batched", "tmg_solve_batched", "tmg_adjoint_batched",
           "tmg_stats_batched", "tmg_error_vs_fp64_batched", "tmg_batch_info", "tmg_batch_group_info", "tmg_batch_tune_info", "tmg_destroy_batched",
           "tmg_heat_setup", "tmg_heat_solve", "tmg_heat_cycle", "tmg_heat_residual", "tmg_heat_stats",
           "tmg_heat_info", "tmg_heat_profile", "tmg_heat_destroy", "tmg_debug_bounds"]


def library_path() -> str:
    """The library in use: the debug build with bounds checks when the
    environment sets TMG_BOUNDS=1, else the normal build."""
    return build_ext.LIB_BOUNDS if os.environ.get("TMG_BOUNDS") == "1" else build_ext.LIB


def _lib():
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libtmg.so not built ({path}); run __graft_entry__.build() "
                              "or python -m paper_1409_5254_gb300.build_ext")
        L = ctypes.CDLL(path)
        L.tmg_opts_default.argtypes = [ctypes.POINTER(_Opts)]
        L.tmg_opts_default.restype = None
        L.tmg_setup.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_Opts), _vp]
        L.tmg_solve.argtypes = [_vp, _vp, ctypes.c_double, _vp]
        L.tmg_solve_host.argtypes = [_vp, _vp, ctypes.c_double, _vp]
        L.tmg_cycle.argtypes = [_vp, _vp, ctypes.c_double, _vp]
        L.tmg_cycle_down.argtypes = [_vp, _vp, ctypes.c_double, _vp, _vp]
        L.tmg_cycle_up.argtypes = [_vp, _vp, _vp]
        L.tmg_cycle_down.restype = ctypes.c_int
        L.tmg_cycle_up.restype = ctypes.c_int
        L.tmg_solve_direct.argtypes = [_vp, _vp, ctypes.c_double, _vp]
        L.tmg_adjoint.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.tmg_residual.argtypes = [_vp, _vp, ctypes.c_double, _vp, _vp]
        L.tmg_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), _dp, _dp, _dp, ctypes.c_int]
        L.tmg_plan_shape.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_double, ctypes.POINTER(_Opts), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int)]
        L.tmg_level_constants.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _dp,
                                          _dp]
        L.tmg_transfer_matrices.argtypes = [ctypes.c_int, _dp, _dp]
        L.tmg_plan_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int64), _dp, ctypes.c_int]
        L.tmg_inspect.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t]
        L.tmg_plan_launches.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
        L.tmg_profile_cycle.argtypes = [_vp, _vp, ctypes.c_double, _vp, ctypes.c_int, _dp, ctypes.c_int]
        L.tmg_residual_norm_noalloc.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                                _vp, ctypes.c_double, _vp, _vp, _vp, _vp]
        L.tmg_residual_norm_noalloc.restype = ctypes.c_int
        L.tmg_destroy.argtypes = [_vp]
        L.tmg_destroy.restype = None
        _ip, _lp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)
        L.tmg_setup_batched.argtypes = [ctypes.POINTER(_vp), ctypes.c_int64, _ip, _dp, _dp, _lp, ctypes.c_double,
                                        ctypes.POINTER(_Opts), _vp]
        L.tmg_solve_batched.argtypes = [_vp, _vp, _vp, _vp]
        L.tmg_adjoint_batched.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.tmg_stats_batched.argtypes = [_vp, _ip, _dp, _dp, _ip]
        L.tmg_error_vs_fp64_batched.argtypes = [_vp, _vp, _vp, _vp, _dp]
        L.tmg_error_vs_fp64_batched.restype = ctypes.c_int
        L.tmg_error_vs_fp64.argtypes = [_vp, _vp, ctypes.c_double, _vp, _dp]
        L.tmg_error_vs_fp64.restype = ctypes.c_int
        L.tmg_batch_info.argtypes = [_vp, _ip, _lp]
        L.tmg_batch_group_info.argtypes = [_vp, ctypes.c_int, _ip, _lp, _lp, _ip, _dp, _dp]
        L.tmg_batch_tune_info.argtypes = [_vp, _dp, _dp]
        L.tmg_destroy_batched.argtypes = [_vp]
        L.tmg_destroy_batched.restype = None
        for name in ("tmg_setup_batched", "tmg_solve_batched", "tmg_adjoint_batched", "tmg_stats_batched",
                     "tmg_batch_info", "tmg_batch_group_info", "tmg_batch_tune_info"):
            getattr(L, name).restype = ctypes.c_int
        L.tmg_heat_setup.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int64, ctypes.POINTER(_Opts), ctypes.c_int, _vp]
        L.tmg_heat_solve.argtypes = [_vp, _vp, _vp, _vp]
        L.tmg_heat_cycle.argtypes = [_vp, _vp, _vp, _vp]
        L.tmg_heat_residual.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.tmg_heat_stats.argtypes = [_vp, _ip, _dp, _dp, ctypes.c_int]
        L.tmg_heat_info.argtypes = [_vp, _ip, _ip, _ip, ctypes.POINTER(ctypes.c_size_t)]
        L.tmg_heat_profile.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _dp, ctypes.c_int]
        for name in ("tmg_heat_setup", "tmg_heat_solve", "tmg_heat_cycle", "tmg_heat_residual", "tmg_heat_stats",
                     "tmg_heat_info", "tmg_heat_profile"):
            getattr(L, name).restype = ctypes.c_int
        L.tmg_heat_destroy.argtypes = [_vp]
        L.tmg_heat_destroy.restype = None
        L.tmg_debug_bounds.argtypes = [ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_ulonglong)]
        L.tmg_debug_bounds.restype = ctypes.c_int
        L.tmg_strerror.argtypes = [ctypes.c_int]
        L.tmg_strerror.restype = ctypes.c_char_p
        L.tmg_last_cuda_error.argtypes = []
        for name in ("tmg_setup", "tmg_solve", "tmg_solve_host", "tmg_solve_direct", "tmg_adjoint", "tmg_cycle", "tmg_residual", "tmg_stats",
                     "tmg_plan_shape", "tmg_level_constants", "tmg_transfer_matrices", "tmg_plan_info",
                     "tmg_plan_launches", "tmg_inspect", "tmg_profile_cycle"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def debug_bounds():
    """(violations, first record) of the debug build's bounds checks since
    the last call (tmg_debug_bounds), or None from the normal build."""
    c, f = ctypes.c_uint(0), ctypes.c_ulonglong(0)
    st = _lib().tmg_debug_bounds(ctypes.byref(c), ctypes.byref(f))
    if st == TMG_EUNSUPPORTED:
        return None
    _check(st, "tmg_debug_bounds")
    return c.value, f.value


def _check(status: int, where: str, ok=(TMG_OK,)):
    if status not in ok:
        raise TmgError(status, where)
    return status


def _dev_ptr(t, d: int, N: int, name: str):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() != N * d:
        raise ValueError(f"{name} has {t.numel()} elements, expected {N}*{d}")
    return ctypes.c_void_p(t.data_ptr())


def _order_after_current(stream, t):
    """A plan on a caller-given stream reads arrays that torch's current stream
    may still be writing: make the plan's stream wait for it first."""
    if stream is not None:
        import torch
        stream.wait_stream(torch.cuda.current_stream(t.device))


@dataclass
class SolveStats:
    status: int
    cycles: int
    rel_res: float
    hist: np.ndarray
    err_vs_fp64: float = float("nan")   # max|u - u_exact| / max|u_exact| (plans built with check_fp64)


class Plan:
    """tmg_setup / tmg_solve / tmg_destroy for one problem (see include/tmg.h)."""

    def __init__(self, p: int, tau: float, lam: float, N: int, levels: int = 0, omega: float = 0.0, *,
                 tol: float = 1e-10, max_cycles: int = 100, nu1: int = 1, nu2: int = 1, gamma: int = 1,
                 precision="mixed", n_min: int = 64, use_graph: bool = True, initial_guess: bool = False,
                 tail_cap: int = 0, use_pdl: bool = True, update_residual: bool = True,
                 fuse_levels=None, check_fp64: bool = False, stream=None):
        L = _lib()
        o = _Opts()
        L.tmg_opts_default(ctypes.byref(o))
        o.tol, o.max_cycles, o.nu1, o.nu2, o.gamma = tol, max_cycles, nu1, nu2, gamma
        o.precision = _PREC[precision]
        o.n_min, o.use_graph, o.initial_guess = n_min, int(use_graph), int(initial_guess)
        o.tail_cap = tail_cap
        o.use_pdl = int(use_pdl)
        o.update_residual = int(update_residual)
        o.fuse_levels = -1 if fuse_levels is None else int(bool(fuse_levels))
        o.check_fp64 = int(bool(check_fp64))
        self.precision = _PREC[precision]
        self.p, self.d, self.N = p, p + 1, N
        self.tau, self.lam = tau, lam
        self._stream = stream
        handle = _vp()
        sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        _check(L.tmg_setup(ctypes.byref(handle), p, tau, lam, N, levels, omega, ctypes.byref(o), sp), "tmg_setup")
        self._h = handle

    def close(self):
        if getattr(self, "_h", None):
            _lib().tmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, f, u0: float, u=None, *, allow_notconv: bool = False) -> "torch.Tensor":
        import torch
        if u is None:
            u = torch.empty((self.N, self.d), dtype=torch.float64, device=f.device)
        _order_after_current(self._stream, f)
        st = _lib().tmg_solve(self._h, _dev_ptr(f, self.d, self.N, "f"), float(u0), _dev_ptr(u, self.d, self.N, "u"))
        _check(st, "tmg_solve", (TMG_OK, TMG_ENOTCONV) if allow_notconv else (TMG_OK,))
        self.last_status = st
        return u

    def solve_direct(self, f, u0: float, u=None):
        """Exact FP64 solve by the parallel scan (tmg_solve_direct); not multigrid."""
        import torch
        if u is None:
            u = torch.empty((self.N, self.d), dtype=torch.float64, device=f.device)
        _order_after_current(self._stream, f)
        _check(_lib().tmg_solve_direct(self._h, _dev_ptr(f, self.d, self.N, "f"), float(u0),
                                       _dev_ptr(u, self.d, self.N, "u")), "tmg_solve_direct")
        return u

    def error_vs_fp64(self, f, u0: float, u) -> float:
        """max|u - u_exact| / max|u_exact| against the exact FP64 solve of the
        same system (tmg_error_vs_fp64)."""
        err = ctypes.c_double(0.0)
        _order_after_current(self._stream, u)
        _check(_lib().tmg_error_vs_fp64(self._h, _dev_ptr(f, self.d, self.N, "f"), float(u0),
                                        _dev_ptr(u, self.d, self.N, "u"), ctypes.byref(err)), "tmg_error_vs_fp64")
        return err.value

    def solve_host(self, f_host, u0: float, u_host) -> int:
        """f_host, u_host: contiguous float64 CPU tensors or numpy arrays (pinned tensors copy fastest)."""
        fp = ctypes.c_void_p(_host_ptr(f_host, self.d, self.N))
        up = ctypes.c_void_p(_host_ptr(u_host, self.d, self.N))
        return _check(_lib().tmg_solve_host(self._h, fp, float(u0), up), "tmg_solve_host")

    def adjoint(self, g, u, *, allow_notconv: bool = False):
        """(dJ/df, dJ/du0, dJ/dlambda) for dJ/du = g at the forward solution u (tmg_adjoint)."""
        import torch
        dJdf = torch.empty_like(g)
        scal = torch.zeros(2, dtype=torch.float64, device=g.device)
        _order_after_current(self._stream, g)
        st = _lib().tmg_adjoint(self._h, _dev_ptr(g, self.d, self.N, "g"), _dev_ptr(u, self.d, self.N, "u"),
                                _dev_ptr(dJdf, self.d, self.N, "dJdf"), ctypes.c_void_p(scal.data_ptr()),
                                ctypes.c_void_p(scal.data_ptr() + 8))
        _check(st, "tmg_adjoint", (TMG_OK, TMG_ENOTCONV) if allow_notconv else (TMG_OK,))
        return dJdf, scal[0], scal[1]

    def cycle(self, f, u0: float, u):
        _order_after_current(self._stream, f)
        _check(_lib().tmg_cycle(self._h, _dev_ptr(f, self.d, self.N, "f"), float(u0),
                                _dev_ptr(u, self.d, self.N, "u")), "tmg_cycle")
        return u

    def coarse_intervals(self) -> int:
        return self.info()["tail_intervals"]

    def cycle_down(self, f, u0: float, u, fc=None):
        """The way down of one V-cycle (tmg_cycle_down): returns the coarsest
        level's right-hand side fc (N_c, p+1) as a float64 CUDA tensor."""
        import torch
        nc = self.coarse_intervals()
        if fc is None:
            fc = torch.empty((nc, self.d), dtype=torch.float64, device=f.device)
        _order_after_current(self._stream, f)
        _check(_lib().tmg_cycle_down(self._h, _dev_ptr(f, self.d, self.N, "f"), float(u0),
                                     _dev_ptr(u, self.d, self.N, "u"), _dev_ptr(fc, self.d, nc, "fc")),
               "tmg_cycle_down")
        return fc

    def cycle_up(self, uc, u):
        """The way up of the cycle begun by cycle_down, from the coarsest
        level's correction uc (tmg_cycle_up); u += c."""
        _order_after_current(self._stream, uc)
        _check(_lib().tmg_cycle_up(self._h, _dev_ptr(uc, self.d, self.coarse_intervals(), "uc"),
                                   _dev_ptr(u, self.d, self.N, "u")), "tmg_cycle_up")
        return u

    def residual(self, f, u0: float, u, r=None):
        import torch
        if r is None:
            r = torch.empty_like(u)
        _order_after_current(self._stream, f)
        _check(_lib().tmg_residual(self._h, _dev_ptr(f, self.d, self.N, "f"), float(u0),
                                   _dev_ptr(u, self.d, self.N, "u"), _dev_ptr(r, self.d, self.N, "r")),
               "tmg_residual")
        return r

    def stats(self, hist_len: int = 512) -> SolveStats:
        cyc = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        err = ctypes.c_double(0.0)
        hist = np.full(hist_len, np.nan)
        _check(_lib().tmg_stats(self._h, ctypes.byref(cyc), ctypes.byref(rel), ctypes.byref(err),
                                hist.ctypes.data_as(_dp), hist_len), "tmg_stats")
        h = hist[: cyc.value + 1].copy()
        return SolveStats(getattr(self, "last_status", TMG_OK), cyc.value, rel.value, h, err.value)

    def profile_cycle(self, f, u0: float, u, reps: int = 10) -> dict:
        """Mean per-kernel milliseconds of one correction cycle (CUDA events on the plan's stream)."""
        ms = np.zeros(6)
        _order_after_current(self._stream, f)
        _check(_lib().tmg_profile_cycle(self._h, _dev_ptr(f, self.d, self.N, "f"), float(u0),
                                        _dev_ptr(u, self.d, self.N, "u"), reps, ms.ctypes.data_as(_dp), 6),
               "tmg_profile_cycle")
        return dict(zip(["down0", "down_levels", "coarse_on_chip", "up_levels", "up0", "cycle"], ms.tolist()))

    def inspect(self, which: str, level: int = 0) -> np.ndarray:
        """Copy an internal level vector ('f', 'u' of a level, the level-0 residual 'r', or the low
        float parts 'rlo' of a residual kept as a float pair) to host."""
        w = {"f": 0, "u": 1, "r": 2, "rlo": 3}[which]
        n = self.N if w >= 2 else self.N >> level
        dt = np.float64 if self.precision == FP64 and w != 3 else np.float32
        out = np.empty((n, self.d), dtype=dt)
        _check(_lib().tmg_inspect(self._h, w, level, ctypes.c_void_p(out.ctypes.data), out.nbytes), "tmg_inspect")
        return out

    def launches_per_cycle(self) -> int:
        """Kernels one cycle launches (tmg_plan_launches)."""
        n = ctypes.c_int(0)
        _check(_lib().tmg_plan_launches(self._h, ctypes.byref(n)), "tmg_plan_launches")
        return n.value

    def info(self):
        nl = ctypes.c_int(0)
        lt = ctypes.c_int(0)
        nt = ctypes.c_int64(0)
        om = np.full(64, np.nan)
        _check(_lib().tmg_plan_info(self._h, ctypes.byref(nl), ctypes.byref(lt), ctypes.byref(nt),
                                    om.ctypes.data_as(_dp), 64), "tmg_plan_info")
        return {"levels": nl.value, "tail_level": lt.value, "tail_intervals": nt.value,
                "omega": om[: nl.value].copy()}


def _host_ptr(x, d: int, N: int) -> int:
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != N * d:
                raise TypeError("host tensor must be contiguous CPU float64 with N*d elements")
            return x.data_ptr()
    except ImportError:
        pass
    a = np.asarray(x)
    if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != N * d:
        raise TypeError("host array must be contiguous float64 with N*d elements")
    return a.ctypes.data


def residual_norm_noalloc(p: int, tau: float, lam: float, f, u0: float, u, r, norm, stream=None) -> None:
    """r = F - L u and ||r||_2 (into the one-element float64 CUDA tensor ``norm``)
    through tmg_residual_norm_noalloc: no plan and no device allocation, for
    callers that may not allocate device memory at that point.  Asynchronous on
    ``stream``; by default torch's current stream on u's device.  A caller-given
    stream first waits for torch's current stream, which may still be writing
    f or u."""
    d = p + 1
    N = f.numel() // d
    import torch
    if not (isinstance(norm, torch.Tensor) and norm.is_cuda and norm.dtype == torch.float64 and norm.numel() == 1):
        raise TypeError("norm must be a one-element float64 CUDA tensor")
    if stream is None:
        stream = torch.cuda.current_stream(u.device)
    else:
        _order_after_current(stream, u)
    sp = ctypes.c_void_p(stream.cuda_stream)
    _check(_lib().tmg_residual_norm_noalloc(p, tau, lam, N, _dev_ptr(f, d, N, "f"), float(u0), _dev_ptr(u, d, N, "u"),
                                            _dev_ptr(r, d, N, "r"), ctypes.c_void_p(norm.data_ptr()), sp),
           "tmg_residual_norm_noalloc")


def _opts(**kw) -> _Opts:
    o = _Opts()
    _lib().tmg_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision":
            v = _PREC[v]
        setattr(o, k, int(v) if isinstance(v, bool) else v)
    return o


def plan_shape(p: int, tau: float, lam: float, N: int, levels: int = 0, omega: float = 0.0, **opts) -> dict:
    """The hierarchy tmg_setup would build (tmg_plan_shape; host only, no GPU).
    Keyword options as tmg_opts fields (precision="fp64"/"mixed", n_min, gamma,
    tail_cap, ...)."""
    nl, lt, sc = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    nt = ctypes.c_int64(0)
    _check(_lib().tmg_plan_shape(p, tau, lam, N, levels, omega, ctypes.byref(_opts(**opts)), ctypes.byref(nl),
                                 ctypes.byref(lt), ctypes.byref(nt), ctypes.byref(sc)), "tmg_plan_shape")
    return {"levels": nl.value, "tail_level": lt.value, "tail_intervals": nt.value, "scan_coarsest": bool(sc.value)}


def level_constants(p: int, z: float, omega: float = 0.0) -> dict:
    """The library's host set-up of one level (tmg_level_constants): A, A^{-1},
    g, c, alpha and the damping, as numpy arrays / floats."""
    d = p + 1
    A, Ai = np.zeros((d, d)), np.zeros((d, d))
    g, c = np.zeros(d), np.zeros(d)
    al, om = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib().tmg_level_constants(p, z, omega, A.ctypes.data_as(_dp), Ai.ctypes.data_as(_dp),
                                      g.ctypes.data_as(_dp), c.ctypes.data_as(_dp), ctypes.byref(al),
                                      ctypes.byref(om)), "tmg_level_constants")
    return {"A": A, "Ainv": Ai, "g": g, "c": c, "alpha": al.value, "omega": om.value}


def transfer_matrices(p: int):
    """The library's prolongation matrices (P1, P2) (tmg_transfer_matrices)."""
    d = p + 1
    P1, P2 = np.zeros((d, d)), np.zeros((d, d))
    _check(_lib().tmg_transfer_matrices(p, P1.ctypes.data_as(_dp), P2.ctypes.data_as(_dp)),
           "tmg_transfer_matrices")
    return P1, P2


class Batch:
    """tmg_setup_batched / tmg_solve_batched / tmg_adjoint_batched (include/tmg.h).

    Instance i has degree p[i], step tau[i], lam[i] and N[i] intervals; device
    arrays are packed [instance][interval][coefficient] (float64)."""

    def __init__(self, p, tau, lam, N, omega: float = 0.0, *, stream=None, **opts):
        p = np.ascontiguousarray(p, dtype=np.int32)
        tau = np.ascontiguousarray(np.broadcast_to(tau, p.shape), dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        N = np.ascontiguousarray(np.broadcast_to(N, p.shape), dtype=np.int64)
        self.p, self.tau, self.lam, self.N = p, tau, lam, N
        self.n = int(p.shape[0])
        self.offsets = np.concatenate([[0], np.cumsum(N * (p + 1))]).astype(np.int64)
        self.total = int(self.offsets[-1])
        self._stream = stream
        o = _opts(**opts)
        h = _vp()
        sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        _check(_lib().tmg_setup_batched(ctypes.byref(h), self.n, p.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        tau.ctypes.data_as(_dp), lam.ctypes.data_as(_dp),
                                        N.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), omega, ctypes.byref(o), sp),
               "tmg_setup_batched")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib().tmg_destroy_batched(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _ptr(self, t, n, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and t.numel() == n):
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor with {n} elements")
        return ctypes.c_void_p(t.data_ptr())

    def solve(self, f, u0, u=None, *, allow_notconv: bool = False):
        import torch
        if u is None:
            u = torch.empty(self.total, dtype=torch.float64, device=f.device)
        _order_after_current(self._stream, f)
        st = _lib().tmg_solve_batched(self._h, self._ptr(f, self.total, "f"), self._ptr(u0, self.n, "u0"),
                                      self._ptr(u, self.total, "u"))
        _check(st, "tmg_solve_batched", (TMG_OK, TMG_ENOTCONV) if allow_notconv else (TMG_OK,))
        return u

    def adjoint(self, g, u, *, allow_notconv: bool = False):
        import torch
        dJdf = torch.empty_like(g)
        du0 = torch.empty(self.n, dtype=torch.float64, device=g.device)
        dlam = torch.empty(self.n, dtype=torch.float64, device=g.device)
        _order_after_current(self._stream, g)
        st = _lib().tmg_adjoint_batched(self._h, self._ptr(g, self.total, "g"), self._ptr(u, self.total, "u"),
                                        self._ptr(dJdf, self.total, "dJdf"), self._ptr(du0, self.n, "dJdu0"),
                                        self._ptr(dlam, self.n, "dJdlambda"))
        _check(st, "tmg_adjoint_batched", (TMG_OK, TMG_ENOTCONV) if allow_notconv else (TMG_OK,))
        return dJdf, du0, dlam

    def stats(self):
        cyc = np.zeros(self.n, dtype=np.int32)
        rel = np.zeros(self.n)
        mx = ctypes.c_int(0)
        _check(_lib().tmg_stats_batched(self._h, cyc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        rel.ctypes.data_as(_dp), None, ctypes.byref(mx)), "tmg_stats_batched")
        return cyc, rel, mx.value

    def error_vs_fp64(self, f, u0, u) -> np.ndarray:
        """Per-instance max|u_i - u_exact,i| / max|u_exact,i| of the given
        results against the exact FP64 solves (tmg_error_vs_fp64_batched)."""
        err = np.zeros(self.n)
        _order_after_current(self._stream, u)
        _check(_lib().tmg_error_vs_fp64_batched(self._h, self._ptr(f, self.total, "f"), self._ptr(u0, self.n, "u0"),
                                                self._ptr(u, self.total, "u"), err.ctypes.data_as(_dp)),
               "tmg_error_vs_fp64_batched")
        return err

    def err_vs_fp64(self) -> np.ndarray:
        """Per-instance max|u_i - u_exact,i| / max|u_exact,i| of the last solve
        against the exact FP64 solve (batches built with check_fp64=True; NAN
        otherwise)."""
        err = np.zeros(self.n)
        _check(_lib().tmg_stats_batched(self._h, None, None, err.ctypes.data_as(_dp), None), "tmg_stats_batched")
        return err

    def info(self):
        ng = ctypes.c_int(0)
        pv = ctypes.c_int64(0)
        _check(_lib().tmg_batch_info(self._h, ctypes.byref(ng), ctypes.byref(pv)), "tmg_batch_info")
        groups = []
        for g in range(ng.value):
            p, sch = ctypes.c_int(0), ctypes.c_int(0)
            Ng, n = ctypes.c_int64(0), ctypes.c_int64(0)
            mg, mc = ctypes.c_double(0), ctypes.c_double(0)
            _check(_lib().tmg_batch_group_info(self._h, g, ctypes.byref(p), ctypes.byref(Ng), ctypes.byref(n),
                                               ctypes.byref(sch), ctypes.byref(mg), ctypes.byref(mc)),
                   "tmg_batch_group_info")
            groups.append({"p_t": p.value, "padded_length": Ng.value, "instances": n.value,
                           "schedule": {1: "grid", 2: "cta"}.get(sch.value, "?"), "ms_grid": mg.value,
                           "ms_cta": mc.value})
        mt, mgr = ctypes.c_double(0), ctypes.c_double(0)
        _check(_lib().tmg_batch_tune_info(self._h, ctypes.byref(mt), ctypes.byref(mgr)), "tmg_batch_tune_info")
        return {"groups": ng.value, "padded_values": pv.value, "group_info": groups,
                "whole_batch_ms": {"tuned": mt.value, "all_grid": mgr.value}}

    def split(self, x):
        """Per-instance views (N_i, p_i + 1) of a packed host array."""
        x = np.asarray(x)
        return [x[self.offsets[i]:self.offsets[i + 1]].reshape(int(self.N[i]), int(self.p[i]) + 1)
                for i in range(self.n)]


class HeatPlan:
    """tmg_heat_setup / tmg_heat_solve / tmg_heat_destroy: the space-time heat
    equation on an n x n grid with N DG-in-time intervals of degree p (see
    include/tmg.h).  Arrays are float64 CUDA tensors of shape (N, p+1, n, n);
    u0 has shape (n, n)."""

    def __init__(self, p: int, tau: float, n: int, N: int, *, tol: float = 1e-10, max_cycles: int = 100,
                 nu1: int = 1, nu2: int = 1, nu_c: int = 2, precision="mixed", use_graph: bool = True,
                 stream=None):
        L = _lib()
        o = _opts(tol=tol, max_cycles=max_cycles, nu1=nu1, nu2=nu2, gamma=1, precision=precision,
                  use_graph=use_graph)
        self.p, self.d, self.n, self.N, self.tau = p, p + 1, n, N, tau
        self._stream = stream
        handle = _vp()
        sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        _check(L.tmg_heat_setup(ctypes.byref(handle), p, tau, n, N, ctypes.byref(o), nu_c, sp), "tmg_heat_setup")
        self._h = handle

    def close(self):
        if getattr(self, "_h", None):
            _lib().tmg_heat_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _ptr(self, t, shape, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
        if tuple(t.shape) != tuple(shape) and t.numel() != int(np.prod(shape)):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        _order_after_current(self._stream, t)
        return ctypes.c_void_p(t.data_ptr())

    def _shape(self):
        return (self.N, self.d, self.n, self.n)

    def solve(self, f, u0, u=None, *, allow_notconv: bool = False):
        import torch
        if u is None:
            u = torch.empty(self._shape(), dtype=torch.float64, device=f.device)
        ok = (TMG_OK, TMG_ENOTCONV) if allow_notconv else (TMG_OK,)
        _check(_lib().tmg_heat_solve(self._h, self._ptr(f, self._shape(), "f"), self._ptr(u0, (self.n, self.n), "u0"),
                                     self._ptr(u, self._shape(), "u")), "tmg_heat_solve", ok)
        return u

    def cycle(self, f, u0, u):
        _check(_lib().tmg_heat_cycle(self._h, self._ptr(f, self._shape(), "f"), self._ptr(u0, (self.n, self.n), "u0"),
                                     self._ptr(u, self._shape(), "u")), "tmg_heat_cycle")
        return u

    def residual(self, f, u0, u, r=None):
        import torch
        if r is None:
            r = torch.empty(self._shape(), dtype=torch.float64, device=f.device)
        _check(_lib().tmg_heat_residual(self._h, self._ptr(f, self._shape(), "f"),
                                        self._ptr(u0, (self.n, self.n), "u0"), self._ptr(u, self._shape(), "u"),
                                        self._ptr(r, self._shape(), "r")), "tmg_heat_residual")
        return r

    def stats(self, hist_len: int = 256) -> SolveStats:
        c = ctypes.c_int(0)
        rel = ctypes.c_double(0)
        hist = np.full(hist_len, np.nan)
        _check(_lib().tmg_heat_stats(self._h, ctypes.byref(c), ctypes.byref(rel),
                                     hist.ctypes.data_as(_dp), hist_len), "tmg_heat_stats")
        return SolveStats(TMG_OK, c.value, rel.value, hist[~np.isnan(hist)])

    def info(self) -> dict:
        tl, sl, lc = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        ws = ctypes.c_size_t(0)
        _check(_lib().tmg_heat_info(self._h, ctypes.byref(tl), ctypes.byref(sl), ctypes.byref(lc), ctypes.byref(ws)),
               "tmg_heat_info")
        return {"time_levels": tl.value, "space_levels": sl.value, "launches_per_cycle": lc.value,
                "workspace_bytes": ws.value}

    def profile(self, f, u0, u, reps: int = 10) -> dict:
        """Per-launch CUDA-event times (ms) of the level-0 kernels and of one
        cycle (tmg_heat_profile); u is left arbitrary."""
        ms = np.zeros(5)
        _check(_lib().tmg_heat_profile(self._h, self._ptr(f, self._shape(), "f"), self._ptr(u0, (self.n, self.n), "u0"),
                                       self._ptr(u, self._shape(), "u"), reps, ms.ctypes.data_as(_dp), 5),
               "tmg_heat_profile")
        return {"resid": ms[0], "pre": ms[1], "post": ms[2], "update": ms[3], "cycle": ms[4]}
