"""Oracle for the time-multigrid DG-in-time solve (Gander & Neumueller, arXiv:1409.5254).

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously-correct FP64 CPU
implementation of what the GPU path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import it.  It shares no code with the CUDA library and never calls it.

Parts (each cites the paper passage it follows):

* ``blocks``/``alpha``/``omega_star``/``transfer`` -- the local DG matrices of
  Section 2 ("Linear system"), the stability value alpha of Lemma
  chap4_theorem2, the damping omega* of Lemma chap4_lemma7 and the local
  transfer matrices R1^T, R2^T of Section 4.2 -- all computed by quadrature from
  the definitions (``tmg_oracle.c``).
* ``fsub`` -- exact block forward substitution for eq.
  chap4_generalLinearSystemODE (the plain definition of the result).
* ``dense_solve`` -- brute-force Gaussian elimination of the assembled system.
* ``mg_solve`` / ``mg_one_cycle`` / ``mg_cycle_down`` / ``mg_cycle_up`` -- a
  textbook recursive multigrid cycle (the last two cut it at a level):
  damped block Jacobi (eq. chap4_ODESmoother), residual, restriction R = P^T
  (eqs. chap4_restrictionTime/chap4_prolongationTime), recursion (V or W) with
  an exact coarsest solve, prolongation, post-smoothing
  (eq. chap4_errorTwoGridCycle).
* ``adj_sweep`` / ``adjoint_grads`` -- the transposed system solved backward in
  time and the gradients of a loss with respect to f, u0 and lambda.
* ``oracle.lfa`` -- the local Fourier analysis of Section 4 (numpy).

Every function works with z = lambda * tau (the step enters only through z).
Arrays are float64 with shape (N, d), d = p + 1, interval-major.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmg_oracle.c")
_SO = os.path.join(_HERE, "_build", "libtmg_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags only) and return the .so path."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c_int, c_long, c_double = ctypes.c_int, ctypes.c_long, ctypes.c_double
            L.orc_max_degree.argtypes = []
            L.orc_max_degree.restype = c_int
            L.orc_blocks.argtypes = [c_int, _dp, _dp, _dp, _dp]
            L.orc_transfer.argtypes = [c_int, _dp, _dp]
            L.orc_alpha.argtypes = [c_int, c_double]
            L.orc_alpha.restype = c_double
            L.orc_omega_star.argtypes = [c_int, c_double]
            L.orc_omega_star.restype = c_double
            L.orc_gesv.argtypes = [c_int, _dp, _dp, _dp]
            L.orc_gesv.restype = c_int
            L.orc_fsub.argtypes = [c_int, c_double, c_long, _dp, c_double, _dp]
            L.orc_dense_solve.argtypes = [c_int, c_double, c_long, _dp, c_double, _dp]
            L.orc_dense_solve.restype = c_int
            L.orc_num_levels.argtypes = [c_long, c_long, c_int]
            L.orc_num_levels.restype = c_int
            L.orc_mg_solve.argtypes = [c_int, c_double, c_long, _dp, c_double, _dp, c_long, c_int,
                                       c_int, c_int, c_int, c_double, c_double, c_int, _dp]
            L.orc_mg_solve.restype = c_int
            L.orc_mg_one_cycle.argtypes = [c_int, c_double, c_long, _dp, _dp, c_long, c_int,
                                           c_int, c_int, c_int, c_double]
            L.orc_residual.argtypes = [c_int, c_double, c_long, _dp, c_double, _dp, _dp]
            L.orc_mg_cycle_split.argtypes = [c_int, c_double, c_long, _dp, _dp, c_long, c_int, c_int, c_int,
                                             c_double, c_int, c_int, _dp, _dp]
            L.orc_adj_sweep.argtypes = [c_int, c_double, c_long, _dp, _dp]
            L.orc_adjoint_grads.argtypes = [c_int, c_double, c_double, c_long, _dp, _dp, _dp, _dp, _dp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def max_degree() -> int:
    """Largest DG degree p the oracle accepts (its fixed local arrays and the
    Gauss rule exact for products of two basis functions)."""
    return lib().orc_max_degree()


def _deg(p: int) -> int:
    if not 0 <= int(p) <= max_degree():
        raise ValueError(f"degree p={p} outside 0..{max_degree()}")
    return int(p)


def _vec(F, p):
    _deg(p)
    F = np.ascontiguousarray(F, dtype=np.float64)
    d = p + 1
    assert F.ndim == 2 and F.shape[1] == d, (F.shape, d)
    return F


def blocks(p: int):
    """(K, Mhat, a, b) on the reference interval; N = outer(a, b) (Section 2)."""
    d = _deg(p) + 1
    K, M, a, b = (np.zeros((d, d)), np.zeros((d, d)), np.zeros(d), np.zeros(d))
    lib().orc_blocks(p, _ptr(K), _ptr(M), _ptr(a), _ptr(b))
    return K, M, a, b


def transfer(p: int):
    """(P1, P2) = (R1^T, R2^T): coarse-to-fine maps onto the two halves (Section 4.2)."""
    d = _deg(p) + 1
    P1, P2 = np.zeros((d, d)), np.zeros((d, d))
    lib().orc_transfer(p, _ptr(P1), _ptr(P2))
    return P1, P2


def alpha(p: int, z: float) -> float:
    """b^T (K + z Mhat)^{-1} a: the nonzero eigenvalue of A^{-1}N (Lemma chap4_theorem2)."""
    return lib().orc_alpha(_deg(p), float(z))


def omega_star(p: int, z: float) -> float:
    """omega* of Lemma chap4_lemma7 at z = lambda*tau_L."""
    return lib().orc_omega_star(_deg(p), float(z))


def num_levels(N: int, n_min: int = 64, max_levels: int = 0) -> int:
    return lib().orc_num_levels(int(N), int(n_min), int(max_levels))


def fsub(p: int, z: float, F, u0: float = 0.0) -> np.ndarray:
    """Exact solution of eq. chap4_generalLinearSystemODE by block forward substitution."""
    F = _vec(F, p)
    u = np.zeros_like(F)
    lib().orc_fsub(p, float(z), F.shape[0], _ptr(F), float(u0), _ptr(u))
    return u


def dense_solve(p: int, z: float, F, u0: float = 0.0) -> np.ndarray:
    """Gaussian elimination on the assembled (N d)x(N d) system (small N only)."""
    F = _vec(F, p)
    u = np.zeros_like(F)
    st = lib().orc_dense_solve(p, float(z), F.shape[0], _ptr(F), float(u0), _ptr(u))
    if st != 0:
        raise ArithmeticError("singular system")
    return u


def residual(p: int, z: float, F, u0: float, u) -> np.ndarray:
    """F - L u with a*u0 added to the first interval."""
    F = _vec(F, p)
    u = _vec(u, p)
    r = np.zeros_like(F)
    lib().orc_residual(p, float(z), F.shape[0], _ptr(F), float(u0), _ptr(u), _ptr(r))
    return r


def mg_solve(p: int, z: float, F, u0: float = 0.0, *, n_min: int = 64, max_levels: int = 0,
             nu1: int = 1, nu2: int = 1, gamma: int = 1, omega: float = 0.0, tol: float = 1e-10,
             max_cycles: int = 100, u_init=None):
    """Textbook multigrid solve.  Returns (u, hist) where hist[k] = ||F - L u_k|| / ||F||."""
    F = _vec(F, p)
    u = np.zeros_like(F) if u_init is None else _vec(u_init, p).copy()
    hist = np.zeros(max_cycles + 1)
    k = lib().orc_mg_solve(p, float(z), F.shape[0], _ptr(F), float(u0), _ptr(u), int(n_min),
                           int(max_levels), int(nu1), int(nu2), int(gamma), float(omega),
                           float(tol), int(max_cycles), _ptr(hist))
    return u, hist[: k + 1].copy()


def mg_one_cycle(p: int, z: float, Fhat, u, *, n_min: int = 64, max_levels: int = 0, nu1: int = 1,
                 nu2: int = 1, gamma: int = 1, omega: float = 0.0) -> np.ndarray:
    """One cycle on L u = Fhat (Fhat already holds a*u0 in its first interval)."""
    Fhat = _vec(Fhat, p)
    u = _vec(u, p).copy()
    lib().orc_mg_one_cycle(p, float(z), Fhat.shape[0], _ptr(Fhat), _ptr(u), int(n_min),
                           int(max_levels), int(nu1), int(nu2), int(gamma), float(omega))
    return u


def mg_cycle_down(p: int, z: float, Fhat, u, stop: int, *, n_min: int = 64, max_levels: int = 0, nu1: int = 1,
                  nu2: int = 1, omega: float = 0.0) -> np.ndarray:
    """The way down of one V-cycle on L u = Fhat to level `stop` of its
    hierarchy: that level's right-hand side (N/2^stop intervals); u unchanged."""
    Fhat = _vec(Fhat, p)
    u = _vec(u, p).copy()
    fc = np.zeros((Fhat.shape[0] >> stop, p + 1))
    lib().orc_mg_cycle_split(p, float(z), Fhat.shape[0], _ptr(Fhat), _ptr(u), int(n_min), int(max_levels), int(nu1),
                             int(nu2), float(omega), int(stop), 0, _ptr(fc), _ptr(fc))
    return fc


def mg_cycle_up(p: int, z: float, Fhat, u, uc, stop: int, *, n_min: int = 64, max_levels: int = 0, nu1: int = 1,
                nu2: int = 1, omega: float = 0.0) -> np.ndarray:
    """The same way down again, then uc as level `stop`'s correction and the
    way up: the cycle's new iterate."""
    Fhat = _vec(Fhat, p)
    u = _vec(u, p).copy()
    uc = np.ascontiguousarray(uc, dtype=np.float64)
    assert uc.shape == (Fhat.shape[0] >> stop, p + 1)
    lib().orc_mg_cycle_split(p, float(z), Fhat.shape[0], _ptr(Fhat), _ptr(u), int(n_min), int(max_levels), int(nu1),
                             int(nu2), float(omega), int(stop), 1, _ptr(uc), _ptr(uc))
    return u


def fold_u0(p: int, F, u0: float) -> np.ndarray:
    """F with a*u0 added to the first interval (the n = 1 term of eq. chap4_discreteVarFormODE)."""
    F = _vec(F, p).copy()
    _, _, a, _ = blocks(p)
    F[0] += a * u0
    return F


def adj_sweep(p: int, z: float, g) -> np.ndarray:
    """mu = L^{-T} g, backward in time."""
    g = _vec(g, p)
    mu = np.zeros_like(g)
    lib().orc_adj_sweep(p, float(z), g.shape[0], _ptr(g), _ptr(mu))
    return mu


def adjoint_grads(p: int, lam: float, tau: float, g, u):
    """(dJ/df, dJ/du0, dJ/dlambda) for dJ/du = g at the solution u."""
    g = _vec(g, p)
    u = _vec(u, p)
    dJdf = np.zeros_like(g)
    du0 = ctypes.c_double(0.0)
    dlam = ctypes.c_double(0.0)
    lib().orc_adjoint_grads(p, float(lam), float(tau), g.shape[0], _ptr(g), _ptr(u), _ptr(dJdf),
                            ctypes.byref(du0), ctypes.byref(dlam))
    return dJdf, du0.value, dlam.value


def nodal_values(p: int, u) -> np.ndarray:
    """Right-endpoint values e_n = b^T u_n."""
    _, _, _, b = blocks(p)
    return _vec(u, p) @ b
