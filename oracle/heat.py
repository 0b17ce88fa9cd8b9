"""Oracle for the space-time heat equation (the paper's outlook, Section 7).

TEST INFRASTRUCTURE ONLY: plain FP64 numpy, slow and obviously correct.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import it; it shares no code with the CUDA library.

Problem: u_t - Delta u = f on the unit square (zero Dirichlet boundary) and
(0, T), u(0) = u0.  Space: the 5-point finite-difference Laplacian A_h on an
n x n interior grid, h = 1/(n+1), n = 2^k - 1.  Time: the DG discretisation
of Section 2 with the shifted Legendre basis, so every interval carries a
(p+1)-vector of spatial fields and the system is block lower-bidiagonal:

    G_tau u_n - (a b^T (x) I) u_{n-1} = F_n,   G_tau = K (x) I + tau Mhat (x) A_h,

(the scalar system of eq. chap4_generalLinearSystemODE with lambda replaced by
the operator A_h).  Arrays are float64 of shape (N, p+1, n, n).

The solver is the multigrid in time of Section 3 with the block Jacobi
smoother of eq. chap4_ODESmoother, in which -- as the paper's outlook for the
heat equation proposes -- the inverse of the block G_tau is replaced by ONE
multigrid V-cycle in space:
* time: damped block Jacobi with omega_t = 1/2 (the uniform damping of the
  remark after Lemma chap4_lemma7, which bounds the smoothing factor of every
  spatial mode at once), residual, restriction R = P^T and prolongation P of
  Section 4.2 acting on the Legendre coefficients of every grid point, V-cycles
  coarsening time by two down to one interval, whose block is solved by
  nu_c spatial V-cycles;
* space: a V(1,1)-cycle on G_tau x = r from a zero start: damped point-block
  Jacobi (omega_s = 4/5) with the (p+1) x (p+1) block K + tau (4/h^2) Mhat of
  each grid point, full-weighting restriction, bilinear prolongation,
  re-discretised coarse operators (h -> 2h) down to one grid point, solved
  exactly.
"""
from __future__ import annotations

import numpy as np

from . import blocks, transfer

OMEGA_T = 0.5
OMEGA_S = 0.8


def grid_h(n: int) -> float:
    return 1.0 / (n + 1)


def laplacian(u, h):
    """A_h u: (4 u_ij - u_(i-1)j - u_(i+1)j - u_i(j-1) - u_i(j+1)) / h^2 over the
    last two axes, zero outside the grid (Dirichlet boundary)."""
    out = 4.0 * u
    out[..., 1:, :] -= u[..., :-1, :]
    out[..., :-1, :] -= u[..., 1:, :]
    out[..., :, 1:] -= u[..., :, :-1]
    out[..., :, :-1] -= u[..., :, 1:]
    return out / (h * h)


def coef_apply(M, x):
    """(M x)_k = sum_l M[k, l] x_l over the coefficient axis (-3)."""
    return np.einsum("kl,...lij->...kij", M, x)


def block_apply(p: int, tau: float, h: float, x):
    """G_tau x = K x + tau Mhat A_h x for every interval."""
    K, Mh, _, _ = blocks(p)
    return coef_apply(K, x) + tau * coef_apply(Mh, laplacian(x, h))


def point_block(p: int, tau: float, h: float):
    """The diagonal block of G_tau at one grid point: K + tau (4/h^2) Mhat."""
    K, Mh, _, _ = blocks(p)
    return K + tau * (4.0 / (h * h)) * Mh


def restrict_space(r):
    """Full weighting onto the (n-1)/2 coarse grid: coarse (I, J) sits on fine
    (2I+1, 2J+1); weights 4 (centre), 2 (edge neighbours), 1 (corners), / 16."""
    c = r[..., 1::2, 1::2] * 4.0
    c = c + 2.0 * (r[..., 0:-1:2, 1::2] + r[..., 2::2, 1::2] + r[..., 1::2, 0:-1:2] + r[..., 1::2, 2::2])
    c = c + r[..., 0:-1:2, 0:-1:2] + r[..., 2::2, 0:-1:2] + r[..., 0:-1:2, 2::2] + r[..., 2::2, 2::2]
    return c / 16.0


def prolong_space(xc, n: int):
    """Bilinear interpolation from the coarse grid onto the n x n fine grid
    (zero on the boundary), the transpose of restrict_space times 4."""
    shape = xc.shape[:-2] + (n + 2, n + 2)
    X = np.zeros(shape)
    X[..., 2:-1:2, 2:-1:2] = xc                       # coarse points (padded index 2I+2)
    X[..., 1::2, 2:-1:2] = 0.5 * (X[..., 0:-1:2, 2:-1:2] + X[..., 2::2, 2:-1:2])
    X[..., :, 1::2] = 0.5 * (X[..., :, 0:-1:2] + X[..., :, 2::2])
    return X[..., 1:-1, 1:-1]


def spatial_vcycle(p: int, tau: float, n: int, r, nu1: int = 1, nu2: int = 1):
    """One V(nu1, nu2)-cycle in space on G_tau x = r from x = 0 (every
    interval at once); returns x."""
    h = grid_h(n)
    Dinv = np.linalg.inv(point_block(p, tau, h))
    if n == 1:
        return coef_apply(Dinv, r)                    # one grid point: G_tau is its point block
    x = np.zeros_like(r)
    for _ in range(nu1):
        x = x + OMEGA_S * coef_apply(Dinv, r - block_apply(p, tau, h, x))
    res = r - block_apply(p, tau, h, x)
    nc = (n - 1) // 2
    xc = spatial_vcycle(p, tau, nc, restrict_space(res), nu1, nu2)
    x = x + prolong_space(xc, n)
    for _ in range(nu2):
        x = x + OMEGA_S * coef_apply(Dinv, r - block_apply(p, tau, h, x))
    return x


def endvals(u):
    """e_n = b^T u_n = sum of the Legendre coefficients, a spatial field."""
    return u.sum(axis=-3)


def time_residual(p: int, tau: float, n: int, F, u, u0=None):
    """r = F - L u: G_tau u_n - a (b^T u_{n-1}) with u0 before the first interval."""
    _, _, a, _ = blocks(p)
    e = np.zeros_like(u[:, 0])
    e[1:] = endvals(u[:-1])
    if u0 is not None:
        e[0] = u0
    return F + a[None, :, None, None] * e[:, None] - block_apply(p, tau, grid_h(n), u)


def fold_u0(p: int, F, u0):
    """F with a (x) u0 added to the first interval."""
    _, _, a, _ = blocks(p)
    F = np.array(F, dtype=np.float64, copy=True)
    F[0] += a[:, None, None] * u0
    return F


def exact_solve(p: int, tau: float, n: int, F, u0):
    """Block forward substitution, each block solved exactly in the sine basis
    that diagonalises A_h (the 2-D discrete sine transform, a library
    routine): the plain definition of the result."""
    from scipy.fft import dstn, idstn
    K, Mh, a, b = blocks(p)
    h = grid_h(n)
    k = np.arange(1, n + 1)
    lam1 = (4.0 / h ** 2) * np.sin(k * np.pi * h / 2.0) ** 2
    lam = lam1[:, None] + lam1[None, :]               # eigenvalues of A_h
    N, d = F.shape[0], p + 1
    u = np.zeros_like(F)
    e_prev = np.array(u0, dtype=np.float64)
    for m in range(N):
        rhs = F[m] + a[:, None, None] * e_prev[None]
        rh = dstn(rhs, type=1, axes=(-2, -1), norm="ortho")
        Ablk = K[None, None] + tau * lam[:, :, None, None] * Mh[None, None]   # (n, n, d, d)
        xh = np.linalg.solve(Ablk, np.moveaxis(rh, 0, -1)[..., None])[..., 0]
        u[m] = idstn(np.moveaxis(xh, -1, 0), type=1, axes=(-2, -1), norm="ortho")
        e_prev = endvals(u[m])
    return u


def _coarse_block_solve(p, tau, n, r, nu_c):
    """nu_c spatial V-cycles on G_tau x = r from zero (the coarsest time level)."""
    h = grid_h(n)
    x = np.zeros_like(r)
    for _ in range(nu_c):
        x = x + spatial_vcycle(p, tau, n, r - block_apply(p, tau, h, x))
    return x


def time_cycle(p: int, tau: float, n: int, Fhat, u, *, nu1: int = 1, nu2: int = 1, nu_c: int = 2,
               exact_blocks: bool = False):
    """One V-cycle in time on L u = Fhat (u0 folded into Fhat), returns the new
    u.  Block Jacobi sweeps u_n += omega_t B^{-1}(Fhat_n + a e_{n-1} - G u_n),
    B^{-1} one spatial V-cycle from zero (or, with exact_blocks, the exact
    block solve -- the pin against the decoupled modes); restriction and
    prolongation on the Legendre axis; time levels down to one interval,
    solved by nu_c spatial V-cycles (exactly, with exact_blocks)."""
    u = np.array(u, dtype=np.float64, copy=True)
    N = u.shape[0]

    def bsolve(t, r):
        return _exact_blocks(p, t, n, r) if exact_blocks else spatial_vcycle(p, t, n, r)

    if N == 1:
        r = time_residual(p, tau, n, Fhat, u)
        return u + (_exact_blocks(p, tau, n, r) if exact_blocks else _coarse_block_solve(p, tau, n, r, nu_c))
    for _ in range(nu1):
        u = u + OMEGA_T * bsolve(tau, time_residual(p, tau, n, Fhat, u))
    r = time_residual(p, tau, n, Fhat, u)
    P1, P2 = transfer(p)
    rc = coef_apply(P1.T, r[0::2]) + coef_apply(P2.T, r[1::2])
    uc = time_cycle(p, 2.0 * tau, n, rc, np.zeros_like(rc), nu1=nu1, nu2=nu2, nu_c=nu_c, exact_blocks=exact_blocks)
    u[0::2] += coef_apply(P1, uc)
    u[1::2] += coef_apply(P2, uc)
    for _ in range(nu2):
        u = u + OMEGA_T * bsolve(tau, time_residual(p, tau, n, Fhat, u))
    return u


def _exact_blocks(p, tau, n, r):
    """G_tau^{-1} applied to every interval independently (no time coupling)."""
    from scipy.fft import dstn, idstn
    K, Mh, _, _ = blocks(p)
    h = grid_h(n)
    k = np.arange(1, n + 1)
    lam1 = (4.0 / h ** 2) * np.sin(k * np.pi * h / 2.0) ** 2
    lam = lam1[:, None] + lam1[None, :]
    rh = dstn(r, type=1, axes=(-2, -1), norm="ortho")            # (N, d, n, n)
    Ablk = K[None, None] + tau * lam[:, :, None, None] * Mh[None, None]
    xh = np.linalg.solve(Ablk[None], np.moveaxis(rh, 1, -1)[..., None])[..., 0]
    return idstn(np.moveaxis(xh, -1, 1), type=1, axes=(-2, -1), norm="ortho")


def solve(p: int, tau: float, n: int, F, u0, *, tol: float = 1e-10, max_cycles: int = 100, **kw):
    """Time cycles from u = 0 until ||F - L u|| <= tol ||F||; returns (u, hist)."""
    Fhat = fold_u0(p, F, u0)
    u = np.zeros_like(Fhat)
    nF = np.linalg.norm(Fhat)
    hist = []
    for _ in range(max_cycles + 1):
        rel = np.linalg.norm(time_residual(p, tau, n, Fhat, u)) / nF
        hist.append(rel)
        if rel <= tol or len(hist) > max_cycles:
            break
        u = time_cycle(p, tau, n, Fhat, u, **kw)
    return u, np.array(hist)
