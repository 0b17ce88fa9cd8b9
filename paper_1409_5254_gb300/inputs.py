"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds no arithmetic of the solver: it draws random problem parameters and
assembles the *load vector* -- the right-hand side that the solver receives
-- by Gauss quadrature of a smooth forcing f(t) against the shifted Legendre
basis, f_n[l] = int_{t_{n-1}}^{t_n} f(t) psi_l^n(t) dt (Section 2, the
definition of the right-hand sides).  Neither the oracle nor the CUDA library
computes the load vector; both take it as input.

Recipes (seed = workload index unless stated):

* ``scalar_problem``      -- one u' + lambda u = f on (0, T): f is a sum of
  4 sinusoids, amplitudes U(-1, 1), integer frequencies U{1..8} scaled to T.
* ``heat_modes``          -- decoupled modes of a 2-D heat equation in mode
  space: lambda_ij = 5-point Laplacian eigenvalues of a 256 x 256 interior grid,
  f_k = (g_k / lambda_k) * (3-term sine series), g_k ~ N(0, 1).
* ``uneven_batch``        -- N log-uniform in [2^6, 2^16] rounded so that the
  coarsest level lands in (32, 64], p uniform in {0..3}, lambda*tau
  log-uniform in [1e-3, 1e3].
* ``random_guess``        -- U(0, 1) initial vectors (the measurement protocol of
  Section 4.2: zero right-hand side, random start).
* ``heat_problem``        -- the space-time heat equation on an n x n grid:
  f(t, x) = sum_{j<3} s_j(x) sin(2 pi m_j t / T), s_j(x) ~ U(-1, 1) per grid
  point, m_j ~ U{1..8}; u0(x) ~ U(-1, 1); tau = T / N.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["Forcing", "scalar_problem", "load_vector", "random_guess", "heat_modes",
           "uneven_batch", "adjoint_problem", "heat_problem"]


class Forcing:
    """f(t) = sum_i A_i sin(2 pi k_i t / T)."""

    def __init__(self, amps, freqs, T):
        self.amps = np.asarray(amps, dtype=np.float64)
        self.freqs = np.asarray(freqs, dtype=np.float64)
        self.T = float(T)

    @classmethod
    def draw(cls, rng: np.random.Generator, T: float, n_terms: int = 4, kmax: int = 8):
        amps = rng.uniform(-1.0, 1.0, n_terms)
        freqs = rng.integers(1, kmax + 1, n_terms)
        return cls(amps, freqs, T)

    def __call__(self, t):
        t = np.asarray(t, dtype=np.float64)
        out = np.zeros_like(t)
        for A, k in zip(self.amps, self.freqs):
            out += A * np.sin((2.0 * math.pi * k / self.T) * t)
        return out


def _legendre_table(p: int, s: np.ndarray) -> np.ndarray:
    """psi_l(s) = P_l(2 s - 1) for l = 0..p (numpy's Legendre evaluation)."""
    x = 2.0 * s - 1.0
    return np.stack([np.polynomial.legendre.legval(x, np.eye(p + 1)[l]) for l in range(p + 1)], axis=1)


def load_vector(p: int, N: int, T: float, f, q: int | None = None, chunk: int = 1 << 20,
                n_stop: int | None = None) -> np.ndarray:
    """Load vector (N, p+1) of forcing ``f`` on the uniform mesh t_n = n T / N
    (only the first n_stop intervals when given), by a q-point Gauss rule per
    interval: 8 points, or p + 2 where that is more, so that every
    coefficient of the load vector is an independent value."""
    if q is None:
        q = max(8, p + 2)
    tau = T / N
    xg, wg = np.polynomial.legendre.leggauss(q)
    s = 0.5 * (xg + 1.0)
    w = 0.5 * wg
    tab = _legendre_table(p, s) * w[:, None]          # (q, d)
    n_out = N if n_stop is None else min(N, n_stop)
    out = np.empty((n_out, p + 1), dtype=np.float64)
    for n0 in range(0, n_out, chunk):
        n1 = min(n_out, n0 + chunk)
        t = (np.arange(n0, n1, dtype=np.float64)[:, None] + s[None, :]) * tau
        out[n0:n1] = tau * (f(t) @ tab)
    return out


def scalar_problem(seed: int, N: int, p: int, lam: float = 1.0, T: float | None = None,
                   tau: float | None = None, u0: float = 1.0):
    """One DG-in-time problem u' + lam u = f, u(0) = u0, uniform steps.

    Give T (then tau = T / N) or tau (then T = N tau).  Returns a dict with the
    load vector ``F`` (N, p+1) and the scalars.
    """
    if (T is None) == (tau is None):
        raise ValueError("give exactly one of T, tau")
    if T is None:
        T = N * tau
    tau = T / N
    rng = np.random.default_rng(seed)
    forcing = Forcing.draw(rng, T)
    F = load_vector(p, N, T, forcing)
    return {"p": p, "N": N, "lam": float(lam), "tau": tau, "T": T, "u0": float(u0), "F": F,
            "forcing": forcing}


def random_guess(seed: int, N: int, d: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, (N, d))


def heat_modes(n_grid: int = 256):
    """Eigenvalues of the 5-point Dirichlet Laplacian on an n x n interior grid, h = 1/(n+1)."""
    h = 1.0 / (n_grid + 1)
    i = np.arange(1, n_grid + 1, dtype=np.float64)
    s = np.sin(i * math.pi * h / 2.0) ** 2
    lam = (4.0 / h**2) * (s[:, None] + s[None, :])
    return lam.reshape(-1)


def heat_mode_forcing(seed: int, lam: np.ndarray, N: int, p: int, T: float = 1.0,
                      q: int = 8) -> np.ndarray:
    """Load vectors (n_modes, N, p+1) for f_k(t) = (g_k/lam_k) sum_j s_kj sin(2 pi m_kj t)."""
    rng = np.random.default_rng(seed)
    n = lam.shape[0]
    g = rng.standard_normal(n)
    s = rng.uniform(-1.0, 1.0, (n, 3))
    m = rng.integers(1, 9, (n, 3)).astype(np.float64)
    tau = T / N
    xg, wg = np.polynomial.legendre.leggauss(q)
    sq = 0.5 * (xg + 1.0)
    tab = _legendre_table(p, sq) * (0.5 * wg)[:, None]      # (q, d)
    t = (np.arange(N, dtype=np.float64)[:, None] + sq[None, :]) * tau   # (N, q)
    out = np.empty((n, N, p + 1), dtype=np.float64)
    for j0 in range(0, n, 256):
        j1 = min(n, j0 + 256)
        ft = np.zeros((j1 - j0, N, q))
        for term in range(3):
            ft += s[j0:j1, term, None, None] * np.sin(2.0 * math.pi * m[j0:j1, term, None, None] * t[None])
        ft *= (g[j0:j1] / lam[j0:j1])[:, None, None]
        out[j0:j1] = tau * (ft @ tab)
    return out


def uneven_batch(seed: int, n_inst: int, nmin_exp: float = 6.0, nmax_exp: float = 16.0):
    """Instance parameters for an uneven batch: (N, p, z = lam*tau) per instance."""
    rng = np.random.default_rng(seed)
    n_raw = np.round(2.0 ** rng.uniform(nmin_exp, nmax_exp, n_inst)).astype(np.int64)
    shift = np.maximum(0, np.ceil(np.log2(n_raw)).astype(np.int64) - 6)
    N = ((n_raw + (1 << shift) - 1) >> shift) << shift
    p = rng.integers(0, 4, n_inst)
    z = 10.0 ** rng.uniform(-3.0, 3.0, n_inst)
    return N, p, z


def adjoint_problem(seed: int, n_inst: int, N: int, p: int = 2, T: float = 1.0):
    """lambda log-uniform in [1, 1e4], u0 ~ N(0,1), nodal targets ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    lam = 10.0 ** rng.uniform(0.0, 4.0, n_inst)
    u0 = rng.standard_normal(n_inst)
    target = rng.standard_normal((n_inst, N))
    return lam, u0, target


# ------------------------------------------------- large batched workloads --
#
# The batched workloads need billions of forcing evaluations, so their load
# vectors are assembled with torch (on the GPU when given a CUDA device); the
# random draws stay in numpy so every side sees the same parameters.

def sine_load_vectors(amps, freqs, T, N: int, p: int, device="cpu", q: int = 8, chunk: int = 1024):
    """Load vectors (n, N, p+1) of f_i(t) = sum_j amps[i, j] sin(2 pi freqs[i, j] t / T)
    for n instances on the same mesh t_n = n T / N (float64)."""
    import torch
    amps = torch.as_tensor(np.asarray(amps, dtype=np.float64), device=device)
    freqs = torch.as_tensor(np.asarray(freqs, dtype=np.float64), device=device)
    n = amps.shape[0]
    tau = T / N
    xg, wg = np.polynomial.legendre.leggauss(q)
    s = 0.5 * (xg + 1.0)
    tab = torch.as_tensor(_legendre_table(p, s) * (0.5 * wg)[:, None], device=device)       # (q, d)
    t = (torch.arange(N, dtype=torch.float64, device=device)[:, None]
         + torch.as_tensor(s, device=device)[None, :]) * tau                                 # (N, q)
    out = torch.empty((n, N, p + 1), dtype=torch.float64, device=device)
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        ft = torch.zeros((i1 - i0, N, q), dtype=torch.float64, device=device)
        for j in range(amps.shape[1]):
            om = (2.0 * math.pi / T) * freqs[i0:i1, j]
            ft += amps[i0:i1, j, None, None] * torch.sin(om[:, None, None] * t[None])
        out[i0:i1] = tau * (ft @ tab)
    return out


def heat_modes_batch(seed: int = 2, n_grid: int = 256, N: int = 4096, p: int = 1, T: float = 1.0):
    """Decoupled modes of a 2-D heat equation: lambda_k = 5-point Laplacian
    eigenvalues of an n_grid^2 interior grid; f_k = (g_k / lambda_k) *
    sum_{j<3} s_kj sin(2 pi m_kj t), g ~ N(0,1), s ~ U(-1,1), m ~ U{1..8}.
    Returns (lam, amps, freqs) for sine_load_vectors."""
    lam = heat_modes(n_grid)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(lam.shape[0])
    s = rng.uniform(-1.0, 1.0, (lam.shape[0], 3))
    m = rng.integers(1, 9, (lam.shape[0], 3)).astype(np.float64)
    return lam, (g / lam)[:, None] * s, m


def sinusoid_batch_params(seed: int, n: int, n_terms: int = 4):
    """Per-instance sinusoid forcings as in the single-problem recipe."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (n, n_terms)), rng.integers(1, 9, (n, n_terms)).astype(np.float64)


def heat_problem(seed: int, N: int, p: int, n: int, T: float = 1.0, q: int = 8):
    """(tau, F, u0): load vectors F of shape (N, p+1, n, n) and u0 of shape (n, n)."""
    rng = np.random.default_rng(seed)
    sx = rng.uniform(-1.0, 1.0, (3, n, n))
    m = rng.integers(1, 9, 3).astype(np.float64)
    u0 = rng.uniform(-1.0, 1.0, (n, n))
    tau = T / N
    xg, wg = np.polynomial.legendre.leggauss(q)
    sq = 0.5 * (xg + 1.0)
    tab = _legendre_table(p, sq) * (0.5 * wg)[:, None]      # (q, d)
    t = (np.arange(N, dtype=np.float64)[:, None] + sq[None, :]) * tau   # (N, q)
    F = np.zeros((N, p + 1, n, n))
    for j in range(3):
        lt = tau * (np.sin(2.0 * math.pi * m[j] / T * t) @ tab)       # (N, d)
        F += lt[:, :, None, None] * sx[j][None, None]
    return tau, F, u0
