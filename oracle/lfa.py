"""Local Fourier (mode) analysis of Section 4 -- TEST INFRASTRUCTURE ONLY.

Builds the Fourier symbols of the paper and the two-grid iteration matrix
M(theta) of Theorem chap4_theorem4, then the asymptotic convergence factor
rho(M_tau) = max over low frequencies of the spectral radius of M(theta)
(definition after Theorem chap4_theorem4).  numpy's eigvals serves as the
eigenvalue routine.

Symbols (z = lambda * tau_L on the fine level, 2z on the coarse level):
  L(theta)  = A(z) - e^{-i theta} N                           (Lemma chap4_lemma3)
  S(theta)  = (1 - w) I + e^{-i theta} w A(z)^{-1} N          (Lemma chap4_lemma3a)
  R(theta)  = e^{-i theta} R1 + R2                            (Lemma chap4_lemma12)
  P(theta)  = 1/2 (e^{i theta} R1^T + R2^T)                   (Lemma chap4_lemma13)
  M(theta)  = diag(S^nu2(t), S^nu2(g t)) K(t) diag(S^nu1(t), S^nu1(g t))
  K(theta)  = I - [P(t); P(g t)] L_2(2t)^{-1} [R(t), R(g t)] diag(L(t), L(g t))
with g t = theta - sign(theta) pi (Lemma chap4_lemma9).  Reading: for theta =
0 the partner frequency is pi; every symbol only sees e^{-i g t} = -e^{-i t},
so the sign convention does not matter.
"""
from __future__ import annotations

import numpy as np

from . import blocks, transfer, alpha, omega_star


def _A(p, z):
    K, M, a, b = blocks(p)
    return K + z * M, np.outer(a, b)


def symbols(p: int, z: float, omega: float):
    """Callables (L, S, R, P, L2) of theta for the fine step z."""
    A, N = _A(p, z)
    A2, _ = _A(p, 2.0 * z)
    Ainv_N = np.linalg.solve(A, N)
    P1, P2 = transfer(p)
    R1, R2 = P1.T, P2.T
    d = p + 1
    I = np.eye(d)

    def L(t):
        return A - np.exp(-1j * t) * N

    def L2(t):
        return A2 - np.exp(-1j * t) * N

    def S(t):
        return (1.0 - omega) * I + np.exp(-1j * t) * omega * Ainv_N

    def R(t):
        return np.exp(-1j * t) * R1 + R2

    def P(t):
        return 0.5 * (np.exp(1j * t) * P1 + P2)

    return L, S, R, P, L2


def two_grid_symbol(p: int, z: float, theta: float, nu1: int = 1, nu2: int = 1,
                    omega: float | None = None) -> np.ndarray:
    """The 2d x 2d matrix M(theta) of Theorem chap4_theorem4."""
    w = omega_star(p, z) if omega is None else omega
    L, S, R, P, L2 = symbols(p, z, w)
    d = p + 1
    tg = theta - np.pi if theta > 0 else theta + np.pi
    Z = np.zeros((d, d))
    blkL = np.block([[L(theta), Z], [Z, L(tg)]])
    Pc = np.vstack([P(theta), P(tg)])
    Rr = np.hstack([R(theta), R(tg)])
    Kc = np.eye(2 * d) - Pc @ np.linalg.solve(L2(2.0 * theta), Rr @ blkL)
    S1 = np.block([[np.linalg.matrix_power(S(theta), nu1), Z], [Z, np.linalg.matrix_power(S(tg), nu1)]])
    S2 = np.block([[np.linalg.matrix_power(S(theta), nu2), Z], [Z, np.linalg.matrix_power(S(tg), nu2)]])
    return S2 @ Kc @ S1


def low_frequencies(N_L: int) -> np.ndarray:
    """Theta_L^low = {2 k pi / N_L} cap (-pi/2, pi/2] (Definition of Fourier frequencies)."""
    k = np.arange(1 - N_L // 2, N_L // 2 + 1)
    th = 2.0 * np.pi * k / N_L
    return th[(th > -np.pi / 2) & (th <= np.pi / 2)]


def two_grid_factor(p: int, z: float, nu1: int = 1, nu2: int = 1, omega: float | None = None,
                    N_L: int = 1024, return_theta: bool = False):
    """rho(M_tau) = max over Theta_low of the spectral radius of M(theta)."""
    best, arg = -1.0, None
    for th in low_frequencies(N_L):
        r = np.max(np.abs(np.linalg.eigvals(two_grid_symbol(p, z, th, nu1, nu2, omega))))
        if r > best:
            best, arg = r, th
    return (best, arg) if return_theta else best


def smoother_radius(p: int, z: float, theta: float, omega: float) -> float:
    """Spectral radius of S(theta) (Lemma chap4_lemma4 gives it in closed form)."""
    _, S, _, _, _ = symbols(p, z, omega)
    return float(np.max(np.abs(np.linalg.eigvals(S(theta)))))


def smoothing_factor(p: int, z: float, omega: float | None = None, N_L: int = 1024) -> float:
    """mu_S = max over high frequencies of rho(S(theta)) (Definition of mu_S)."""
    w = omega_star(p, z) if omega is None else omega
    k = np.arange(1 - N_L // 2, N_L // 2 + 1)
    th = 2.0 * np.pi * k / N_L
    high = th[(th <= -np.pi / 2) | (th > np.pi / 2)]
    return max(smoother_radius(p, z, t, w) for t in high)


def s_hat(omega: float, a: float, theta: float) -> float:
    """S_hat of Lemma chap4_lemma4: |1 - w + e^{-i theta} w alpha|."""
    return abs(1.0 - omega + np.exp(-1j * theta) * omega * a)


def periodic_two_grid_matrix(p: int, z: float, N: int, nu1: int = 1, nu2: int = 1,
                             omega: float | None = None) -> np.ndarray:
    """Dense two-grid error propagator for the time-periodic system (eq.
    chap4_equationLinearSystemODEPeriodic) with the circulant U_N, for which
    the Fourier analysis is exact."""
    w = omega_star(p, z) if omega is None else omega
    d = p + 1
    A, Nb = _A(p, z)
    A2, _ = _A(p, 2.0 * z)

    def periodic_L(Ablk, n):
        L = np.zeros((n * d, n * d))
        for i in range(n):
            L[i * d:(i + 1) * d, i * d:(i + 1) * d] = Ablk
            j = (i - 1) % n
            L[i * d:(i + 1) * d, j * d:(j + 1) * d] -= Nb
        return L

    Lf = periodic_L(A, N)
    Lc = periodic_L(A2, N // 2)
    Dinv = np.kron(np.eye(N), np.linalg.inv(A))
    S = np.eye(N * d) - w * Dinv @ Lf
    P1, P2 = transfer(p)
    R = np.zeros((N // 2 * d, N * d))
    for m in range(N // 2):
        R[m * d:(m + 1) * d, (2 * m) * d:(2 * m + 1) * d] = P1.T
        R[m * d:(m + 1) * d, (2 * m + 1) * d:(2 * m + 2) * d] = P2.T
    P = R.T
    CG = np.eye(N * d) - P @ np.linalg.solve(Lc, R @ Lf)
    return np.linalg.matrix_power(S, nu2) @ CG @ np.linalg.matrix_power(S, nu1)


__all__ = ["symbols", "two_grid_symbol", "low_frequencies", "two_grid_factor", "smoother_radius",
           "smoothing_factor", "s_hat", "periodic_two_grid_matrix", "alpha", "omega_star"]
