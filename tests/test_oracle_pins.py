"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: a
closed form printed in the paper, a textbook identity, a brute-force solve, an
independent Runge-Kutta method, or a property the paper proves.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lfa
from paper_1409_5254_gb300 import inputs
from conftest import load_golden

PS = [0, 1, 2, 3, 4, 5]
# the higher degrees of the p_t study (p_t = 10, 20) beside the paper's 0..5
PS_WIDE = PS + [10, 20]


def pade(p, z):
    """P_{p,p+1}(z) from the golden fixture (the paper's list, Section 2)."""
    for row in load_golden("pade_subdiagonal.txt"):
        if int(row[0][0]) == p:
            num = sum(c * z**i for i, c in enumerate(row[1]))
            den = sum(c * z**i for i, c in enumerate(row[2]))
            return num / den
    raise KeyError(p)


def pade_closed_form(m, n, z):
    """The [m/n] Pade approximant of exp(z) from its classical closed form
    (numerator sum_j (m+n-j)! m! / ((m+n)! j! (m-j)!) z^j, denominator the same
    with n and -z), independent of the paper's printed list and of the oracle."""
    from math import factorial as fa
    num = sum(fa(m + n - j) * fa(m) / (fa(m + n) * fa(j) * fa(m - j)) * z**j for j in range(m + 1))
    den = sum(fa(m + n - j) * fa(n) / (fa(m + n) * fa(j) * fa(n - j)) * (-z) ** j for j in range(n + 1))
    return num / den


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_pade_closed_form_reproduces_the_papers_list(p):
    for z in (-3.0, -0.5, 0.25, 2.0):
        assert pade_closed_form(p, p + 1, z) == pytest.approx(pade(p, z), rel=1e-14)


@pytest.mark.parametrize("p", [4, 5])
@pytest.mark.parametrize("z", [1e-3, 0.5, 2.0, 40.0])
def test_homogeneous_nodal_values_higher_degrees(p, z):
    """Degrees beyond the paper's printed list: with f = 0 the nodal values
    follow R(-z)^n with R the (p, p+1) sub-diagonal Pade approximant
    (Corollary chap4_corollary1) from its closed form."""
    N = 60
    u = O.fsub(p, z, np.zeros((N, p + 1)), 1.0)
    e = O.nodal_values(p, u)
    R = pade_closed_form(p, p + 1, -z)
    np.testing.assert_allclose(e, R ** np.arange(1, N + 1), rtol=1e-10, atol=1e-300)
    assert O.alpha(p, z) == pytest.approx(R, rel=1e-12, abs=1e-15)



def pade_exact(m, n, z):
    """The same closed form evaluated in exact rational arithmetic (z is a
    float, so exactly representable): at p = 20 the alternating sums lose
    every digit in double."""
    from fractions import Fraction
    from math import factorial as fa
    z = Fraction(z)
    num = sum(Fraction(fa(m + n - j) * fa(m), fa(m + n) * fa(j) * fa(m - j)) * z**j for j in range(m + 1))
    den = sum(Fraction(fa(m + n - j) * fa(n), fa(m + n) * fa(j) * fa(n - j)) * (-z) ** j
              for j in range(n + 1))
    return float(num / den)


@pytest.mark.parametrize("p", [10, 20])
@pytest.mark.parametrize("z", [1e-3, 0.5, 2.0, 40.0, 1e3])
def test_homogeneous_nodal_values_degrees_10_and_20(p, z):
    """With f = 0 the nodal values are R(-z)^n u0 (Corollary chap4_corollary1)
    with R the (p, p+1) sub-diagonal Pade approximant, here at p_t = 10 and 20.
    alpha is a difference of O(1) terms, so its error is absolute (~1e-16):
    at p = 20, z = 40 the value itself is 5.5e-10."""
    N = 40
    u = O.fsub(p, z, np.zeros((N, p + 1)), 1.0)
    e = O.nodal_values(p, u)
    R = pade_exact(p, p + 1, -z)
    n = np.arange(1, N + 1)
    assert np.all(np.abs(e - R ** n) <= 1e-12 * np.abs(R) ** n + 1e-14 * n)
    assert O.alpha(p, z) == pytest.approx(R, rel=1e-12, abs=1e-15)


def polynomial_case(p, lam=1.3, T=1.0, N=16, seed=0):
    """A problem whose exact solution q is a polynomial of degree p on (0, T):
    f = q' + lam q, u0 = q(0).  Returns (z, F, u0, U) with F[n,k] = tau
    int_0^1 f(t_n + tau s) psi_k(s) ds and U[n] the shifted-Legendre
    coefficients of q on interval n, both by a (p+12)-point Gauss rule with
    numpy's Legendre routines."""
    Lg = np.polynomial.legendre
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(p + 1)                       # q(t) = sum_j c_j P_j(2t/T - 1)
    dc = Lg.legder(c) * (2.0 / T)
    q = lambda t: Lg.legval(2.0 * t / T - 1.0, c)              # noqa: E731
    dq = lambda t: Lg.legval(2.0 * t / T - 1.0, dc) if p else 0.0 * t   # noqa: E731
    xg, wg = Lg.leggauss(p + 12)
    s, w = 0.5 * (xg + 1.0), 0.5 * wg
    psi = np.stack([Lg.legval(2.0 * s - 1.0, np.eye(p + 1)[k]) for k in range(p + 1)])
    tau = T / N
    F, U = np.zeros((N, p + 1)), np.zeros((N, p + 1))
    for n in range(N):
        t = n * tau + tau * s
        F[n] = tau * (psi * (w * (dq(t) + lam * q(t)))).sum(axis=1)
        U[n] = (psi * (w * q(t))).sum(axis=1) * (2.0 * np.arange(p + 1) + 1.0)
    return lam * tau, F, float(q(0.0)), U


@pytest.mark.parametrize("p", PS_WIDE)
def test_dg_reproduces_polynomial_solutions(p):
    """Galerkin consistency of the variational form eq. chap4_discreteVarFormODE:
    an exact solution inside the trial space (a polynomial of degree p, continuous,
    so every upwind jump vanishes) satisfies the discrete equations, and the
    block system returns its coefficients on every interval."""
    z, F, u0, U = polynomial_case(p)
    u = O.fsub(p, z, F, u0)
    assert np.abs(u - U).max() <= 1e-13 * np.abs(U).max()
    # the multigrid solve reaches the same coefficients
    um, hist = O.mg_solve(p, z, F, u0, n_min=2, tol=1e-14, max_cycles=100)
    assert np.abs(um - U).max() <= 1e-12 * np.abs(U).max()

# --------------------------------------------------------------- blocks --

@pytest.mark.parametrize("p", PS_WIDE)
def test_blocks_match_legendre_identities(p):
    """K, Mhat, a, b against Legendre identities: P_k(1) = 1, P_k(-1) = (-1)^k,
    int_{-1}^{1} P_k P_l = 2/(2k+1) delta_kl, and P_k' = sum_{j<k, k-j odd} (2j+1) P_j,
    which give K[k,l] = 1 - 2 [l < k and k+l odd], Mhat = diag(1/(2k+1))."""
    K, M, a, b = O.blocks(p)
    d = p + 1
    Kx = np.array([[1.0 - 2.0 * (l < k and (k + l) % 2 == 1) for l in range(d)] for k in range(d)])
    np.testing.assert_allclose(K, Kx, atol=1e-14)
    np.testing.assert_allclose(M, np.diag([1.0 / (2 * k + 1) for k in range(d)]), atol=1e-14)
    np.testing.assert_allclose(a, [(-1.0) ** k for k in range(d)], atol=1e-15)
    np.testing.assert_allclose(b, np.ones(d), atol=1e-15)


@pytest.mark.parametrize("p", PS_WIDE)
def test_prolongation_is_exact_injection(p):
    """P1, P2 carry a coarse polynomial onto each half exactly (L2 projection of a
    polynomial of the same degree): check pointwise with numpy's Legendre evaluation."""
    P1, P2 = O.transfer(p)
    rng = np.random.default_rng(p)
    d = p + 1
    uc = rng.standard_normal(d)
    s = np.linspace(0.0, 1.0, 11)
    leg = np.polynomial.legendre.legval
    coarse_first = leg(2.0 * (0.5 * s) - 1.0, uc)
    coarse_second = leg(2.0 * (0.5 * (s + 1.0)) - 1.0, uc)
    np.testing.assert_allclose(leg(2.0 * s - 1.0, P1 @ uc), coarse_first, atol=1e-14)
    np.testing.assert_allclose(leg(2.0 * s - 1.0, P2 @ uc), coarse_second, atol=1e-14)


def dense_L(p, z, N):
    K, M, a, b = O.blocks(p)
    d = p + 1
    A = K + z * M
    L = np.zeros((N * d, N * d))
    for n in range(N):
        L[n * d:(n + 1) * d, n * d:(n + 1) * d] = A
        if n:
            L[n * d:(n + 1) * d, (n - 1) * d:n * d] = -np.outer(a, b)
    return L


@pytest.mark.parametrize("p", PS_WIDE)
@pytest.mark.parametrize("z", [1e-3, 0.7, 50.0])
def test_galerkin_coarse_operator_equals_rediscretisation(p, z):
    """R L_tau P = L_{2tau}: with exact injection and the upwind DG form the
    midpoint jump terms cancel, so the Galerkin coarse operator is the
    re-discretised one (the operator the two-grid cycle of eq.
    chap4_errorTwoGridCycle inverts)."""
    N = 8
    d = p + 1
    P1, P2 = O.transfer(p)
    R = np.zeros((N // 2 * d, N * d))
    for m in range(N // 2):
        R[m * d:(m + 1) * d, 2 * m * d:(2 * m + 1) * d] = P1.T
        R[m * d:(m + 1) * d, (2 * m + 1) * d:(2 * m + 2) * d] = P2.T
    np.testing.assert_allclose(R @ dense_L(p, z, N) @ R.T, dense_L(p, 2 * z, N // 2), atol=1e-12)


# --------------------------------------------------------- exact solves --

@pytest.mark.parametrize("z", [1e-3, 0.25, 3.0, 1e3])
def test_p0_is_backward_euler(z):
    """p_t = 0 gives backward Euler (end of Section 2 "Linear system"):
    (1 + z) u_n = u_{n-1} + int f; with f = 0, u_n = u0 (1+z)^{-n} exactly."""
    N = 200
    u = O.fsub(0, z, np.zeros((N, 1)), 1.5)
    n = np.arange(1, N + 1)
    np.testing.assert_allclose(u[:, 0], 1.5 * (1.0 + z) ** (-n.astype(float)), rtol=1e-13, atol=1e-290)
    F = np.random.default_rng(3).standard_normal((N, 1))
    u = O.fsub(0, z, F, 0.3)
    prev = np.concatenate([[0.3], u[:-1, 0]])
    np.testing.assert_allclose((1.0 + z) * u[:, 0], prev + F[:, 0], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("z", [1e-3, 0.5, 2.0, 40.0])
def test_homogeneous_nodal_values_follow_pade(p, z):
    """With f = 0 the nodal values are e_n = R(-z)^n u0 with R the (p, p+1)
    sub-diagonal Pade approximant (Corollary chap4_corollary1, Lemma
    chap4_theorem2 eq. chap4_theorem2_equ2); the Pade forms are the paper's."""
    N = 60
    u = O.fsub(p, z, np.zeros((N, p + 1)), 1.0)
    e = O.nodal_values(p, u)
    R = pade(p, -z)
    np.testing.assert_allclose(e, R ** np.arange(1, N + 1), rtol=1e-11, atol=1e-300)
    assert O.alpha(p, z) == pytest.approx(R, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("p", PS_WIDE)
@pytest.mark.parametrize("z", [1e-3, 1.0, 1e3])
def test_fsub_matches_dense_brute_force(p, z):
    for N in (1, 2, 5, 64):
        F = np.random.default_rng(N + 10 * p).standard_normal((N, p + 1))
        u_d = O.dense_solve(p, z, F, 0.7)
        u_f = O.fsub(p, z, F, 0.7)
        scale = np.abs(u_d).max()
        assert np.abs(u_f - u_d).max() <= 1e-12 * scale


def radau_ia_tableau(s):
    """s-stage Radau IA from its defining conditions: left Radau nodes (zeros of
    P_{s-1}(x) + P_s(x), x = 2c-1, which include c = 0), weights from
    quadrature exactness B(s), and A from the conditions D(s):
    sum_i b_i c_i^{k-1} a_ij = b_j (1 - c_j^k) / k, k = 1..s."""
    coef = np.zeros(s + 1)
    coef[s - 1] += 1.0
    coef[s] += 1.0
    x = np.sort(np.real(np.polynomial.legendre.legroots(coef)))
    c = 0.5 * (x + 1.0)
    c[0] = 0.0
    V = np.vander(c, s, increasing=True).T                    # V[k, j] = c_j^k
    b = np.linalg.solve(V, 1.0 / np.arange(1, s + 1))
    A = np.zeros((s, s))
    W = V * b[None, :]                                         # W[k, i] = b_i c_i^k
    for j in range(s):
        rhs = b[j] * (1.0 - c[j] ** np.arange(1, s + 1)) / np.arange(1, s + 1)
        A[:, j] = np.linalg.solve(W, rhs)
    return c, b, A


@pytest.mark.parametrize("p", PS)
def test_dg_with_radau_rhs_equals_radau_ia(p):
    """Theorem chap4_theorem1a: with the right-hand side integrated by the Radau
    rule of order 2p+1 the DG scheme is the (p+1)-stage Radau IA method."""
    s = p + 1
    c, bw, A = radau_ia_tableau(s)
    lam, T, N, u0 = 1.3, 1.0, 40, 0.8
    tau = T / N
    f = lambda t: np.cos(3.0 * t) + t**2
    leg = np.polynomial.legendre.legval
    psi_at_c = np.stack([leg(2.0 * c - 1.0, np.eye(s)[l]) for l in range(s)], axis=1)  # (stage, l)
    F = np.zeros((N, s))
    for n in range(N):
        fc = f(n * tau + c * tau)
        F[n] = tau * (bw * fc) @ psi_at_c
    e = O.nodal_values(p, O.fsub(p, lam * tau, F, u0))
    u = u0
    rk = []
    for n in range(N):
        tj = n * tau + c * tau
        # stages U = u + tau A (f(t) - lam U)
        U = np.linalg.solve(np.eye(s) + tau * lam * A, u + tau * A @ f(tj))
        u = u + tau * bw @ (f(tj) - lam * U)
        rk.append(u)
    np.testing.assert_allclose(e, rk, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------- multigrid --

@pytest.mark.parametrize("p", PS_WIDE)
@pytest.mark.parametrize("gamma", [1, 2])
def test_mg_converges_to_forward_substitution(p, gamma):
    prob = inputs.scalar_problem(0, 256, p, lam=2.0, T=1.0, u0=1.0)
    z = prob["lam"] * prob["tau"]
    u_ex = O.fsub(p, z, prob["F"], prob["u0"])
    u, hist = O.mg_solve(p, z, prob["F"], prob["u0"], n_min=4, gamma=gamma, tol=1e-13, max_cycles=200)
    assert hist[-1] <= 1e-13
    assert np.abs(u - u_ex).max() <= 1e-11 * np.abs(u_ex).max()


def _p0_cycle_extended(z, F, u, n_min, nu1, nu2):
    """One V-cycle of the p_t = 0 system (backward Euler: (1+z_l) u_n - u_{n-1}
    = f_n on level l, z_l = z 2^l), written independently of the oracle in
    extended precision (numpy longdouble): damped Jacobi with
    omega* = 1/(1 + alpha^2), alpha = 1/(1+z_l); restriction by pair sums
    (R = P^T with P piecewise-constant injection); exact coarsest solve."""
    LD = np.longdouble
    z = LD(z)

    def Lu(u, zl):
        return (1 + zl) * u - np.concatenate([[LD(0)], u[:-1]])

    def smooth(u, f, zl, nu):
        om = LD(1) / (LD(1) + (LD(1) / (LD(1) + zl)) ** 2)
        for _ in range(nu):
            u = (1 - om) * u + om * (f + np.concatenate([[LD(0)], u[:-1]])) / (1 + zl)
        return u

    def cycle(l, f, u):
        zl = z * LD(2) ** l
        if len(f) % 2 or len(f) <= n_min:
            e, out = LD(0), np.empty_like(f)
            for n in range(len(f)):
                e = (f[n] + e) / (1 + zl)
                out[n] = e
            return out
        u = smooth(u, f, zl, nu1)
        r = f - Lu(u, zl)
        uc = cycle(l + 1, r[0::2] + r[1::2], np.zeros(len(f) // 2, dtype=LD))
        u = u.copy()
        u[0::2] += uc
        u[1::2] += uc
        return smooth(u, f, zl, nu2)

    return cycle(0, F.astype(LD), u.astype(LD))


@pytest.mark.skipif(np.finfo(np.longdouble).eps >= 1e-18, reason="needs an extended long double")
@pytest.mark.parametrize("N,nu", [(1 << 12, (1, 1)), (1 << 13, (2, 2)), (3 << 10, (1, 1))])
def test_mg_cycle_rounding_against_extended_precision(N, nu):
    """The FP64 textbook cycle against the same cycle in extended precision
    (p_t = 0, written apart from the oracle): two cycles agree to 1e-13 on
    hierarchies of up to ten levels, the regime of the FP64 parity tests'
    1e-12 bar.  (On deep hierarchies the oracle's A (omega A^{-1} f) carries
    one rounding of 1/(1+z) into every interval alike; restriction adds those
    up coherently, and at 13 levels the FP64 oracle is 5e-12 from the
    extended value while the kernels' tracked A u stay at 3e-15.)"""
    prob = inputs.scalar_problem(5, N, 0, lam=1.0, T=1.0, u0=0.5)
    z = prob["tau"]
    Fhat = O.fold_u0(0, prob["F"], prob["u0"])
    u64 = np.zeros_like(Fhat)
    uex = np.zeros(N, dtype=np.longdouble)
    for k in range(2):
        u64 = O.mg_one_cycle(0, z, Fhat, u64, n_min=64, nu1=nu[0], nu2=nu[1])
        uex = _p0_cycle_extended(z, Fhat[:, 0], uex, 64, nu[0], nu[1])
        err = np.abs(u64[:, 0] - uex.astype(np.float64)).max() / np.abs(uex).max()
        assert err <= 1e-13, (k, float(err))


def test_mg_levels_one_is_exact_solve():
    """With a single level the cycle is the exact coarsest solve."""
    prob = inputs.scalar_problem(1, 64, 2, lam=1.0, T=1.0, u0=0.5)
    u, hist = O.mg_solve(2, prob["tau"], prob["F"], prob["u0"], max_levels=1, tol=1e-14)
    assert len(hist) <= 3 and hist[-1] <= 1e-14


# ------------------------------------------------------- Fourier analysis --

@pytest.mark.parametrize("z", [1e-4, 1e-2, 0.1, 1.0, 10.0])
def test_lfa_p0_closed_form(z):
    """Section 4.2: for p_t = 0, nu1 = nu2 = 1 and omega*, rho = 1/(2 + 2 tau + tau^2),
    attained at theta* = pi/2 (tau read as z = lambda tau)."""
    rho, th = lfa.two_grid_factor(0, z, N_L=512, return_theta=True)
    assert rho == pytest.approx(1.0 / (2.0 + 2.0 * z + z * z), rel=1e-12)
    assert th == pytest.approx(np.pi / 2)


@pytest.mark.parametrize("p", PS_WIDE)
@pytest.mark.parametrize("z", [0.05, 0.6, 5.0])
def test_lfa_equals_periodic_two_grid(p, z):
    """The Fourier analysis is exact for the time-periodic system
    (eq. chap4_equationLinearSystemODEPeriodic): compare with the dense
    two-grid propagator built from its definition."""
    N = 16
    rho_dense = np.max(np.abs(np.linalg.eigvals(lfa.periodic_two_grid_matrix(p, z, N))))
    assert lfa.two_grid_factor(p, z, N_L=N) == pytest.approx(rho_dense, rel=1e-9, abs=1e-12)


def test_lfa_claims_of_section_4():
    """p >= 1 factors are about half the p = 0 factor at small steps; the factor
    tends to 0 for large steps; at the zero of alpha for odd p (z = 3 for p = 1)
    two smoothing steps solve exactly."""
    r0 = lfa.two_grid_factor(0, 1e-4, N_L=256)
    for p in (1, 2, 3):
        assert lfa.two_grid_factor(p, 1e-4, N_L=256) == pytest.approx(0.5 * r0, rel=0.02)
        assert lfa.two_grid_factor(p, 1e3, N_L=256) < 1e-3
    assert abs(O.alpha(1, 3.0)) < 1e-15
    # a defective (Jordan) eigenvalue at 0: rounding of size eps shows as ~sqrt(eps)
    assert lfa.two_grid_factor(1, 3.0, N_L=256) < 1e-6


@pytest.mark.parametrize("p", PS_WIDE)
def test_alpha_range_and_smoothing_bounds(p):
    """Lemma chap4_lemma7: (5 - 3 sqrt 3)/2 <= alpha <= 1 and mu_S <= 1/sqrt 2 with
    omega*; Lemma chap4_lemma8: max_theta S_hat <= |alpha| (1 + |alpha|) / (1 + alpha^2);
    Lemma chap4_lemma4: rho(S(theta)) = max(|1 - omega|, S_hat) (S_hat alone for p = 0)."""
    lo = (5.0 - 3.0 * math.sqrt(3.0)) / 2.0
    K, M, a, b = O.blocks(p)
    for z in np.logspace(-4, 4, 33):
        al = O.alpha(p, z)
        # eigenvalue rounding of the rank-one A^{-1}N: eps |S| times the condition
        # |A^{-1}a| |b| / |alpha| of its simple eigenvalue alpha (at p = 20 alpha
        # falls to ~1e-8 at large z)
        g = np.linalg.norm(np.linalg.solve(K + z * M, a)) * np.linalg.norm(b)
        tol = 1e-10 + 16 * np.finfo(float).eps * g * g / max(abs(al), 1e-300)
        assert lo - 1e-12 <= al <= 1.0
        w = O.omega_star(p, z)
        assert w == pytest.approx(1.0 / (1.0 + al * al) if al >= 0 else 1.0)
        assert lfa.smoothing_factor(p, z, N_L=64) <= 1.0 / math.sqrt(2.0) + 1e-12
        bound = abs(al) * (1 + abs(al)) / (1 + al * al)
        for th in np.linspace(-np.pi, np.pi, 13):
            assert lfa.s_hat(w, al, th) <= bound + 1e-12
            # the eigenvalue 1 - omega comes from the zero eigenvalue of A^{-1}N,
            # which exists only when N_t = p + 1 >= 2
            expect = max(abs(1 - w), lfa.s_hat(w, al, th)) if p >= 1 else lfa.s_hat(w, al, th)
            assert lfa.smoother_radius(p, z, th, w) == pytest.approx(expect, abs=tol)


@pytest.mark.parametrize("al", [-0.09, -0.03, 0.0, 0.2, 0.6, 0.95])
def test_omega_star_is_minimax(al):
    """Lemma chap4_lemma6 by brute force over omega in (0, 1] and theta in [pi/2, pi]."""
    ws = np.linspace(1e-3, 1.0, 2000)
    th = np.linspace(np.pi / 2, np.pi, 200)
    worst = np.array([max(lfa.s_hat(w, al, t) for t in th) for w in ws])
    w_star = 1.0 / (1.0 + al * al) if al >= 0 else 1.0
    best_val = al / math.sqrt(1 + al * al) if al >= 0 else abs(al)
    assert worst.min() == pytest.approx(best_val, abs=2e-3)
    assert max(lfa.s_hat(w_star, al, t) for t in th) == pytest.approx(best_val, abs=1e-12)


@pytest.mark.parametrize("p", [0, 1, 2, 3])
@pytest.mark.parametrize("z", [1e-4, 1e-2, 0.3, 1.0, 3.0, 30.0])
def test_measured_two_grid_factor_matches_lfa(p, z):
    """Protocol of Section 4.2: N_L = 1024, f = 0, random start in [0,1], two-grid
    cycles until 1e-140 reduction; the measured asymptotic ratio (geometric mean
    of the second half of ||r^{k+1}|| / ||r^k||) agrees with rho(M_tau), over
    the degrees and steps of the paper's plots.  At p = 1, z = 3 (the zero of
    alpha) two smoothing steps solve exactly: the LFA value is rounding
    (~sqrt(eps), a defective eigenvalue) and the measured one is below it."""
    N = 1024
    u_init = inputs.random_guess(7, N, p + 1)
    _, hist = O.mg_solve(p, z, np.zeros((N, p + 1)), 0.0, max_levels=2, tol=1e-140 * 0 + 0.0,
                         max_cycles=60, u_init=u_init)
    ratios = hist[1:] / hist[:-1]
    ratios = ratios[np.isfinite(ratios) & (hist[1:] > 1e-280)]
    half = ratios[len(ratios) // 2:]
    geo = float(np.exp(np.mean(np.log(half))))
    rho = lfa.two_grid_factor(p, z, N_L=N)
    if rho < 1e-6:
        assert geo <= 1e-6
    else:
        assert geo == pytest.approx(rho, rel=0.05)
    assert ratios.max() <= max(1.35 * rho, rho + 0.15)


# --------------------------------------------------------------- adjoint --

@pytest.mark.parametrize("p", [0, 1, 2])
def test_adjoint_sweep_matches_transposed_dense_solve(p):
    N, z = 24, 0.4
    g = np.random.default_rng(5).standard_normal((N, p + 1))
    mu = O.adj_sweep(p, z, g)
    mu_d = np.linalg.solve(dense_L(p, z, N).T, g.reshape(-1)).reshape(N, p + 1)
    np.testing.assert_allclose(mu, mu_d, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("p", [0, 2])
def test_adjoint_gradients_match_finite_differences(p):
    """J = 1/2 sum_n (e_n - y_n)^2 over nodal values; gradients from the adjoint
    against central differences of the forward substitution."""
    N, T = 32, 1.0
    tau = T / N
    rng = np.random.default_rng(11)
    F = rng.standard_normal((N, p + 1)) * tau
    y = rng.standard_normal(N)
    lam, u0 = 3.0, 0.4
    _, _, _, b = O.blocks(p)

    def J(F_, u0_, lam_):
        e = O.nodal_values(p, O.fsub(p, lam_ * tau, F_, u0_))
        return 0.5 * np.sum((e - y) ** 2)

    u = O.fsub(p, lam * tau, F, u0)
    g = np.outer(O.nodal_values(p, u) - y, b)
    dJdf, dJdu0, dJdlam = O.adjoint_grads(p, lam, tau, g, u)
    h = 1e-6
    assert dJdu0 == pytest.approx((J(F, u0 + h, lam) - J(F, u0 - h, lam)) / (2 * h), rel=1e-7)
    assert dJdlam == pytest.approx((J(F, u0, lam + h) - J(F, u0, lam - h)) / (2 * h), rel=1e-6)
    for (n, k) in [(0, 0), (5, p), (N - 1, 0)]:
        Fp, Fm = F.copy(), F.copy()
        Fp[n, k] += h
        Fm[n, k] -= h
        assert dJdf[n, k] == pytest.approx((J(Fp, u0, lam) - J(Fm, u0, lam)) / (2 * h), rel=1e-6, abs=1e-9)


def test_load_vector_p0_matches_exact_integral():
    """The generator's load vector for p = 0 is int f over each interval; for a
    sinusoid the antiderivative is known."""
    T, N = 2.0, 50
    fz = inputs.Forcing([0.7], [3], T)
    F = inputs.load_vector(0, N, T, fz)
    om = 2 * math.pi * 3 / T
    t = np.arange(N + 1) * T / N
    exact = 0.7 * (np.cos(om * t[:-1]) - np.cos(om * t[1:])) / om
    np.testing.assert_allclose(F[:, 0], exact, rtol=1e-12, atol=1e-15)
