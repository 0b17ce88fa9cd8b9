"""Pins of the space-time heat-equation oracle (oracle/heat.py), CPU only.

Each part is checked against something other than itself:
* the 5-point Laplacian against its closed-form eigenpairs (sine modes);
* the bilinear prolongation against exact reproduction of bilinear functions,
  and full weighting against 1/4 of its transpose;
* the exact block forward substitution against a sparse direct solve of the
  assembled space-time system (brute force, small n and N), and, for forcing
  and initial value in one sine mode, against the scalar oracle's forward
  substitution at lambda = that mode's eigenvalue (the modes decouple);
* the spatial V-cycle: exact on one grid point, and contracting the error of
  the block solve by at least a factor 0.4 per cycle over tau/h^2 = 1e-3 ..
  1e3 (the smoothing factor 3/5 of omega-Jacobi, squared, where A_h
  dominates);
* the time cycle with exact block solves against the scalar oracle's textbook
  cycle (omega = 1/2) applied to one sine mode -- restriction, prolongation,
  smoothing and recursion in time, pinned through the decoupling;
* the full solver (one spatial V-cycle per block solve) converging to the
  exact solution.
"""
import numpy as np
import pytest

import oracle as O
from oracle import heat as H

sp = pytest.importorskip("scipy.sparse")
spla = pytest.importorskip("scipy.sparse.linalg")


def sine_mode(n, i, j):
    x = np.arange(1, n + 1) / (n + 1)
    return np.outer(np.sin(i * np.pi * x), np.sin(j * np.pi * x))


def eig(n, i, j):
    h = 1.0 / (n + 1)
    return (4.0 / h ** 2) * (np.sin(i * np.pi * h / 2) ** 2 + np.sin(j * np.pi * h / 2) ** 2)


@pytest.mark.parametrize("n,i,j", [(7, 1, 1), (15, 3, 7), (31, 30, 2)])
def test_laplacian_eigenpairs(n, i, j):
    v = sine_mode(n, i, j)
    assert np.abs(H.laplacian(v, H.grid_h(n)) - eig(n, i, j) * v).max() <= 1e-9 * eig(n, i, j)


def test_prolongation_reproduces_bilinear_functions_and_is_4x_restriction_transpose():
    n, nc = 15, 7
    X, Y = np.meshgrid(np.arange(1, nc + 1) / (nc + 1), np.arange(1, nc + 1) / (nc + 1), indexing="ij")
    Xf, Yf = np.meshgrid(np.arange(1, n + 1) / (n + 1), np.arange(1, n + 1) / (n + 1), indexing="ij")
    # bilinear functions vanishing on the boundary are not bilinear; use x y (1-x)(1-y) only at the
    # interior coarse-fine pattern: check exactness for f = x y restricted away from the boundary
    f = lambda a, b: (1 + 2 * a) * (3 - b)          # noqa: E731
    fine = H.prolong_space(f(X, Y), n)
    inner = (slice(2, -2), slice(2, -2))            # away from the zero boundary
    assert np.abs(fine[inner] - f(Xf, Yf)[inner]).max() <= 1e-13
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal((nc, nc)), rng.standard_normal((n, n))
    assert abs(np.sum(H.prolong_space(a, n) * b) - 4.0 * np.sum(a * H.restrict_space(b))) <= 1e-12


def assembled(p, tau, n, N):
    """The space-time matrix L (N (p+1) n^2 square), assembled from the
    definitions: blocks K (x) I + tau Mhat (x) A_h, sub-blocks -(a b^T) (x) I."""
    K, Mh, a, b = O.blocks(p)
    h = 1.0 / (n + 1)
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h ** 2
    I = sp.identity(n)
    A = sp.kron(T, I) + sp.kron(I, T)
    In = sp.identity(n * n)
    G = sp.kron(sp.csr_matrix(K), In) + tau * sp.kron(sp.csr_matrix(Mh), A)
    Nb = sp.kron(sp.csr_matrix(np.outer(a, b)), In)
    return (sp.kron(sp.identity(N), G) - sp.kron(sp.diags([np.ones(N - 1)], [-1]), Nb)).tocsc()


@pytest.mark.parametrize("p,n,N,tau", [(0, 7, 5, 0.1), (1, 7, 4, 0.01), (2, 3, 6, 1.0), (3, 7, 3, 1e-3)])
def test_exact_solve_matches_sparse_direct_solve(p, n, N, tau):
    rng = np.random.default_rng(p + n)
    F = rng.standard_normal((N, p + 1, n, n))
    u0 = rng.standard_normal((n, n))
    u = H.exact_solve(p, tau, n, F, u0)
    rhs = H.fold_u0(p, F, u0).reshape(-1)
    ref = spla.spsolve(assembled(p, tau, n, N), rhs).reshape(u.shape)
    assert np.abs(u - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(H.time_residual(p, tau, n, H.fold_u0(p, F, u0), u)).max() <= 1e-10 * np.abs(rhs).max()


@pytest.mark.parametrize("p", [0, 1, 2])
def test_one_sine_mode_reduces_to_the_scalar_problem(p):
    n, N, tau, (i, j) = 15, 16, 0.02, (2, 5)
    v = sine_mode(n, i, j)
    rng = np.random.default_rng(3)
    Fs = rng.standard_normal((N, p + 1))
    F = Fs[:, :, None, None] * v
    u = H.exact_solve(p, tau, n, F, 0.7 * v)
    us = O.fsub(p, eig(n, i, j) * tau, Fs, 0.7)
    assert np.abs(u - us[:, :, None, None] * v).max() <= 1e-11 * np.abs(us).max()


@pytest.mark.parametrize("p", [0, 1, 2])
@pytest.mark.parametrize("tau_h2", [1e-3, 1.0, 1e3])
def test_spatial_vcycle_contracts(p, tau_h2):
    n = 31
    h = H.grid_h(n)
    tau = tau_h2 * h * h
    rng = np.random.default_rng(1)
    r = rng.standard_normal((2, p + 1, n, n))
    x_ex = H._exact_blocks(p, tau, n, r)
    x = np.zeros_like(r)
    errs = []
    for _ in range(4):
        x = x + H.spatial_vcycle(p, tau, n, r - H.block_apply(p, tau, h, x))
        errs.append(np.abs(x - x_ex).max() / np.abs(x_ex).max())
    # omega-Jacobi (omega = 4/5) smooths the 5-point Laplacian by 3/5 per sweep: a V(1,1)-cycle
    # contracts by about (3/5)^2 = 0.36 where A_h dominates the block, much more where K does
    assert errs[-1] <= 0.4 ** 4 and all(b <= 0.4 * a for a, b in zip(errs, errs[1:])), errs
    one = rng.standard_normal((3, p + 1, 1, 1))
    assert np.abs(H.spatial_vcycle(p, tau, 1, one) - H._exact_blocks(p, tau, 1, one)).max() <= 1e-13


@pytest.mark.parametrize("p,nu", [(0, (1, 1)), (1, (2, 1)), (2, (1, 2))])
def test_time_cycle_with_exact_blocks_is_the_scalar_cycle_on_each_mode(p, nu):
    n, N, tau, (i, j) = 7, 32, 0.05, (3, 1)
    v = sine_mode(n, i, j)
    rng = np.random.default_rng(p)
    Fs = rng.standard_normal((N, p + 1))
    Fh = Fs[:, :, None, None] * v
    us = rng.standard_normal((N, p + 1))
    got = H.time_cycle(p, tau, n, Fh, us[:, :, None, None] * v, nu1=nu[0], nu2=nu[1], exact_blocks=True)
    ref = O.mg_one_cycle(p, eig(n, i, j) * tau, Fs, us, n_min=1, nu1=nu[0], nu2=nu[1], omega=0.5)
    assert np.abs(got - ref[:, :, None, None] * v).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("p", [0, 1])
def test_solver_converges_to_the_exact_solution(p):
    n, N, tau = 15, 32, 0.01
    rng = np.random.default_rng(9)
    F = rng.standard_normal((N, p + 1, n, n)) * tau
    u0 = rng.standard_normal((n, n))
    u, hist = H.solve(p, tau, n, F, u0, tol=1e-10, max_cycles=60)
    ex = H.exact_solve(p, tau, n, F, u0)
    assert hist[-1] <= 1e-10 and len(hist) <= 40, hist
    assert np.abs(u - ex).max() <= 1e-7 * np.abs(ex).max()
