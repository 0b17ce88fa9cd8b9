"""Adjoint solve on the GPU (tmg_adjoint) against the oracle.

mu = L^{-T} g is compared with the oracle's exact backward sweep; the scalar
gradients with the oracle's formulas on the same mu; and dJ/du0, dJ/dlambda
with central finite differences of the exact discrete loss.

Tolerances: the relative error of mu is at most cond(L) times the relative
residual the solve reaches, and cond(L) ~ 2/z for small z = lambda tau
(||L^{-1}|| ~ sum_k alpha^k ~ 1/z).  The cases go down to z = 6e-5
(cond ~ 3e4): the FP64 adjoint solve runs to 1e-12 (its own rounding floor is
~cond * 1e-16) and the allowance is 1e-7; mixed precision runs to 1e-10 and
the allowance is 1e-5.  Finite differences with h = 1e-5 (relative) have
truncation error ~h^2 and rounding error ~1e-16 / h: 1e-6 relative.
"""
import numpy as np
import pytest

import oracle as O
from paper_1409_5254_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5254_gb300 import build_ext
    build_ext.build()
    return torch.device("cuda:0")


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def problem(seed, N, p, lam, T=1.0):
    prob = inputs.scalar_problem(seed, N, p, lam=lam, T=T, u0=0.8)
    rng = np.random.default_rng(seed + 100)
    target = rng.standard_normal(N)
    return prob, target


CASES = [
    (1, 1024, 2.0, "fp64"),        # on-chip solver from level 0
    (2, 1 << 14, 10.0, "fp64"),    # streaming levels + on-chip tail
    (0, 1 << 14, 1.0, "fp64"),
    (3, 1 << 13, 300.0, "fp64"),
    (2, 1 << 14, 10.0, "mixed"),
    (1, 1 << 15, 1.0, "mixed"),
    (5, 1 << 13, 5.0, "fp64"),      # higher degrees
    (4, 1 << 14, 1.0, "mixed"),
]


W_CASES = [
    # W-cycles over streaming levels (on-chip part from 256 intervals down)
    (0, 1 << 14, 1.0, "fp64", 2),
    (2, 1 << 14, 10.0, "mixed", 2),
]


@pytest.mark.parametrize("p,N,lam,prec,gamma", [c + (1,) for c in CASES] + W_CASES)
def test_adjoint_matches_oracle(dev, p, N, lam, prec, gamma):
    from paper_1409_5254_gb300 import tmg
    prob, target = problem(p + N % 7, N, p, lam)
    tau = prob["tau"]
    z = lam * tau
    tol = 1e-12 if prec == "fp64" else 1e-10
    extra = {"gamma": 2, "tail_cap": 256} if gamma == 2 else {}
    with tmg.Plan(p, tau, lam, N, precision=prec, tol=tol, max_cycles=400, **extra) as plan:
        F = torch.from_numpy(prob["F"]).to(dev)
        u = plan.solve(F, prob["u0"])
        uh = u.cpu().numpy()
        _, _, _, b = O.blocks(p)
        g = np.outer(O.nodal_values(p, uh) - target, b)          # J = 1/2 sum (e_n - y_n)^2
        dJdf, du0, dlam = plan.adjoint(torch.from_numpy(g).to(dev), u)
        st = plan.stats()
    mu = dJdf.cpu().numpy()
    mu_ref = O.adj_sweep(p, z, g)
    allow = 1e-7 if prec == "fp64" else 1e-5
    assert rel(mu, mu_ref) <= allow, rel(mu, mu_ref)
    _, du0_ref, dlam_ref = O.adjoint_grads(p, lam, tau, g, uh)
    assert float(du0) == pytest.approx(du0_ref, rel=allow, abs=1e-14)
    assert float(dlam) == pytest.approx(dlam_ref, rel=allow, abs=1e-14)
    print(f"p={p} N={N} {prec} gamma={gamma}: adjoint cycles={st.cycles} mu err={rel(mu, mu_ref):.2e}")


@pytest.mark.parametrize("p", [0, 2])
def test_adjoint_gradients_match_finite_differences(dev, p):
    """GPU gradients against central differences of the exact discrete loss
    (forward substitution), i.e. the derivative the adjoint must reproduce."""
    from paper_1409_5254_gb300 import tmg
    N, lam = 4096, 3.0
    prob, target = problem(11, N, p, lam)
    tau = prob["tau"]
    F = torch.from_numpy(prob["F"]).to(dev)
    _, _, _, b = O.blocks(p)

    def J(u0, lam_):
        e = O.nodal_values(p, O.fsub(p, lam_ * tau, prob["F"], u0))
        return 0.5 * np.sum((e - target) ** 2)

    with tmg.Plan(p, tau, lam, N, precision="fp64", tol=1e-13, max_cycles=400) as plan:
        u = plan.solve(F, prob["u0"])
        g = np.outer(O.nodal_values(p, u.cpu().numpy()) - target, b)
        _, du0, dlam = plan.adjoint(torch.from_numpy(g).to(dev), u)
    h0, hl = 1e-5 * abs(prob["u0"]), 1e-5 * lam
    fd_u0 = (J(prob["u0"] + h0, lam) - J(prob["u0"] - h0, lam)) / (2 * h0)
    fd_lam = (J(prob["u0"], lam + hl) - J(prob["u0"], lam - hl)) / (2 * hl)
    assert float(du0) == pytest.approx(fd_u0, rel=1e-6)
    assert float(dlam) == pytest.approx(fd_lam, rel=1e-6)
