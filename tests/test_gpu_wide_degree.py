"""Parity of the wide-degree paths, p_t = 10 and 20 (11 x 11 and 21 x 21
blocks, the largest degrees of the paper's scaling tables), with the FP64
oracle.

At these degrees the plan runs the per-level streaming kernels and solves its
coarsest level by the grid-wide scan in every cycle (no two-level kernels, no
on-chip coarse solver).  Tolerances as in the lower-degree parity tests:
* FP64 form: the blocks are well conditioned (cond(K + z Mhat) <= 21 at
  p_t = 10 and <= 41 at p_t = 20 for every z >= 0), so the iterates agree to
  1e-12 relative after each of three cycles;
* mixed form (the level-0 residual recomputed from u in FP64 every cycle):
  FP64 relative residual of the returned u, evaluated by the oracle,
  <= 1e-10 (x1.05 for the oracle's own rounding);
* adjoint: mu against the oracle's backward sweep within cond(L) times the
  reached residual, as in the lower-degree adjoint tests.
"""
import numpy as np
import pytest

import oracle as O
from paper_1409_5254_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DEGREES = [10, 20]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5254_gb300 import build_ext
    build_ext.build()
    return torch.device("cuda:0")


def tmg():
    from paper_1409_5254_gb300 import tmg as T
    return T


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def rel_residual(P, z, F, u0, u):
    r = O.residual(P, z, F, u0, u)
    return np.linalg.norm(r) / np.linalg.norm(O.fold_u0(P, F, u0))


CASES = [
    # (N, lam, n_min, levels, nu1, nu2, gamma, omega)
    (1 << 12, 1.0, 64, 0, 1, 1, 1, 0.0),      # 7 levels, coarsest 64 by the scan
    (1 << 12, 30.0, 2, 0, 2, 1, 1, 0.0),      # down to 2 intervals
    (3 * 1024, 1.0, 2, 0, 1, 1, 1, 0.0),      # odd coarsest level (3)
    (20002, 2.0, 15000, 0, 1, 1, 1, 0.0),     # coarsest 10001: several scan tiles, ragged last
    (1 << 12, 1.0, 64, 0, 0, 2, 1, 0.0),      # no pre-smoothing
    (1 << 12, 1.0, 64, 0, 1, 0, 1, 0.0),      # no post-smoothing
    (1 << 12, 1.0, 64, 0, 3, 2, 1, 0.0),      # wider halos
    (1 << 12, 1.0, 64, 0, 1, 1, 1, 0.5),      # uniform omega = 1/2
    (1 << 12, 1.0, 64, 3, 1, 1, 1, 0.0),      # capped level count: coarsest 1024
    (1 << 11, 1.0, 64, 0, 1, 1, 2, 0.0),      # W-cycle: streaming levels twice, a scan per visit
    (1 << 11, 3.0, 64, 0, 2, 2, 2, 0.0),
    (100, 1.0, 64, 0, 1, 1, 1, 0.0),          # two levels (100, 50)
    (37, 1.0, 64, 0, 1, 1, 1, 0.0),           # one level: each cycle is the exact scan
]


@pytest.mark.parametrize("P", DEGREES)
@pytest.mark.parametrize("case", CASES)
def test_cycles_match_textbook_cycle(dev, P, case):
    N, lam, n_min, levels, nu1, nu2, gamma, omega = case
    prob = inputs.scalar_problem(N % 97, N, P, lam=lam, T=1.0, u0=0.75)
    z = lam * prob["tau"]
    Fhat = O.fold_u0(P, prob["F"], prob["u0"])
    with tmg().Plan(P, prob["tau"], lam, N, levels, omega, precision="fp64", nu1=nu1, nu2=nu2, gamma=gamma,
                    n_min=n_min) as plan:
        info = plan.info()
        Fd = torch.from_numpy(prob["F"]).to(dev)
        u_d = torch.zeros_like(Fd)
        got = []
        for _ in range(3):
            plan.cycle(Fd, prob["u0"], u_d)
            got.append(u_d.cpu().numpy().copy())
    assert info["levels"] == O.num_levels(N, n_min, levels)
    assert info["tail_level"] == info["levels"] - 1      # the coarsest level, by the scan
    u = np.zeros_like(prob["F"])
    for k in range(3):
        u = O.mg_one_cycle(P, z, Fhat, u, n_min=n_min, max_levels=levels, nu1=nu1, nu2=nu2, gamma=gamma,
                           omega=omega)
        assert rel_err(got[k], u) <= 1e-12, (k, rel_err(got[k], u))


@pytest.mark.parametrize("P", DEGREES)
@pytest.mark.parametrize("gamma", [1, 2])
def test_solve_matches_forward_substitution(dev, P, gamma):
    N = 1 << 13
    prob = inputs.scalar_problem(3, N, P, lam=1.0, T=4.0, u0=1.0)
    z = prob["tau"]
    with tmg().Plan(P, prob["tau"], 1.0, N, precision="fp64", tol=1e-13, max_cycles=300, gamma=gamma) as plan:
        u = plan.solve(torch.from_numpy(prob["F"]).to(dev), prob["u0"]).cpu().numpy()
        st = plan.stats()
    assert rel_residual(P, z, prob["F"], prob["u0"], u) <= 1.05e-13
    assert rel_err(u, O.fsub(P, z, prob["F"], prob["u0"])) <= 1e-11
    # the device-side history follows the oracle's textbook solve cycle by cycle
    _, hist = O.mg_solve(P, z, prob["F"], prob["u0"], gamma=gamma, tol=1e-13, max_cycles=300)
    assert abs(st.cycles - (len(hist) - 1)) <= 1
    m = min(len(hist), len(st.hist))
    big = hist[:m] > 1e-9
    np.testing.assert_allclose(st.hist[:m][big], hist[:m][big], rtol=1e-6)


@pytest.mark.parametrize("P", DEGREES)
def test_large_solve_in_graph(dev, P):
    """2^20 intervals (1.2e7 unknowns at p_t = 10, 2.2e7 at 20): the graph
    solve to 1e-12 against forward substitution over the whole vector.  (With
    tau = 1e-2 the rounding floor of the relative residual, that of forward
    substitution itself, is 4.7e-14 at p_t = 10; it grows like 1/tau, as
    |u| / |F| does.)"""
    N = 1 << 20
    prob = inputs.scalar_problem(11, N, P, lam=1.0, tau=1e-2, u0=1.0)
    z = prob["tau"]
    with tmg().Plan(P, prob["tau"], 1.0, N, precision="fp64", tol=1e-12, nu1=2, nu2=2) as plan:
        u = plan.solve(torch.from_numpy(prob["F"]).to(dev), prob["u0"]).cpu().numpy()
        st = plan.stats()
    assert st.rel_res <= 1e-12
    assert rel_residual(P, z, prob["F"], prob["u0"], u) <= 1.05e-12
    assert rel_err(u, O.fsub(P, z, prob["F"], prob["u0"])) <= 1e-10


@pytest.mark.parametrize("P", DEGREES)
@pytest.mark.parametrize("N", [1, 5, 2049, 100003])
def test_direct_scan_solve(dev, P, N):
    """The exact scan solve; at p_t = 20 each thread chunk holds four
    intervals (a tile of 1024), so 100003 intervals span 98 tiles, the last
    one ragged."""
    prob = inputs.scalar_problem(N % 13, N, P, lam=3.0, T=1.0, u0=0.9)
    z = 3.0 * prob["tau"]
    with tmg().Plan(P, prob["tau"], 3.0, N, levels=1, precision="fp64") as plan:
        u = plan.solve_direct(torch.from_numpy(prob["F"]).to(dev), prob["u0"]).cpu().numpy()
    assert rel_residual(P, z, prob["F"], prob["u0"], u) <= max(1e-13, 1e-15 * np.sqrt(N * (P + 1)))
    assert rel_err(u, O.fsub(P, z, prob["F"], prob["u0"])) <= max(1e-12, 8 * N * 2.2e-16)


@pytest.mark.parametrize("P", DEGREES)
def test_residual_entry_point(dev, P):
    N = 3000
    prob = inputs.scalar_problem(9, N, P, lam=1.0, T=1.0, u0=0.4)
    u = np.random.default_rng(0).standard_normal((N, P + 1))
    with tmg().Plan(P, prob["tau"], 1.0, N, precision="fp64") as plan:
        r = plan.residual(torch.from_numpy(prob["F"]).to(dev), prob["u0"], torch.from_numpy(u).to(dev))
    np.testing.assert_allclose(r.cpu().numpy(), O.residual(P, prob["tau"], prob["F"], prob["u0"], u),
                               rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("P", DEGREES)
@pytest.mark.parametrize("zscale", [1e-3, 1.0, 1e3])
def test_mixed_solve_reaches_tolerance(dev, P, zscale):
    N = 1 << 13
    lam = zscale * N
    prob = inputs.scalar_problem(20, N, P, lam=lam, T=1.0, u0=1.0)
    z = lam * prob["tau"]
    with tmg().Plan(P, prob["tau"], lam, N, precision="mixed", tol=1e-10, max_cycles=200) as plan:
        u = plan.solve(torch.from_numpy(prob["F"]).to(dev), prob["u0"]).cpu().numpy()
        st = plan.stats()
    rr = rel_residual(P, z, prob["F"], prob["u0"], u)
    assert rr <= 1.05e-10, rr
    assert st.rel_res <= 1e-10
    err = rel_err(u, O.fsub(P, z, prob["F"], prob["u0"]))
    print(f"p={P} mixed z={z:.1e} cycles={st.cycles} rel_res={rr:.2e} err_vs_fp64={err:.2e}")
    assert err <= 1e-6


@pytest.mark.parametrize("P", DEGREES)
def test_mixed_large_solve(dev, P):
    N = 1 << 20
    prob = inputs.scalar_problem(11, N, P, lam=1.0, tau=1e-2, u0=1.0)
    z = prob["tau"]
    with tmg().Plan(P, prob["tau"], 1.0, N, precision="mixed", tol=1e-10, nu1=2, nu2=2) as plan:
        u = plan.solve(torch.from_numpy(prob["F"]).to(dev), prob["u0"]).cpu().numpy()
        st = plan.stats()
    rr = rel_residual(P, z, prob["F"], prob["u0"], u)
    assert st.rel_res <= 1e-10 and rr <= 1.05e-10, (st.rel_res, rr)
    assert rel_err(u, O.fsub(P, z, prob["F"], prob["u0"])) <= 1e-7


@pytest.mark.parametrize("P", DEGREES)
@pytest.mark.parametrize("prec,lam", [("fp64", 2.0), ("mixed", 40.0)])
def test_adjoint_matches_oracle(dev, P, prec, lam):
    """The transposed, backward-in-time solve at the wide degrees: mu = L^{-T} g
    against the oracle's backward sweep (allowance cond(L) ~ 2/z times the
    reached residual, as at p_t <= 5), the gradients dJ/du0 = a^T mu_1 and
    dJ/dlambda = -tau sum mu_n^T Mhat u_n against the oracle's formulas."""
    T = tmg()
    N = 1 << 12
    prob = inputs.scalar_problem(5 + P, N, P, lam=lam, T=1.0, u0=0.8)
    tau = prob["tau"]
    z = lam * tau
    tol = 1e-12 if prec == "fp64" else 1e-10
    target = np.random.default_rng(P).standard_normal(N)
    with T.Plan(P, tau, lam, N, precision=prec, tol=tol, max_cycles=300) as plan:
        u = plan.solve(torch.from_numpy(prob["F"]).to(dev), prob["u0"])
        uh = u.cpu().numpy()
        _, _, _, b = O.blocks(P)
        g = np.outer(O.nodal_values(P, uh) - target, b)
        dJdf, du0, dlam = plan.adjoint(torch.from_numpy(g).to(dev), u)
        st = plan.stats()
    mu = dJdf.cpu().numpy()
    mu_ref = O.adj_sweep(P, z, g)
    allow = 2.0 / z * tol * 10
    assert rel_err(mu, mu_ref) <= allow, (rel_err(mu, mu_ref), allow)
    _, du0_ref, dlam_ref = O.adjoint_grads(P, lam, tau, g, uh)
    assert float(du0) == pytest.approx(du0_ref, rel=allow, abs=1e-14)
    assert float(dlam) == pytest.approx(dlam_ref, rel=allow, abs=1e-14)
    print(f"p={P} {prec}: adjoint cycles={st.cycles} mu err={rel_err(mu, mu_ref):.2e}")


@pytest.mark.parametrize("P", DEGREES)
def test_adjoint_cycles_contract(dev, P):
    """Cycle by cycle: the FP64 adjoint run for exactly k cycles (tol = 0,
    max_cycles = k) contracts its error against the oracle's backward sweep by
    at least one half per V(1,1) cycle, as the forward cycle does (the oracle
    has no reversed-time cycle to compare iterates with)."""
    T = tmg()
    N, lam = 1 << 11, 3.0
    prob = inputs.scalar_problem(2, N, P, lam=lam, T=1.0, u0=0.5)
    tau = prob["tau"]
    g = np.random.default_rng(7).standard_normal((N, P + 1))
    mu_ref = O.adj_sweep(P, lam * tau, g)
    errs = []
    for k in (1, 2, 3, 6):
        with T.Plan(P, tau, lam, N, precision="fp64", tol=0.0, max_cycles=k) as plan:
            u = torch.zeros((N, P + 1), dtype=torch.float64, device=dev)
            mu, _, _ = plan.adjoint(torch.from_numpy(g).to(dev), u, allow_notconv=True)
            assert plan.stats().cycles == k
        errs.append(rel_err(mu.cpu().numpy(), mu_ref))
    # the error falls by at least one half per cycle (the measured factor is
    # about 0.25, the two-grid estimate at p_t >= 1)
    for a, b_ in zip(errs, errs[1:3]):
        assert b_ <= 0.5 * a, errs
    assert errs[-1] <= 0.5 ** 5 * errs[0], errs
