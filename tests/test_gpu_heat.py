"""GPU parity of the space-time heat-equation solver (tmg_heat_* in include/tmg.h)
against the FP64 oracle (oracle/heat.py), through the C ABI.

* one and two cycles from zero and from a random start: every value of the
  iterate within 1e-12 of the oracle's (relative to the largest value), over
  degrees 0..5, grids of 1, 3, 7, 15 and 31 points a side (one to five
  spatial levels) and 1..64 intervals (one to seven time levels);
* the residual r = F - L u value by value;
* full solves: the residual history matches the oracle's cycle by cycle, and
  the converged solution matches the exact block forward substitution;
* at the benchmark size (n = 127, N = 4096, p_t = 1): the solve converges,
  and sampled intervals match the exact forward substitution -- the GPU
  solution's end values seed the oracle's exact step from that interval on;
* invalid sizes and options are rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1409_5254_gb300 import inputs, tmg  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_ITER = 1e-12


def _H():
    from oracle import heat
    return heat


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("p,n,N", [(0, 7, 16), (1, 7, 16), (2, 15, 8), (1, 15, 64), (3, 3, 4), (5, 7, 2),
                                   (1, 31, 8), (4, 1, 8), (1, 7, 1), (2, 1, 1)])
def test_cycle_iterates(p, n, N):
    H = _H()
    tau, F, u0 = inputs.heat_problem(10 + p + n + N, N, p, n)
    Fhat = H.fold_u0(p, F, u0)
    rng = np.random.default_rng(N + n)
    start = rng.uniform(-1.0, 1.0, F.shape)
    with tmg.HeatPlan(p, tau, n, N, nu_c=2) as plan:
        Fd, u0d = _dev(F), _dev(u0)
        for u_init in (np.zeros_like(F), start):
            ud = _dev(u_init)
            want = u_init
            for _ in range(2):
                plan.cycle(Fd, u0d, ud)
                want = H.time_cycle(p, tau, n, Fhat, want, nu_c=2)
                got = ud.cpu().numpy()
                assert _rel(got, want) <= TOL_ITER, (p, n, N, _rel(got, want))


@pytest.mark.parametrize("nu1,nu2,nu_c", [(2, 1, 1), (0, 2, 3), (1, 0, 2)])
def test_cycle_smoothing_counts(nu1, nu2, nu_c):
    H = _H()
    p, n, N = 1, 15, 16
    tau, F, u0 = inputs.heat_problem(3, N, p, n)
    Fhat = H.fold_u0(p, F, u0)
    with tmg.HeatPlan(p, tau, n, N, nu1=nu1, nu2=nu2, nu_c=nu_c) as plan:
        ud = torch.zeros(F.shape, dtype=torch.float64, device="cuda")
        plan.cycle(_dev(F), _dev(u0), ud)
    want = H.time_cycle(p, tau, n, Fhat, np.zeros_like(F), nu1=nu1, nu2=nu2, nu_c=nu_c)
    assert _rel(ud.cpu().numpy(), want) <= TOL_ITER


@pytest.mark.parametrize("p,n,N", [(1, 15, 16), (3, 7, 8)])
def test_residual(p, n, N):
    H = _H()
    tau, F, u0 = inputs.heat_problem(5, N, p, n)
    u = np.random.default_rng(7).uniform(-1.0, 1.0, F.shape)
    with tmg.HeatPlan(p, tau, n, N) as plan:
        r = plan.residual(_dev(F), _dev(u0), _dev(u)).cpu().numpy()
    want = H.time_residual(p, tau, n, F, u, u0)
    assert np.max(np.abs(r - want)) <= 1e-12 * max(np.max(np.abs(want)), 1.0)


@pytest.mark.parametrize("p,n,N", [(0, 15, 32), (1, 31, 16), (2, 7, 64)])
def test_solve_history_and_exact(p, n, N):
    H = _H()
    tau, F, u0 = inputs.heat_problem(20 + p, N, p, n)
    with tmg.HeatPlan(p, tau, n, N, tol=1e-10, max_cycles=60) as plan:
        u = plan.solve(_dev(F), _dev(u0)).cpu().numpy()
        st = plan.stats()
    _, hist = H.solve(p, tau, n, F, u0, tol=1e-10, max_cycles=60)
    assert st.cycles == len(hist) - 1
    assert st.rel_res <= 1e-10
    # relative residuals agree to rounding (both are norms of the same iterates)
    assert np.max(np.abs(st.hist - hist)) <= 1e-12
    ex = H.exact_solve(p, tau, n, F, u0)
    assert _rel(u, ex) <= 1e-7


def test_benchmark_size_sampled():
    """n = 127, N = 4096, p_t = 1 (1.3e8 space-time values): converged, and
    sampled intervals equal the exact forward substitution started from the
    GPU solution's end values of the interval before."""
    H = _H()
    p, n, N = 1, 127, 4096
    tau, F, u0 = inputs.heat_problem(1, N, p, n)
    with tmg.HeatPlan(p, tau, n, N, tol=1e-10, max_cycles=40) as plan:
        u = plan.solve(_dev(F), _dev(u0)).cpu().numpy()
        st = plan.stats()
    assert st.rel_res <= 1e-10 and st.cycles <= 40
    scale = np.max(np.abs(u))
    for m in (0, 1, 777, 2048, N - 1):
        prev = u0 if m == 0 else u[m - 1].sum(axis=0)
        ex = H.exact_solve(p, tau, n, F[m:m + 1], prev)[0]
        assert np.max(np.abs(u[m] - ex)) <= 1e-7 * scale, m


def test_rejects_bad_sizes():
    for args in ((1, 1e-3, 6, 16), (1, 1e-3, 7, 12), (6, 1e-3, 7, 16), (1, 0.0, 7, 16), (1, 1e-3, 0, 16)):
        with pytest.raises(tmg.TmgError):
            tmg.HeatPlan(*args)
    with pytest.raises(tmg.TmgError):
        tmg.HeatPlan(1, 1e-3, 7, 16, nu_c=0)
    with pytest.raises(tmg.TmgError):
        tmg.HeatPlan(1, 1e-3, 7, 16, nu1=0, nu2=0)
