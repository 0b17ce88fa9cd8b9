"""GPU parity of the space-time heat-equation solver (tmg_heat_* in include/tmg.h)
against the FP64 oracle (oracle/heat.py), through the C ABI.

* one and two cycles from zero and from a random start: every value of the
  iterate within 1e-12 of the oracle's (relative to the largest value), over
  degrees 0..5, grids of 1 to 255 points a side (one to eight spatial
  levels; whole-row warps with 1, 2 or 4 columns per lane and several
  intervals per warp on the small grids, 64-column strips on the others) and
  1..64 intervals (one to seven time levels);
* the residual r = F - L u value by value;
* full solves: the residual history matches the oracle's cycle by cycle, and
  the converged solution matches the exact block forward substitution;
* at the benchmark size (n = 127, N = 4096, p_t = 1): the solve converges,
  and sampled intervals match the exact forward substitution -- the GPU
  solution's end values seed the oracle's exact step from that interval on;
* the mixed form (FP32 cycles on the FP64 residual): one cycle within FP32
  rounding of the oracle's cycle, solves to the same FP64 tolerance and the
  same exact solution, graph replay identical to direct issue;
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
                                   (1, 31, 8), (4, 1, 8), (1, 7, 1), (2, 1, 1), (1, 63, 4), (3, 63, 2),
                                   (1, 127, 2), (0, 255, 2)])
def test_cycle_iterates(p, n, N):
    H = _H()
    tau, F, u0 = inputs.heat_problem(10 + p + n + N, N, p, n)
    Fhat = H.fold_u0(p, F, u0)
    rng = np.random.default_rng(N + n)
    start = rng.uniform(-1.0, 1.0, F.shape)
    with tmg.HeatPlan(p, tau, n, N, nu_c=2, precision="fp64") as plan:
        Fd, u0d = _dev(F), _dev(u0)
        for u_init in (np.zeros_like(F), start):
            ud = _dev(u_init)
            want = u_init
            for _ in range(2):
                plan.cycle(Fd, u0d, ud)
                want = H.time_cycle(p, tau, n, Fhat, want, nu_c=2)
                got = ud.cpu().numpy()
                assert _rel(got, want) <= TOL_ITER, (p, n, N, _rel(got, want))


@pytest.mark.parametrize("nu1,nu2,nu_c", [(2, 1, 1), (0, 2, 3), (1, 0, 2), (2, 2, 1), (3, 3, 1)])
def test_cycle_smoothing_counts(nu1, nu2, nu_c):
    H = _H()
    p, n, N = 1, 15, 16
    tau, F, u0 = inputs.heat_problem(3, N, p, n)
    Fhat = H.fold_u0(p, F, u0)
    with tmg.HeatPlan(p, tau, n, N, nu1=nu1, nu2=nu2, nu_c=nu_c, precision="fp64") as plan:
        ud = torch.zeros(F.shape, dtype=torch.float64, device="cuda")
        plan.cycle(_dev(F), _dev(u0), ud)
    want = H.time_cycle(p, tau, n, Fhat, np.zeros_like(F), nu1=nu1, nu2=nu2, nu_c=nu_c)
    assert _rel(ud.cpu().numpy(), want) <= TOL_ITER


@pytest.mark.parametrize("p,n,N", [(1, 15, 16), (3, 7, 8)])
def test_residual(p, n, N):
    H = _H()
    tau, F, u0 = inputs.heat_problem(5, N, p, n)
    u = np.random.default_rng(7).uniform(-1.0, 1.0, F.shape)
    with tmg.HeatPlan(p, tau, n, N, precision="fp64") as plan:
        r = plan.residual(_dev(F), _dev(u0), _dev(u)).cpu().numpy()
    want = H.time_residual(p, tau, n, F, u, u0)
    assert np.max(np.abs(r - want)) <= 1e-12 * max(np.max(np.abs(want)), 1.0)


@pytest.mark.parametrize("p,n,N", [(0, 15, 32), (1, 31, 16), (2, 7, 64)])
def test_solve_history_and_exact(p, n, N):
    H = _H()
    tau, F, u0 = inputs.heat_problem(20 + p, N, p, n)
    with tmg.HeatPlan(p, tau, n, N, tol=1e-10, max_cycles=60, precision="fp64") as plan:
        u = plan.solve(_dev(F), _dev(u0)).cpu().numpy()
        st = plan.stats()
    _, hist = H.solve(p, tau, n, F, u0, tol=1e-10, max_cycles=60)
    assert st.cycles == len(hist) - 1
    assert st.rel_res <= 1e-10
    # relative residuals agree to rounding (both are norms of the same iterates)
    assert np.max(np.abs(st.hist - hist)) <= 1e-12
    ex = H.exact_solve(p, tau, n, F, u0)
    assert _rel(u, ex) <= 1e-7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_benchmark_size_sampled(precision):
    """n = 127, N = 4096, p_t = 1 (1.3e8 space-time values): converged, and
    sampled intervals equal the exact forward substitution started from the
    GPU solution's end values of the interval before."""
    H = _H()
    p, n, N = 1, 127, 4096
    tau, F, u0 = inputs.heat_problem(1, N, p, n)
    with tmg.HeatPlan(p, tau, n, N, tol=1e-10, max_cycles=40, precision=precision) as plan:
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


@pytest.mark.parametrize("p,n,N", [(1, 15, 16), (2, 31, 8), (0, 7, 64), (5, 7, 4), (1, 1, 8), (1, 63, 4),
                                   (1, 127, 2), (3, 127, 2), (0, 255, 2)])
def test_mixed_cycle_within_fp32(p, n, N):
    """u + C(F - L u) with the cycle C in FP32: within FP32 rounding of the
    oracle's FP64 cycle, measured against the size of the correction."""
    H = _H()
    tau, F, u0 = inputs.heat_problem(40 + p, N, p, n)
    Fhat = H.fold_u0(p, F, u0)
    start = np.random.default_rng(4).uniform(-1.0, 1.0, F.shape)
    with tmg.HeatPlan(p, tau, n, N, precision="mixed") as plan:
        ud = _dev(start)
        plan.cycle(_dev(F), _dev(u0), ud)
        got = ud.cpu().numpy()
    want = H.time_cycle(p, tau, n, Fhat, start)
    corr = np.max(np.abs(want - start))
    assert np.max(np.abs(got - want)) <= 2e-5 * corr


@pytest.mark.parametrize("p,n,N", [(1, 31, 32), (3, 15, 16)])
def test_mixed_solve_reaches_fp64_solution(p, n, N):
    H = _H()
    tau, F, u0 = inputs.heat_problem(60 + p, N, p, n)
    with tmg.HeatPlan(p, tau, n, N, tol=1e-10, max_cycles=60, precision="mixed") as plan:
        u = plan.solve(_dev(F), _dev(u0)).cpu().numpy()
        st = plan.stats()
        info = plan.info()
    _, hist = H.solve(p, tau, n, F, u0, tol=1e-10, max_cycles=60)
    assert st.rel_res <= 1e-10
    assert abs(st.cycles - (len(hist) - 1)) <= 2
    # the FP64 residual confirms every step: the oracle's residual of the result
    r = H.time_residual(p, tau, n, F, u, u0)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(H.fold_u0(p, F, u0))
    assert _rel(u, H.exact_solve(p, tau, n, F, u0)) <= 1e-7
    assert info["launches_per_cycle"] > 0 and info["time_levels"] == int(np.log2(N)) + 1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_matches_direct_issue(precision):
    p, n, N = 2, 15, 32
    tau, F, u0 = inputs.heat_problem(8, N, p, n)
    out = []
    for graph in (True, False):
        with tmg.HeatPlan(p, tau, n, N, tol=1e-9, precision=precision, use_graph=graph) as plan:
            out.append(plan.solve(_dev(F), _dev(u0)).cpu().numpy())
            # a second solve into another array re-captures for the new pointers
            u2 = plan.solve(_dev(F), _dev(u0), torch.empty(F.shape, dtype=torch.float64, device="cuda"))
            assert np.array_equal(u2.cpu().numpy(), out[-1])
    assert np.array_equal(out[0], out[1])
