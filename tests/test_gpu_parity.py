"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written from the arithmetic):
* FP64 form, iterate parity with the oracle's textbook cycle after k cycles:
  1e-12 relative (both evaluate the same linear map in FP64; they differ only
  in rounding order -- the GPU works in correction form with the block
  inverse applied as a mat-vec).
* FP64 form solved to tol 1e-13 vs exact forward substitution: 1e-11 relative
  (the error is bounded by the residual times ||L^{-1}||).
* Mixed form: FP64 relative residual of the returned u, evaluated by the
  oracle, <= 1e-10 (x1.05 for the oracle's own rounding); the error against
  forward substitution is reported.
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


def tmg():
    from paper_1409_5254_gb300 import tmg as T
    return T


def rel_err(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def rel_residual(p, z, F, u0, u):
    r = O.residual(p, z, F, u0, u)
    return np.linalg.norm(r) / np.linalg.norm(O.fold_u0(p, F, u0))


def gpu_cycles(dev, p, tau, lam, F, u0, k, **kw):
    N = F.shape[0]
    with tmg().Plan(p, tau, lam, N, precision="fp64", **kw) as plan:
        Fd = torch.from_numpy(F).to(dev)
        u = torch.zeros_like(Fd)
        out = []
        for _ in range(k):
            plan.cycle(Fd, u0, u)
            out.append(u.cpu().numpy().copy())
        info = plan.info()
    return out, info


CYCLE_CASES = [
    # (p, N, lam, T, n_min, levels, nu1, nu2, gamma, omega)
    (1, 1024, 1.0, 1.0, 2, 0, 1, 1, 1, 0.0),          # small: on-chip solver from level 0
    (0, 1 << 14, 1.0, 1.0, 64, 0, 1, 1, 1, 0.0),      # streaming levels + on-chip tail
    (1, 1 << 14, 3.0, 2.0, 64, 0, 1, 1, 1, 0.0),
    (2, 1 << 14, 1.0, 1.0, 16, 0, 1, 1, 1, 0.0),
    (3, 1 << 14, 50.0, 1.0, 64, 0, 1, 1, 1, 0.0),
    (1, 1 << 14, 1.0, 1.0, 64, 0, 2, 2, 1, 0.0),      # more sweeps: wider halos
    (2, 1 << 13, 1.0, 1.0, 64, 0, 3, 1, 1, 0.0),
    (1, 1 << 14, 1.0, 1.0, 64, 0, 1, 0, 1, 0.0),      # no post-smoothing
    (1, 1 << 14, 1.0, 1.0, 64, 0, 0, 2, 1, 0.0),      # no pre-smoothing
    (1, 1 << 14, 1.0, 1.0, 64, 0, 1, 1, 1, 0.5),      # uniform omega = 1/2
    (0, 4096, 1.0, 1.0, 4, 0, 1, 1, 2, 0.0),          # W-cycle (on chip)
    (1, 1 << 14, 1.0, 1.0, 64, 4, 1, 1, 1, 0.0),      # capped level count: large coarsest scan
    (1, 3 * 1024, 1.0, 1.0, 2, 0, 1, 1, 1, 0.0),      # N = 3 * 2^10: odd coarsest level (3)
    (2, 1 << 16, 1.0, 1.0, 16384, 0, 1, 1, 1, 0.0),   # coarsest level (16384) solved by the grid-wide scan
    (0, 20002, 2.0, 1.0, 15000, 0, 1, 1, 1, 0.0),     # odd coarsest level of 10001 by the scan (ragged last tile)
    (4, 1 << 14, 2.0, 1.0, 64, 0, 1, 1, 1, 0.0),      # higher degrees (p_t = 4, 5)
    (5, 1 << 13, 1.0, 1.0, 16, 0, 2, 1, 1, 0.0),
    (5, 1 << 14, 30.0, 1.0, 2, 0, 1, 2, 1, 0.0),
]


@pytest.mark.parametrize("case", CYCLE_CASES)
def test_fp64_cycles_match_textbook_cycle(dev, case):
    p, N, lam, T, n_min, levels, nu1, nu2, gamma, omega = case
    prob = inputs.scalar_problem(N % 97, N, p, lam=lam, T=T, u0=0.75)
    z = lam * prob["tau"]
    Fhat = O.fold_u0(p, prob["F"], prob["u0"])
    got, info = gpu_cycles(dev, p, prob["tau"], lam, prob["F"], prob["u0"], 3, levels=levels, omega=omega,
                           nu1=nu1, nu2=nu2, gamma=gamma, n_min=n_min)
    assert info["levels"] == O.num_levels(N, n_min, levels)
    u = np.zeros_like(prob["F"])
    for k in range(3):
        u = O.mg_one_cycle(p, z, Fhat, u, n_min=n_min, max_levels=levels, nu1=nu1, nu2=nu2, gamma=gamma,
                           omega=omega)
        assert rel_err(got[k], u) <= 1e-12, (k, rel_err(got[k], u))


W_CASES = [
    # (p, N, lam, n_min, tail_cap, nu1, nu2): W-cycles over streaming levels --
    # every level below 1 visited twice per visit of its parent, the second
    # visit starting from the first one's result
    (0, 1 << 14, 1.0, 64, 64, 1, 1),        # 7 streaming levels, coarsest (64) by the on-chip solver
    (1, 1 << 14, 3.0, 64, 512, 2, 1),       # 4 streaming levels, W inside the on-chip part (512 .. 64)
    (2, 1 << 13, 1.0, 64, 1024, 1, 2),
    (1, 1 << 14, 1.0, 64, 0, 2, 2),         # default cap 8192: level 1 is on chip, visited twice
    (1, 1 << 16, 1.0, 16384, 0, 1, 1),      # coarsest level 16384 > 8192: the exact scan on each visit
    (3, 1 << 13, 20.0, 64, 128, 0, 2),      # no pre-smoothing
    (1, 1 << 13, 1.0, 64, 128, 1, 0),       # no post-smoothing
]


@pytest.mark.parametrize("case", W_CASES)
def test_w_cycles_over_streaming_levels_match_textbook_cycle(dev, case):
    """W-cycles whose streaming levels are visited twice (k_down_nz/k_up_nz
    on second visits, the on-chip solver or the exact scan started from the
    first visit's result): three FP64 cycles match the oracle's recursive
    W-cycle to 1e-12."""
    p, N, lam, n_min, cap, nu1, nu2 = case
    prob = inputs.scalar_problem(N % 89, N, p, lam=lam, T=1.0, u0=0.5)
    z = lam * prob["tau"]
    Fhat = O.fold_u0(p, prob["F"], prob["u0"])
    got, info = gpu_cycles(dev, p, prob["tau"], lam, prob["F"], prob["u0"], 3, nu1=nu1, nu2=nu2, gamma=2,
                           n_min=n_min, tail_cap=cap)
    assert info["tail_level"] >= 1
    u = np.zeros_like(prob["F"])
    for k in range(3):
        u = O.mg_one_cycle(p, z, Fhat, u, n_min=n_min, nu1=nu1, nu2=nu2, gamma=2)
        assert rel_err(got[k], u) <= 1e-12, (k, rel_err(got[k], u))


@pytest.mark.parametrize("p", [0, 1])
def test_w_cycle_mixed_solve_reaches_tolerance(dev, p):
    """A mixed-precision solve with W-cycles over streaming levels reaches the
    FP64 tolerance; p_t = 0, whose V-cycles degrade on long horizons, needs
    far fewer W-cycles than V-cycles."""
    N = 1 << 16
    prob = inputs.scalar_problem(31, N, p, lam=1.0, T=N * 1e-4, u0=1.0)
    Fd = torch.from_numpy(prob["F"]).to(dev)
    cycles = {}
    for gamma in (1, 2):
        with tmg().Plan(p, prob["tau"], 1.0, N, precision="mixed", gamma=gamma, tail_cap=256,
                        max_cycles=300) as plan:
            u = plan.solve(Fd, prob["u0"])
            cycles[gamma] = plan.stats().cycles
            assert rel_residual(p, prob["tau"], prob["F"], prob["u0"], u.cpu().numpy()) <= 1.05e-10
    print(f"p={p}: V-cycles {cycles[1]}, W-cycles {cycles[2]}")
    assert cycles[2] <= cycles[1]


@pytest.mark.parametrize("tail_cap", [64, 128])
@pytest.mark.parametrize("nu", [(1, 1), (2, 1), (0, 2), (1, 0), (3, 2)])
def test_fused_level_pairs_match_textbook_cycle(dev, tail_cap, nu):
    """Streaming levels run two per kernel (levels l and l+1, level l+1 never
    stored).  With a small on-chip solver there are 8 (tail_cap 64: four pairs)
    or 7 (tail_cap 128: three pairs and a single level) streaming levels; the
    FP64 iterates match the textbook cycle to 1e-12 for several sweep counts,
    and the unfused kernels give the same iterates to rounding."""
    p, N, lam = 1, 1 << 15, 4.0
    nu1, nu2 = nu
    prob = inputs.scalar_problem(13, N, p, lam=lam, T=1.0, u0=0.5)
    z = lam * prob["tau"]
    Fhat = O.fold_u0(p, prob["F"], prob["u0"])
    got, info = gpu_cycles(dev, p, prob["tau"], lam, prob["F"], prob["u0"], 2, nu1=nu1, nu2=nu2, n_min=2,
                           tail_cap=tail_cap, fuse_levels=True)
    assert info["tail_level"] == (9 if tail_cap == 64 else 8)
    unf, _ = gpu_cycles(dev, p, prob["tau"], lam, prob["F"], prob["u0"], 2, nu1=nu1, nu2=nu2, n_min=2,
                        tail_cap=tail_cap, fuse_levels=False)
    u = np.zeros_like(prob["F"])
    for k in range(2):
        u = O.mg_one_cycle(p, z, Fhat, u, n_min=2, nu1=nu1, nu2=nu2)
        assert rel_err(got[k], u) <= 1e-12, (k, rel_err(got[k], u))
        assert rel_err(got[k], unf[k]) <= 1e-13


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
def test_fp64_solve_matches_forward_substitution(dev, p):
    N = 1 << 13
    prob = inputs.scalar_problem(p, N, p, lam=1.0, T=4.0, u0=1.0)
    z = prob["tau"]
    Fd = torch.from_numpy(prob["F"]).to(dev)
    gamma = 1
    with tmg().Plan(p, prob["tau"], 1.0, N, precision="fp64", tol=1e-13, max_cycles=300, gamma=gamma) as plan:
        u = plan.solve(Fd, prob["u0"]).cpu().numpy()
        st = plan.stats()
    u_ex = O.fsub(p, z, prob["F"], prob["u0"])
    assert rel_residual(p, z, prob["F"], prob["u0"], u) <= 1.05e-13
    assert rel_err(u, u_ex) <= 1e-11
    # the device-side history matches the oracle's textbook solve cycle by cycle
    _, hist = O.mg_solve(p, z, prob["F"], prob["u0"], tol=1e-13, max_cycles=300)
    assert abs(st.cycles - (len(hist) - 1)) <= 1
    m = min(len(hist), len(st.hist))
    big = hist[:m] > 1e-9
    np.testing.assert_allclose(st.hist[:m][big], hist[:m][big], rtol=1e-6)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("zscale", [1e-3, 1.0, 1e3])
def test_mixed_solve_reaches_tolerance(dev, p, zscale):
    N = 1 << 14
    T = 1.0
    lam = zscale * N / T
    prob = inputs.scalar_problem(10 + p, N, p, lam=lam, T=T, u0=1.0)
    z = lam * prob["tau"]
    Fd = torch.from_numpy(prob["F"]).to(dev)
    with tmg().Plan(p, prob["tau"], lam, N, precision="mixed", tol=1e-10, max_cycles=200) as plan:
        u = plan.solve(Fd, prob["u0"]).cpu().numpy()
        st = plan.stats()
    rr = rel_residual(p, z, prob["F"], prob["u0"], u)
    assert rr <= 1.05e-10, rr
    assert st.rel_res <= 1e-10
    u_ex = O.fsub(p, z, prob["F"], prob["u0"])
    err = rel_err(u, u_ex)
    print(f"p={p} z={z:.1e} cycles={st.cycles} rel_res={rr:.2e} err_vs_fp64={err:.2e}")
    assert err <= 1e-6


EDGE = [
    (1, 1, 1.0),        # one interval
    (2, 2, 1.0),
    (0, 5, 1.0),        # odd: no coarsening, exact on-chip scan
    (3, 1001, 1.0),
    (1, 8192, 0.0),     # lambda = 0
    (1, 4096, 1e3),     # large steps
]


@pytest.mark.parametrize("p,N,lam", EDGE)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_edge_cases(dev, p, N, lam, prec):
    prob = inputs.scalar_problem(N, N, p, lam=lam, T=1.0, u0=-0.3)
    z = lam * prob["tau"]
    Fd = torch.from_numpy(prob["F"]).to(dev)
    with tmg().Plan(p, prob["tau"], lam, N, precision=prec, tol=1e-12 if prec == "fp64" else 1e-10,
                    n_min=2) as plan:
        u = plan.solve(Fd, prob["u0"]).cpu().numpy()
    u_ex = O.fsub(p, z, prob["F"], prob["u0"])
    assert rel_residual(p, z, prob["F"], prob["u0"], u) <= (1.05e-12 if prec == "fp64" else 1.05e-10)
    assert rel_err(u, u_ex) <= (1e-10 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("p,N,lam,n_min", [e + (2,) for e in EDGE] + [(2, 1 << 14, 1e3 * (1 << 14), 1)])
def test_edge_case_cycles_match_textbook_cycle(dev, p, N, lam, n_min):
    """The edge cases above (one and two intervals, an odd length without
    coarsening, 1001 = 7 * 11 * 13, lambda = 0, lambda tau = 1e3) and a
    15-level hierarchy with z up to 1.6e7 on its coarsest level, held at the
    iterate level: the FP64 iterates after 1, 2 and 3 cycles against the
    oracle's textbook cycle (eq. chap4_errorTwoGridCycle with omega* of Lemma
    chap4_lemma7 per level), 1e-12 relative."""
    prob = inputs.scalar_problem(N, N, p, lam=lam, T=1.0, u0=-0.3)
    z = lam * prob["tau"]
    Fhat = O.fold_u0(p, prob["F"], prob["u0"])
    got, info = gpu_cycles(dev, p, prob["tau"], lam, prob["F"], prob["u0"], 3, n_min=n_min)
    assert info["levels"] == O.num_levels(N, n_min, 0)
    u = np.zeros_like(prob["F"])
    for k in range(3):
        u = O.mg_one_cycle(p, z, Fhat, u, n_min=n_min)
        assert rel_err(got[k], u) <= 1e-12, (k, rel_err(got[k], u))


def test_deep_hierarchy_large_z(dev):
    """lambda tau = 1e3 with many levels (z up to ~1e7 on the coarsest level)."""
    N = 1 << 14
    p = 2
    lam = 1e3 * N
    prob = inputs.scalar_problem(3, N, p, lam=lam, T=1.0, u0=1.0)
    Fd = torch.from_numpy(prob["F"]).to(dev)
    for prec in ("fp64", "mixed"):
        with tmg().Plan(p, prob["tau"], lam, N, precision=prec, n_min=1) as plan:
            u = plan.solve(Fd, prob["u0"]).cpu().numpy()
            assert plan.info()["levels"] == 15
        assert rel_residual(p, lam * prob["tau"], prob["F"], prob["u0"], u) <= 1.05e-10


def test_initial_guess_and_host_entry(dev):
    N, p = 1 << 13, 1
    prob = inputs.scalar_problem(5, N, p, lam=2.0, T=1.0, u0=1.0)
    z = 2.0 * prob["tau"]
    u_ex = O.fsub(p, z, prob["F"], prob["u0"])
    Fd = torch.from_numpy(prob["F"]).to(dev)
    with tmg().Plan(p, prob["tau"], 2.0, N, precision="fp64", initial_guess=True, tol=1e-12) as plan:
        u = torch.from_numpy(u_ex * (1 + 1e-6)).to(dev)
        plan.solve(Fd, prob["u0"], u)
        st = plan.stats()
        # the start is 1e-6 from the solution: about log(1e-6)/log(rho ~ 0.25) = 10 cycles
        assert st.hist[0] == pytest.approx(1e-6, rel=0.2) and st.cycles <= 12
        assert rel_err(u.cpu().numpy(), u_ex) <= 1e-10
    with tmg().Plan(p, prob["tau"], 2.0, N, precision="mixed") as plan:
        out = torch.empty((N, p + 1), dtype=torch.float64).pin_memory()
        plan.solve_host(torch.from_numpy(prob["F"]).pin_memory(), prob["u0"], out)
        assert rel_residual(p, z, prob["F"], prob["u0"], out.numpy()) <= 1.05e-10


def test_residual_entry_point(dev):
    N, p = 3000, 3
    prob = inputs.scalar_problem(9, N, p, lam=1.0, T=1.0, u0=0.4)
    u = np.random.default_rng(0).standard_normal((N, p + 1))
    with tmg().Plan(p, prob["tau"], 1.0, N) as plan:
        r = plan.residual(torch.from_numpy(prob["F"]).to(dev), prob["u0"], torch.from_numpy(u).to(dev))
    np.testing.assert_allclose(r.cpu().numpy(), O.residual(p, prob["tau"], prob["F"], prob["u0"], u),
                               rtol=1e-13, atol=1e-13)


def test_graph_eager_and_pdl_agree_and_are_deterministic(dev):
    N, p = 1 << 15, 1
    prob = inputs.scalar_problem(2, N, p, lam=1.0, T=8.0, u0=1.0)
    Fd = torch.from_numpy(prob["F"]).to(dev)
    outs = []
    for use_graph, use_pdl in ((True, True), (True, True), (False, True), (True, False), (False, False)):
        with tmg().Plan(p, prob["tau"], 1.0, N, precision="mixed", use_graph=use_graph, use_pdl=use_pdl) as plan:
            outs.append(plan.solve(Fd, prob["u0"]).cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


def test_not_converged_status(dev):
    N, p = 1 << 12, 1
    prob = inputs.scalar_problem(4, N, p, lam=1.0, T=1.0, u0=1.0)
    Fd = torch.from_numpy(prob["F"]).to(dev)
    T = tmg()
    with T.Plan(p, prob["tau"], 1.0, N, max_cycles=2, tol=1e-14) as plan:
        with pytest.raises(T.TmgError) as ei:
            plan.solve(Fd, prob["u0"])
        assert ei.value.status == T.TMG_ENOTCONV
        u = plan.solve(Fd, prob["u0"], allow_notconv=True)
        assert plan.stats().cycles == 2


@pytest.mark.parametrize("n_min", [64, 1 << 17])
def test_full_size_long_horizon_sampled(dev, n_min):
    """The benchmark workload (N = 2^24, tau = 1e-6, lambda = 1, p = 1, V(2,2)),
    in the launch configuration the benchmark times (coarsest level 2^17
    intervals, solved by the grid-wide affine scan) and with the library's
    default hierarchy (coarsest 64 intervals): FP64 residual of the whole GPU
    result, and sampled intervals against exact forward substitution."""
    N, p = 1 << 24, 1
    prob = inputs.scalar_problem(1, N, p, lam=1.0, tau=1e-6, u0=1.0)
    Fd = torch.from_numpy(prob["F"]).to(dev)
    with tmg().Plan(p, 1e-6, 1.0, N, precision="mixed", nu1=2, nu2=2, n_min=n_min) as plan:
        u = plan.solve(Fd, prob["u0"])
        r = plan.residual(Fd, prob["u0"], u)
        st = plan.stats()
    Fhat = O.fold_u0(p, prob["F"], prob["u0"])
    rr = float(torch.linalg.vector_norm(r).item()) / np.linalg.norm(Fhat)
    assert rr <= 1.05e-10, rr
    u_ex = O.fsub(p, 1e-6, prob["F"], prob["u0"])
    idx = np.random.default_rng(0).integers(0, N, 4096)
    idx = np.concatenate([idx, [0, 1, N - 2, N - 1]])
    uh = u.cpu().numpy()
    err = np.abs(uh[idx] - u_ex[idx]).max() / np.abs(u_ex).max()
    print(f"full size: cycles={st.cycles} rel_res={rr:.2e} sampled err={err:.2e}")
    assert err <= 1e-6


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("N", [1, 5, 2047, 2048, 2049, 100003, (1 << 20) + 3])
def test_direct_scan_solve(dev, p, N):
    """tmg_solve_direct (three-pass FP64 scan) against forward substitution.

    Backward error: the scan's residual is at the rounding level
    (max(1e-13, 1e-15 sqrt(N (p+1)))).  Forward
    error: both methods apply a correctly rounded multiplier alpha (off by up
    to half an ulp, the same bias at every step), and the recurrence turns
    that into a difference of up to ~N eps in alpha^N; the allowance is
    max(1e-12, 8 N eps) relative."""
    prob = inputs.scalar_problem(N % 13, N, p, lam=3.0, T=1.0, u0=0.9)
    z = 3.0 * prob["tau"]
    with tmg().Plan(p, prob["tau"], 3.0, N, levels=1) as plan:
        u = plan.solve_direct(torch.from_numpy(prob["F"]).to(dev), prob["u0"]).cpu().numpy()
    # per-component rounding of ~eps |u| over N (p+1) components (a random-walk sum)
    assert rel_residual(p, z, prob["F"], prob["u0"], u) <= max(1e-13, 1e-15 * np.sqrt(N * (p + 1)))
    ex = O.fsub(p, z, prob["F"], prob["u0"])
    assert rel_err(u, ex) <= max(1e-12, 8 * N * 2.2e-16), rel_err(u, ex)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_level_large_problem_uses_scan(dev, prec):
    """One level too large for the on-chip solver: each cycle is residual,
    exact scan of the correction, update (FP32 scan for the mixed form)."""
    N, p = 100000, 1
    prob = inputs.scalar_problem(6, N, p, lam=1.0, T=10.0, u0=1.0)
    z = prob["tau"]
    with tmg().Plan(p, prob["tau"], 1.0, N, levels=1, precision=prec, tol=1e-10) as plan:
        assert plan.info()["levels"] == 1
        u = plan.solve(torch.from_numpy(prob["F"]).to(dev), 1.0).cpu().numpy()
        st = plan.stats()
    assert st.cycles <= (2 if prec == "fp64" else 6)
    assert rel_residual(p, z, prob["F"], 1.0, u) <= 1.05e-10



@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("zscale", [1e-3, 1.0, 1e3])
def test_updated_residual_matches_fp64_residual(dev, p, zscale):
    """Mixed form: after one cycle the level-0 residual kept as a float pair
    (r + low, updated by r -= L c without FP64 arithmetic) equals F - L u of
    the FP64 iterate, evaluated by the oracle.  The update carries ~2^-48 of
    its terms, |L| |c| with c ~ u after the first cycle, and u += c rounds u
    in FP64: 1e-13 S per component, S = (2 + z)(p + 1) max|u| bounding |L| |u|
    (Legendre blocks: |K| entries <= 1, plus the coupling).  The stored low
    part resolves 2^-16 ulp of the high part (2^-39 relative), once for the
    recomputed residual the cycle starts from (|r| <= |F| + S) and once for
    the update: 2^-37 (max|F| + S)."""
    N = 4096 + 64
    T = 1.0
    lam = zscale * N / T
    prob = inputs.scalar_problem(20 + p, N, p, lam=lam, T=T, u0=0.7)
    z = lam * prob["tau"]
    Fd = torch.from_numpy(prob["F"]).to(dev)
    with tmg().Plan(p, prob["tau"], lam, N, precision="mixed", tail_cap=256) as plan:
        assert plan.info()["tail_level"] >= 1
        u = torch.zeros_like(Fd)
        for k in range(3):
            plan.cycle(Fd, prob["u0"], u)
            uh = u.cpu().numpy()
            r_pair = plan.inspect("r").astype(np.float64) + plan.inspect("rlo").astype(np.float64)
            r_ex = O.residual(p, z, prob["F"], prob["u0"], uh)
            S = (2 + z) * (p + 1) * np.abs(uh).max()
            allow = 1e-13 * S + 2.0 ** -37 * (np.abs(O.fold_u0(p, prob["F"], prob["u0"])).max() + S)
            err = np.abs(r_pair - r_ex).max()
            print(f"p={p} z={z:.1e} cycle {k + 1}: |r|={np.abs(r_ex).max():.2e} pair err={err:.2e}")
            assert err <= allow, (err, allow)


@pytest.mark.parametrize("p", [1, 3])
def test_updated_residual_over_several_cycles_at_multi_tile_size(dev, p):
    """The same comparison after 6 cycles that each update the residual of
    the previous one (no recomputation from u: tol = 0, max_cycles = 6), at a
    size where every warp of the level-0 kernel processes several tiles
    (2^21 + 64 intervals): the halo lanes of a tile then read pairs that other
    warps update in the same launch.  The allowance adds up the per-cycle
    rounding of the update and of u += c, 6 x 1e-13 S, and the storage of the
    low parts, 2^-39 of each stored residual: at most 2^-39 sum_k |r_k| <=
    2^-37 max|F| for residuals that shrink by a factor <= 1/2 per cycle."""
    N = (1 << 21) + 64
    prob = inputs.scalar_problem(40 + p, N, p, lam=1.0, tau=1e-6, u0=1.0)
    z = prob["tau"]
    Fd = torch.from_numpy(prob["F"]).to(dev)
    with tmg().Plan(p, prob["tau"], 1.0, N, precision="mixed", tol=0.0, max_cycles=6) as plan:
        u = plan.solve(Fd, prob["u0"], allow_notconv=True)
        assert plan.stats().cycles == 6
        uh = u.cpu().numpy()
        r_pair = plan.inspect("r").astype(np.float64) + plan.inspect("rlo").astype(np.float64)
    r_ex = O.residual(p, z, prob["F"], prob["u0"], uh)
    S = (2 + z) * (p + 1) * np.abs(uh).max()
    allow = 6e-13 * S + 2.0 ** -37 * np.abs(O.fold_u0(p, prob["F"], prob["u0"])).max()
    err = np.abs(r_pair - r_ex).max()
    print(f"p={p} N={N}: |r|={np.abs(r_ex).max():.2e} pair err after 6 cycles={err:.2e}")
    assert err <= allow, (err, allow)


@pytest.mark.parametrize("p", [0, 1, 3])
def test_updated_and_recomputed_residual_forms_agree(dev, p):
    """The two mixed forms (residual updated between cycles, or recomputed
    from u in FP64 every cycle) take the same number of cycles up to one, both
    meet the tolerance, and their solutions differ by no more than the
    tolerance allows: cond(L) ~ 2/z times 1e-10 relative (z = 0.05 here)."""
    N = 1 << 14
    lam = 0.05 * N
    prob = inputs.scalar_problem(30 + p, N, p, lam=lam, T=1.0, u0=1.0)
    z = lam * prob["tau"]
    Fd = torch.from_numpy(prob["F"]).to(dev)
    res = {}
    for upd in (True, False):
        with tmg().Plan(p, prob["tau"], lam, N, precision="mixed", update_residual=upd, max_cycles=300) as plan:
            u = plan.solve(Fd, prob["u0"]).cpu().numpy()
            res[upd] = (u, plan.stats())
        assert rel_residual(p, z, prob["F"], prob["u0"], u) <= 1.05e-10
    (u1, s1), (u0_, s0) = res[True], res[False]
    print(f"p={p}: cycles updated={s1.cycles} recomputed={s0.cycles} diff={rel_err(u1, u0_):.2e}")
    assert abs(s1.cycles - s0.cycles) <= 1
    assert rel_err(u1, u0_) <= 2.0 / z * 1e-10 * 4
    # the solve stops on a residual confirmed from u: the reported value is the
    # FP64 residual of the returned u (FP32 norm: 1e-4 relative)
    assert s1.rel_res == pytest.approx(rel_residual(p, z, prob["F"], prob["u0"], u1), rel=1e-4)


def test_confirmation_rejects_an_updated_residual_below_the_fp64_floor(dev):
    """A tolerance below what FP64 can confirm: the updated residual may drop
    under it, but the FP64 residual from u cannot, so the solve must run to
    max_cycles and report TMG_ENOTCONV instead of stopping early."""
    N, p = 1 << 13, 1
    prob = inputs.scalar_problem(7, N, p, lam=1.0, T=1.0, u0=1.0)
    Fd = torch.from_numpy(prob["F"]).to(dev)
    T_ = tmg()
    with T_.Plan(p, prob["tau"], 1.0, N, precision="mixed", tol=1e-19, max_cycles=40) as plan:
        u = plan.solve(Fd, prob["u0"], allow_notconv=True)
        assert plan.last_status == T_.TMG_ENOTCONV
        st = plan.stats()
    assert st.cycles == 40
    assert rel_residual(p, prob["tau"], prob["F"], prob["u0"], u.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_input_reports_numeric_error_and_plan_stays_usable(dev, prec, bad):
    """A non-finite value in f makes the first residual norm non-finite: the
    solve stops at once with TMG_ENUMERIC (no cycles run on garbage), and the
    same plan then solves a clean problem."""
    N, p = 1 << 12, 1
    prob = inputs.scalar_problem(8, N, p, lam=1.0, T=1.0, u0=1.0)
    T_ = tmg()
    F_bad = prob["F"].copy()
    F_bad[N // 3, 1] = bad
    with T_.Plan(p, prob["tau"], 1.0, N, precision=prec) as plan:
        with pytest.raises(T_.TmgError) as ei:
            plan.solve(torch.from_numpy(F_bad).to(dev), prob["u0"])
        assert ei.value.status == T_.TMG_ENUMERIC
        assert plan.stats().cycles == 0
        u = plan.solve(torch.from_numpy(prob["F"]).to(dev), prob["u0"]).cpu().numpy()
    assert rel_residual(p, prob["tau"], prob["F"], prob["u0"], u) <= 1.05e-10


def test_plan_on_a_torch_stream_orders_after_the_current_stream(dev):
    """A plan created on a caller's (non-blocking) torch stream: the load
    vector written by torch on the current stream just before the call must be
    complete when the solve reads it."""
    N, p = 1 << 20, 1
    prob = inputs.scalar_problem(14, N, p, lam=1.0, tau=1e-6, u0=1.0)
    src = torch.from_numpy(prob["F"]).to(dev)
    s = torch.cuda.Stream(device=dev)
    with tmg().Plan(p, 1e-6, 1.0, N, precision="mixed", stream=s) as plan:
        for k in range(3):
            F = torch.zeros_like(src)
            F.copy_(src)                       # queued on the current stream, no host sync
            F.mul_(1.0 + k)                    # the solve must see the scaled load vector
            u = plan.solve(F, prob["u0"] * (1.0 + k))
            assert rel_residual(p, 1e-6, prob["F"] * (1.0 + k), prob["u0"] * (1.0 + k),
                                u.cpu().numpy()) <= 1.05e-10


@pytest.mark.slow
def test_largest_size_ragged_hierarchy(dev):
    """A horizon six times the benchmark's: N = 3 * 2^25 (about 10^8 intervals,
    1.6 GB load vector), whose hierarchy ends on a 48-interval level; the FP64
    residual of the whole result by the oracle, and sampled intervals against
    exact forward substitution."""
    N, p, tau = 3 << 25, 1, 1e-6
    rng = np.random.default_rng(77)
    A = rng.uniform(-1.0, 1.0, (1, 4))
    K = rng.integers(1, 9, (1, 4)).astype(float)
    F = inputs.sine_load_vectors(A, K, N * tau, N, p, device=dev)[0]
    with tmg().Plan(p, tau, 1.0, N, precision="mixed", nu1=2, nu2=2) as plan:
        info = plan.info()
        u = plan.solve(F, 1.0)
        st = plan.stats()
    assert info["levels"] == 22 and (N >> (info["levels"] - 1)) == 48
    Fh, uh = F.cpu().numpy(), u.cpu().numpy()
    del F, u
    rr = rel_residual(p, tau, Fh, 1.0, uh)
    assert rr <= 1.05e-10, rr
    ex = O.fsub(p, tau, Fh, 1.0)
    idx = np.concatenate([rng.integers(0, N, 4096), [0, 1, N // 2, N - 2, N - 1]])
    err = np.abs(uh[idx] - ex[idx]).max() / np.abs(ex).max()
    print(f"N={N}: cycles={st.cycles} rel_res={rr:.2e} sampled err={err:.2e}")
    assert err <= 1e-6


def test_launch_count_per_cycle(dev):
    """tmg_plan_launches counts the kernels of one cycle: for the benchmark's
    structure (mixed, V(2,2), 2^20 intervals, 15 levels, coarsest 64 intervals)
    that is k_down0, 6 two-level down kernels (levels 1-12), the single level
    13 (whose last block solves the coarsest level), its up kernel, 6 two-level
    up kernels and k_updown0: 16."""
    N = 1 << 20
    prob = inputs.scalar_problem(3, N, 1, lam=1.0, tau=1e-6, u0=1.0)
    with tmg().Plan(1, 1e-6, 1.0, N, precision="mixed", nu1=2, nu2=2) as plan:
        assert plan.launches_per_cycle() == 0
        plan.solve(torch.from_numpy(prob["F"]).to(dev), 1.0)
        info = plan.info()
        assert info["levels"] == 15 and info["tail_level"] == 14
        assert plan.launches_per_cycle() == 16


@pytest.mark.parametrize("p,N,kw", [
    (1, 1 << 24, {"n_min": 1 << 17}), (1, 1 << 14, {}), (0, 4096, {"gamma": 2}),
    (1, 1 << 14, {"gamma": 2, "tail_cap": 128}), (2, 1 << 16, {"n_min": 16384}), (1, 3 * 1024, {"n_min": 2}),
    (10, 1 << 12, {"precision": "fp64"}), (10, 37, {})])
def test_plan_shape_matches_the_plan_setup_builds(dev, p, N, kw):
    """tmg_plan_shape (host only) reports the hierarchy tmg_setup builds."""
    T = tmg()
    s = T.plan_shape(p, 1e-3, 1.0, N, **kw)
    with T.Plan(p, 1e-3, 1.0, N, **kw) as plan:
        info = plan.info()
    assert (s["levels"], s["tail_level"], s["tail_intervals"]) == (info["levels"], info["tail_level"],
                                                                    info["tail_intervals"])


@pytest.mark.parametrize("p,N,lam", [(1, 1 << 14, 1.0), (3, 4096, 200.0), (0, 1001, 5.0), (10, 2048, 3.0)])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_error_against_fp64_is_reported(dev, p, N, lam, prec):
    """opts.check_fp64: tmg_stats reports max|u - u_exact| / max|u_exact| of
    the solve against the exact FP64 solve; it agrees with the same error taken
    against the oracle's forward substitution, up to the exact solves' own
    difference (a few N eps, from the rounding of alpha in the recurrence)."""
    prob = inputs.scalar_problem(N + 1, N, p, lam=lam, T=1.0, u0=0.4)
    z = lam * prob["tau"]
    Fd = torch.from_numpy(prob["F"]).to(dev)
    with tmg().Plan(p, prob["tau"], lam, N, precision=prec, tol=1e-10, check_fp64=True) as plan:
        u = plan.solve(Fd, prob["u0"]).cpu().numpy()
        st = plan.stats()
    with tmg().Plan(p, prob["tau"], lam, N, precision=prec, tol=1e-10) as plan:
        plan.solve(Fd, prob["u0"])
        assert np.isnan(plan.stats().err_vs_fp64)
    ex = O.fsub(p, z, prob["F"], prob["u0"])
    err_or = rel_err(u, ex)
    assert np.isfinite(st.err_vs_fp64)
    assert abs(st.err_vs_fp64 - err_or) <= max(2e-13, 8 * N * 2.2e-16) + 1e-6 * err_or, (st.err_vs_fp64, err_or)
