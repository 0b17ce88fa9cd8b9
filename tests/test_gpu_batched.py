"""Batched solves (tmg_setup_batched / tmg_solve_batched / tmg_adjoint_batched)
against the oracle, instance by instance.

Tolerances: each instance stops at its own relative residual <= tol; the test
evaluates that residual with the oracle in FP64 (<= 1.05 tol) and the error
against forward substitution, which is at most cond(L_i) * tol with
cond(L_i) <= 2/z_i (bounded by 2 N_i): the allowance is 2 N_i tol.
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


def make_batch(seed, p, N, z):
    """Packed load vectors on (0, 1) per instance, tau_i = 1/N_i, lambda_i = z_i N_i."""
    rng = np.random.default_rng(seed)
    Fs, u0 = [], rng.standard_normal(len(p))
    for i in range(len(p)):
        forcing = inputs.Forcing.draw(rng, 1.0)
        Fs.append(inputs.load_vector(int(p[i]), int(N[i]), 1.0, forcing))
    tau = 1.0 / np.asarray(N, dtype=np.float64)
    lam = np.asarray(z) / tau
    return Fs, u0, tau, lam


def check_solution(Fs, u0, tau, lam, p, N, u_packed, batch, tol):
    us = batch.split(u_packed)
    worst = 0.0
    for i in range(len(p)):
        z = lam[i] * tau[i]
        r = O.residual(int(p[i]), z, Fs[i], u0[i], us[i])
        rel = np.linalg.norm(r) / np.linalg.norm(O.fold_u0(int(p[i]), Fs[i], u0[i]))
        assert rel <= 1.05 * tol, (i, rel)
        ex = O.fsub(int(p[i]), z, Fs[i], u0[i])
        err = np.abs(us[i] - ex).max() / np.abs(ex).max()
        assert err <= 2 * N[i] * tol, (i, err)
        worst = max(worst, err)
    return worst


def group_length(N, n_min=64):
    """The length of the system the batched solver solves for an instance of
    N intervals.  An instance whose own hierarchy (coarsen while even and
    longer than nmin = min(n_min, 64) intervals) coarsens at least once down
    to at most nmin intervals is solved on its own N intervals; any other is
    padded at its end to a power of two (at least 2) with a zero right-hand
    side."""
    nmin = min(n_min, 64)
    s, m = 0, N
    while m % 2 == 0 and m > nmin:
        m //= 2
        s += 1
    if s >= 1 and m <= nmin:
        return N
    Ng = 2
    while Ng < N:
        Ng *= 2
    return Ng


def oracle_batched_iterates(p, z, F, u0, k, n_min=64, **kw):
    """The oracle's textbook cycle (eq. chap4_errorTwoGridCycle) applied k
    times to the instance as the batched solver holds it (group_length),
    coarsened while a level is even and longer than min(n_min, 64)
    intervals; the first N intervals of each iterate."""
    N = F.shape[0]
    Fh = np.zeros((group_length(N, n_min), p + 1))
    Fh[:N] = O.fold_u0(p, F, u0)
    u = np.zeros_like(Fh)
    out = []
    for _ in range(k):
        u = O.mg_one_cycle(p, z, Fh, u, n_min=min(n_min, 64), **kw)
        out.append(u[:N].copy())
    return out


BATCH_CYCLE_N = [1, 2, 3, 5, 64, 100, 1001, 4096, 16384, 12000, 777, 2048, 96, 33, 8192, 300, 5000, 130]


def test_uneven_lengths_are_not_padded():
    """The uneven-batch recipe rounds every N to m 2^s with m in (32, 64]: each
    such instance is solved on its own intervals (no padding beyond 5%: only
    the instances of at most 64 intervals are padded)."""
    N, p, z = inputs.uneven_batch(3, 10000)
    real = int((N * (p + 1)).sum())
    solved = sum(group_length(int(n)) * (int(q) + 1) for n, q in zip(N, p))
    assert solved <= 1.05 * real


@pytest.mark.parametrize("schedule", ["grid", "cta"])
@pytest.mark.parametrize("nu", [(1, 1), (2, 2), (0, 2), (3, 1)])
def test_batched_fp64_cycles_match_textbook_cycle(dev, schedule, nu):
    """Iterate-level parity of the batched FP64 path with the paper's cycle:
    an uneven batch (p_t = 0..5, lengths 1 .. 16384 including non-powers of
    two, z = 1e-3 .. 1e3) run for exactly k = 1, 2, 3 cycles (tol = 0,
    max_cycles = k) in each schedule, every instance against k applications
    of the oracle's textbook cycle on that instance's own hierarchy, 1e-12
    relative.  The CTA form takes the groups that fit one CTA (the others fall
    back to the grid form)."""
    from paper_1409_5254_gb300 import tmg
    rng = np.random.default_rng(31 + nu[0] + 4 * nu[1])
    N = np.array(BATCH_CYCLE_N)
    p = np.arange(len(N)) % 6
    z = 10.0 ** rng.uniform(-3, 3, len(N))
    Fs, u0, tau, lam = make_batch(31, p, N, z)
    f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
    u0d = torch.from_numpy(u0).to(dev)
    sched = tmg.SCHED_GRID if schedule == "grid" else tmg.SCHED_CTA
    ref = [oracle_batched_iterates(int(p[i]), lam[i] * tau[i], Fs[i], u0[i], 3, nu1=nu[0], nu2=nu[1])
           for i in range(len(N))]
    for k in (1, 2, 3):
        with tmg.Batch(p, tau, lam, N, precision="fp64", tol=0.0, max_cycles=k, schedule=sched, nu1=nu[0],
                       nu2=nu[1]) as B:
            u = B.solve(f, u0d, allow_notconv=True)
            cyc, rel, mx = B.stats()
            kinds = {g["schedule"] for g in B.info()["group_info"]}
            us = B.split(u.cpu().numpy())
        assert kinds == ({"grid"} if schedule == "grid" else {"grid", "cta"}), kinds
        for i in range(len(N)):
            # an instance whose residual is exactly zero stops early, as it should
            c = int(cyc[i])
            assert 1 <= c <= k and (c == k or rel[i] == 0.0), (i, c, rel[i])
            e = np.abs(us[i] - ref[i][c - 1]).max() / max(np.abs(ref[i][c - 1]).max(), 1e-300)
            assert e <= 1e-12, (k, i, int(p[i]), int(N[i]), z[i], e)


@pytest.mark.parametrize("schedule,cap", [("grid", 0), ("grid", 8192), ("cta", 0)])
@pytest.mark.parametrize("nu", [(1, 1), (2, 1)])
def test_batched_w_cycles_match_textbook_cycle(dev, schedule, cap, nu):
    """W-cycles (gamma = 2) in the batched solve at the iterate level: every
    level below level 0 visited twice per visit of its parent, the second
    visit from the first one's result.  The grid form launches the streaming
    levels once per visit down to the first level of at most tail_cap
    intervals (the default 2048, and 8192) and runs the rest in one CTA per
    instance; the CTA form runs the whole
    recursion on chip.  Against k = 1, 2, 3 applications of the oracle's
    textbook W-cycle (eq. chap4_errorTwoGridCycle recursed twice per level),
    1e-12 relative; lengths up to 2^16 so that the grid form has streaming
    W levels above its on-chip part."""
    from paper_1409_5254_gb300 import tmg
    rng = np.random.default_rng(47 + nu[0])
    N = np.array([65536, 40000, 16384, 9000, 4096, 777, 100, 5, 1, 33000, 2048, 65])
    p = np.array([0, 1, 0, 2, 3, 0, 1, 0, 2, 0, 5, 4])
    z = 10.0 ** rng.uniform(-3, 3, len(N))
    Fs, u0, tau, lam = make_batch(47, p, N, z)
    f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
    u0d = torch.from_numpy(u0).to(dev)
    sched = tmg.SCHED_GRID if schedule == "grid" else tmg.SCHED_CTA
    ref = [oracle_batched_iterates(int(p[i]), lam[i] * tau[i], Fs[i], u0[i], 3, nu1=nu[0], nu2=nu[1], gamma=2)
           for i in range(len(N))]
    for k in (1, 2, 3):
        with tmg.Batch(p, tau, lam, N, precision="fp64", tol=0.0, max_cycles=k, schedule=sched, nu1=nu[0],
                       nu2=nu[1], gamma=2, tail_cap=cap) as B:
            u = B.solve(f, u0d, allow_notconv=True)
            cyc, rel, mx = B.stats()
            us = B.split(u.cpu().numpy())
        for i in range(len(N)):
            c = int(cyc[i])
            assert 1 <= c <= k and (c == k or rel[i] == 0.0), (i, c, rel[i])
            e = np.abs(us[i] - ref[i][c - 1]).max() / max(np.abs(ref[i][c - 1]).max(), 1e-300)
            assert e <= 1e-12, (k, i, int(p[i]), int(N[i]), z[i], e)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batched_w_cycles_reach_tolerance_in_fewer_cycles_at_degree_0(dev, prec):
    """The point of W-cycles at p_t = 0, where V-cycles degrade with depth
    (the paper's Section 7): a batch of p_t = 0 instances of 2^12 .. 2^16
    intervals, lambda tau = 1e-3 .. 1, solved to 1e-10 with V(2,2) and with
    W(2,2); the W solve needs fewer cycles and meets the oracle's residual."""
    from paper_1409_5254_gb300 import tmg
    rng = np.random.default_rng(53)
    N = np.array([4096, 8192, 16384, 32768, 65536, 12288, 40960, 65536])
    p = np.zeros(len(N), dtype=int)
    z = 10.0 ** rng.uniform(-3, 0, len(N))
    Fs, u0, tau, lam = make_batch(53, p, N, z)
    f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
    out = {}
    for gamma in (1, 2):
        with tmg.Batch(p, tau, lam, N, precision=prec, tol=1e-10, max_cycles=300, nu1=2, nu2=2, gamma=gamma,
                       schedule=tmg.SCHED_GRID) as B:
            u = B.solve(f, torch.from_numpy(u0).to(dev))
            cyc, rel, mx = B.stats()
            out[gamma] = (mx, B.split(u.cpu().numpy()), B)
        assert (rel <= 1e-10).all()
    check_solution(Fs, u0, tau, lam, p, N, np.concatenate([x.reshape(-1) for x in out[2][1]]), out[2][2], 1e-10)
    print(f"p_t = 0 {prec}: V(2,2) {out[1][0]} cycles, W(2,2) {out[2][0]} cycles")
    assert out[2][0] < out[1][0]


def test_wide_degree_batch_fp64_cycles_match_textbook_cycle(dev):
    """p_t = 10 and 20 instances (with p_t = 1 ones) in one batch: per-level
    kernels, the residual recomputed from u; FP64 iterates after 1, 2, 3
    cycles against the oracle's textbook cycle on each instance, 1e-12."""
    from paper_1409_5254_gb300 import tmg
    N = np.array([4096, 1000, 64, 3, 2048, 700, 1, 8192])
    p = np.array([10, 20, 10, 20, 20, 10, 20, 1])
    z = np.array([1e-3, 0.5, 30.0, 1.0, 1e-2, 1e3, 2.0, 0.1])
    Fs, u0, tau, lam = make_batch(61, p, N, z)
    f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
    u0d = torch.from_numpy(u0).to(dev)
    ref = [oracle_batched_iterates(int(p[i]), lam[i] * tau[i], Fs[i], u0[i], 3) for i in range(len(N))]
    for k in (1, 2, 3):
        with tmg.Batch(p, tau, lam, N, precision="fp64", tol=0.0, max_cycles=k) as B:
            u = B.solve(f, u0d, allow_notconv=True)
            cyc, rel, mx = B.stats()
            us = B.split(u.cpu().numpy())
        for i in range(len(N)):
            c = int(cyc[i])
            assert 1 <= c <= k and (c == k or rel[i] == 0.0), (i, c, rel[i])
            e = np.abs(us[i] - ref[i][c - 1]).max() / max(np.abs(ref[i][c - 1]).max(), 1e-300)
            assert e <= 1e-12, (k, i, int(p[i]), int(N[i]), z[i], e)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_wide_degree_batch_solve_and_adjoint(dev, prec):
    """A batch of p_t = 10 and 20 instances solved to tolerance (every
    instance at the oracle's residual) and its gradients through the adjoint
    against the oracle's backward sweep and gradient formulas."""
    from paper_1409_5254_gb300 import tmg
    N = np.array([4096, 2048, 300, 1024, 5000, 64])
    p = np.array([10, 20, 10, 20, 10, 20])
    z = np.array([1e-2, 0.3, 5.0, 1e-1, 2e-3, 40.0])
    Fs, u0, tau, lam = make_batch(67, p, N, z)
    tol = 1e-12 if prec == "fp64" else 1e-10
    rng = np.random.default_rng(67)
    with tmg.Batch(p, tau, lam, N, precision=prec, tol=tol, max_cycles=300) as B:
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        cyc, rel, mx = B.stats()
        assert (rel <= tol).all(), rel
        us = B.split(u.cpu().numpy())
        gs = []
        for i in range(len(p)):
            _, _, _, b = O.blocks(int(p[i]))
            gs.append(np.outer(O.nodal_values(int(p[i]), us[i]) - rng.standard_normal(int(N[i])), b))
        g = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gs])).to(dev)
        dJdf, du0, dlam = B.adjoint(g, u)
    check_solution(Fs, u0, tau, lam, p, N, u.cpu().numpy(), B, tol)
    mus = B.split(dJdf.cpu().numpy())
    du0, dlam = du0.cpu().numpy(), dlam.cpu().numpy()
    for i in range(len(p)):
        zi = lam[i] * tau[i]
        allow = 2.0 * max(N[i], 1.0 / zi) * tol * 10
        mu_ref = O.adj_sweep(int(p[i]), zi, gs[i])
        assert np.abs(mus[i] - mu_ref).max() <= allow * np.abs(mu_ref).max(), i
        _, d0, dl = O.adjoint_grads(int(p[i]), lam[i], tau[i], gs[i], us[i])
        assert du0[i] == pytest.approx(d0, rel=allow, abs=1e-12)
        assert dlam[i] == pytest.approx(dl, rel=allow, abs=1e-12)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batched_error_against_fp64_is_reported(dev, prec):
    """opts.check_fp64 on a batch: per-instance max|u_i - u_exact,i| /
    max|u_exact,i| against the exact FP64 solve (one warp per instance, chunk
    maps scanned across the warp), equal to the same error taken against the
    oracle's forward substitution up to the exact solves' own difference."""
    from paper_1409_5254_gb300 import tmg
    N, p, z = inputs.uneven_batch(41, 30, nmin_exp=0.0, nmax_exp=14.0)
    Fs, u0, tau, lam = make_batch(41, p, N, z)
    f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
    with tmg.Batch(p, tau, lam, N, precision=prec, tol=1e-10, max_cycles=300, check_fp64=True) as B:
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        err = B.err_vs_fp64()
        us = B.split(u.cpu().numpy())
    for i in range(len(p)):
        ex = O.fsub(int(p[i]), lam[i] * tau[i], Fs[i], u0[i])
        err_or = np.abs(us[i] - ex).max() / np.abs(ex).max()
        assert abs(err[i] - err_or) <= max(2e-13, 8 * N[i] * 2.2e-16) + 1e-6 * err_or, (i, err[i], err_or)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_uniform_batch(dev, prec):
    from paper_1409_5254_gb300 import tmg
    n, p, N = 96, 1, 2048
    z = 10.0 ** np.random.default_rng(1).uniform(-3, 2, n)
    Fs, u0, tau, lam = make_batch(1, [p] * n, [N] * n, z)
    with tmg.Batch([p] * n, tau, lam, [N] * n, precision=prec, tol=1e-10, max_cycles=200) as B:
        assert B.info()["groups"] == 1
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        cyc, rel, mx = B.stats()
    assert (rel <= 1e-10).all()
    err = check_solution(Fs, u0, tau, lam, [p] * n, [N] * n, u.cpu().numpy(), B, 1e-10)
    print(f"uniform {prec}: max cycles {mx}, worst err {err:.2e}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nu", [(1, 1), (2, 2), (3, 1), (0, 2)])
def test_two_level_kernels_match_one_level(dev, prec, nu):
    """The grid schedule's streaming levels two per kernel (kb_down2/kb_up2,
    each lane four intervals, the halo restarting at every instance) against
    one level per kernel: the same cycles, solutions within rounding of each
    other, and both at the oracle's residual.  Lengths 256 .. 16384 give 1 to
    7 streaming levels: pairs and a single level, instance boundaries inside
    the lanes' windows."""
    from paper_1409_5254_gb300 import tmg
    rng = np.random.default_rng(11)
    N = [int(x) for x in 2 ** rng.integers(8, 15, 24)]
    p = [int(x) for x in rng.integers(0, 4, 24)]
    z = 10.0 ** rng.uniform(-3, 1, 24)
    Fs, u0, tau, lam = make_batch(11, p, N, z)
    f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
    out = {}
    for fuse in (True, False):
        with tmg.Batch(p, tau, lam, N, precision=prec, tol=1e-10, max_cycles=300, nu1=nu[0], nu2=nu[1],
                       fuse_levels=fuse, schedule=1) as B:
            u = B.solve(f, torch.from_numpy(u0).to(dev)).cpu().numpy()
            cyc, rel, mx = B.stats()
            out[fuse] = (u, cyc, B)
    assert np.abs(out[True][1] - out[False][1]).max() <= 1
    err = check_solution(Fs, u0, tau, lam, p, N, out[True][0], out[True][2], 1e-10)
    print(f"two-level {prec} nu={nu}: max cycles {out[True][1].max()}, worst err {err:.2e}")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_tiny_instances_in_a_batch(dev, prec):
    """Instances of 1, 2, 3 and 5 intervals (padded groups of 2 to 8
    intervals, a single level: the exact warp solve and u += c) next to
    larger ones, every degree; each against the oracle."""
    from paper_1409_5254_gb300 import tmg
    N = [1, 2, 3, 5, 1, 2, 64, 300, 1, 4096]
    p = [0, 1, 2, 3, 5, 4, 1, 2, 3, 1]
    z = [1.0, 0.1, 10.0, 1e-3, 2.0, 50.0, 0.5, 1e-2, 1e3, 1e-3]
    Fs, u0, tau, lam = make_batch(17, p, N, z)
    with tmg.Batch(p, tau, lam, N, precision=prec, tol=1e-10, max_cycles=300) as B:
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        cyc, rel, mx = B.stats()
    assert (rel <= 1e-10).all(), rel
    check_solution(Fs, u0, tau, lam, p, N, u.cpu().numpy(), B, 1e-10)


def test_uneven_batch_matches_oracle(dev):
    """Different degrees, lengths (not powers of two) and steps in one batch."""
    from paper_1409_5254_gb300 import tmg
    N, p, z = inputs.uneven_batch(3, 40, nmin_exp=3.0, nmax_exp=12.0)
    Fs, u0, tau, lam = make_batch(3, p, N, z)
    with tmg.Batch(p, tau, lam, N, precision="mixed", tol=1e-10, max_cycles=300) as B:
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        info = B.info()
    assert info["groups"] >= 4
    check_solution(Fs, u0, tau, lam, p, N, u.cpu().numpy(), B, 1e-10)


@pytest.mark.parametrize("nu", [(2, 2), (1, 3), (3, 1)])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_uneven_batch_other_sweep_counts(dev, nu, prec):
    """The batched kernels with more smoothing sweeps (wider halos per tile):
    every instance of an uneven batch against the oracle."""
    from paper_1409_5254_gb300 import tmg
    N, p, z = inputs.uneven_batch(7, 24, nmin_exp=3.0, nmax_exp=12.0)
    Fs, u0, tau, lam = make_batch(7, p, N, z)
    with tmg.Batch(p, tau, lam, N, precision=prec, tol=1e-10, max_cycles=300, nu1=nu[0], nu2=nu[1]) as B:
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        cyc, rel, mx = B.stats()
    assert (rel <= 1e-10).all()
    check_solution(Fs, u0, tau, lam, p, N, u.cpu().numpy(), B, 1e-10)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("schedule", ["cta", "grid", "auto"])
def test_schedules_match_oracle(dev, prec, schedule):
    """The two batched schedules -- level kernels over a whole group, or one
    CTA per instance with its hierarchy in shared memory and every cycle in one
    launch -- and the setup autotuner that picks between them, on an uneven
    batch of small and large instances; every instance against the oracle."""
    from paper_1409_5254_gb300 import tmg
    N, p, z = inputs.uneven_batch(11, 40, nmin_exp=2.0, nmax_exp=13.0)
    Fs, u0, tau, lam = make_batch(11, p, N, z)
    sched = {"auto": tmg.SCHED_AUTO, "grid": tmg.SCHED_GRID, "cta": tmg.SCHED_CTA}[schedule]
    with tmg.Batch(p, tau, lam, N, precision=prec, tol=1e-10, max_cycles=300, schedule=sched, nu1=2, nu2=2) as B:
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        cyc, rel, mx = B.stats()
        info = B.info()
    assert (rel <= 1e-10).all()
    check_solution(Fs, u0, tau, lam, p, N, u.cpu().numpy(), B, 1e-10)
    kinds = [g["schedule"] for g in info["group_info"]]
    small = [g for g in info["group_info"] if g["padded_length"] <= 256]
    assert small, info
    if schedule == "grid":
        assert set(kinds) == {"grid"}
    elif schedule == "cta":
        assert all(g["schedule"] == "cta" for g in small)
    else:
        # every group that fits one CTA was timed both ways; it runs the faster
        # form, unless the whole concurrent batch ran faster with every group on
        # the grid form (the setup's second check), which then applies to all
        whole = info["whole_batch_ms"]
        for g in small:
            assert np.isfinite(g["ms_grid"]) and np.isfinite(g["ms_cta"])
        if np.isfinite(whole["tuned"]) and whole["all_grid"] < whole["tuned"]:
            assert set(kinds) == {"grid"}
        else:
            for g in small:
                assert g["schedule"] == ("cta" if g["ms_cta"] < g["ms_grid"] else "grid")
        timed = [g for g in info["group_info"] if np.isfinite(g["ms_cta"]) and np.isfinite(g["ms_grid"])]
        if not any(g["ms_cta"] < g["ms_grid"] for g in timed):
            assert not np.isfinite(whole["tuned"])     # no CTA choice: the whole-batch check does not run
    print(schedule, prec, [(g["p_t"], g["padded_length"], g["schedule"], round(g["ms_grid"], 3),
                            round(g["ms_cta"], 3)) for g in info["group_info"]])


def test_cta_schedule_adjoint_matches_oracle(dev):
    """Gradients through the CTA-per-instance schedule (reversed-time solves)."""
    from paper_1409_5254_gb300 import tmg
    N, p, z = inputs.uneven_batch(12, 16, nmin_exp=4.0, nmax_exp=10.0)
    Fs, u0, tau, lam = make_batch(12, p, N, z)
    rng = np.random.default_rng(3)
    with tmg.Batch(p, tau, lam, N, precision="mixed", tol=1e-10, max_cycles=300, schedule=tmg.SCHED_CTA) as B:
        assert all(g["schedule"] == "cta" for g in B.info()["group_info"])
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        us = B.split(u.cpu().numpy())
        gs = []
        for i in range(len(p)):
            _, _, _, b = O.blocks(int(p[i]))
            gs.append(np.outer(O.nodal_values(int(p[i]), us[i]) - rng.standard_normal(int(N[i])), b))
        g = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gs])).to(dev)
        dJdf, du0, dlam = B.adjoint(g, u)
    mus = B.split(dJdf.cpu().numpy())
    du0, dlam = du0.cpu().numpy(), dlam.cpu().numpy()
    for i in range(len(p)):
        zi = lam[i] * tau[i]
        allow = 2.0 * max(N[i], 1.0 / zi) * 1e-10 * 10
        mu_ref = O.adj_sweep(int(p[i]), zi, gs[i])
        assert np.abs(mus[i] - mu_ref).max() <= allow * np.abs(mu_ref).max(), i
        _, d0, dl = O.adjoint_grads(int(p[i]), lam[i], tau[i], gs[i], us[i])
        assert du0[i] == pytest.approx(d0, rel=allow, abs=1e-12)
        assert dlam[i] == pytest.approx(dl, rel=allow, abs=1e-12)


@pytest.mark.parametrize("schedule", ["grid", "cta"])
def test_higher_degree_batch(dev, schedule):
    """p_t = 4 and 5 instances (with one of p_t = 1) in both schedules."""
    from paper_1409_5254_gb300 import tmg
    rng = np.random.default_rng(21)
    p = np.array([4, 5, 4, 5, 1, 5, 4, 4])
    N = np.array([64, 96, 256, 512, 128, 1024, 32, 200])
    z = 10.0 ** rng.uniform(-3, 2, len(p))
    Fs, u0, tau, lam = make_batch(21, p, N, z)
    sched = tmg.SCHED_GRID if schedule == "grid" else tmg.SCHED_CTA
    with tmg.Batch(p, tau, lam, N, precision="mixed", tol=1e-10, max_cycles=300, schedule=sched) as B:
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        cyc, rel, mx = B.stats()
    assert (rel <= 1e-10).all()
    check_solution(Fs, u0, tau, lam, p, N, u.cpu().numpy(), B, 1e-10)


def test_batch_of_one_matches_single_solve(dev):
    from paper_1409_5254_gb300 import tmg
    prob = inputs.scalar_problem(4, 4096, 2, lam=3.0, T=1.0, u0=0.5)
    F = torch.from_numpy(prob["F"]).to(dev)
    with tmg.Plan(2, prob["tau"], 3.0, 4096, precision="fp64", tol=1e-12) as plan:
        u1 = plan.solve(F, 0.5).cpu().numpy()
    with tmg.Batch([2], [prob["tau"]], [3.0], [4096], precision="fp64", tol=1e-12) as B:
        u2 = B.solve(F.reshape(-1), torch.tensor([0.5], dtype=torch.float64, device=dev)).cpu().numpy()
    ex = O.fsub(2, 3.0 * prob["tau"], prob["F"], 0.5)
    assert np.abs(u2.reshape(-1, 3) - ex).max() <= 1e-9 * np.abs(ex).max()
    assert np.abs(u1 - ex).max() <= 1e-9 * np.abs(ex).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_adjoint_matches_oracle(dev, prec):
    from paper_1409_5254_gb300 import tmg
    N, p, z = inputs.uneven_batch(5, 12, nmin_exp=4.0, nmax_exp=11.0)
    Fs, u0, tau, lam = make_batch(5, p, N, z)
    tol = 1e-12 if prec == "fp64" else 1e-10
    rng = np.random.default_rng(9)
    with tmg.Batch(p, tau, lam, N, precision=prec, tol=tol, max_cycles=400) as B:
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev)
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        us = B.split(u.cpu().numpy())
        gs = []
        for i in range(len(p)):
            _, _, _, b = O.blocks(int(p[i]))
            y = rng.standard_normal(int(N[i]))
            gs.append(np.outer(O.nodal_values(int(p[i]), us[i]) - y, b))
        g = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gs])).to(dev)
        dJdf, du0, dlam = B.adjoint(g, u)
    mus = B.split(dJdf.cpu().numpy())
    du0, dlam = du0.cpu().numpy(), dlam.cpu().numpy()
    for i in range(len(p)):
        zi = lam[i] * tau[i]
        allow = 2.0 * max(N[i], 1.0 / zi) * tol * 10
        mu_ref = O.adj_sweep(int(p[i]), zi, gs[i])
        assert np.abs(mus[i] - mu_ref).max() <= allow * np.abs(mu_ref).max(), i
        _, d0, dl = O.adjoint_grads(int(p[i]), lam[i], tau[i], gs[i], us[i])
        assert du0[i] == pytest.approx(d0, rel=allow, abs=1e-12)
        assert dlam[i] == pytest.approx(dl, rel=allow, abs=1e-12)


def _sampled_check(B, f_dev_parts, u, idx, pv, Nv, tau, lam, u0, tol, params):
    """Oracle check of sampled instances; their load vectors are rebuilt on the CPU."""
    us = B.split(u.cpu().numpy())
    A, K, T = params
    for i in idx:
        p, N = int(pv[i]), int(Nv[i])
        F = inputs.sine_load_vectors(A[i:i + 1], K[i:i + 1], T, N, p, device="cpu")[0].numpy()
        z = lam[i] * tau[i]
        r = O.residual(p, z, F, u0[i], us[i])
        rel = np.linalg.norm(r) / np.linalg.norm(O.fold_u0(p, F, u0[i]))
        assert rel <= 1.05 * tol, (i, rel)
        ex = O.fsub(p, z, F, u0[i])
        assert np.abs(us[i] - ex).max() <= 2 * max(N, 1.0 / z) * tol * np.abs(ex).max(), i


def test_full_size_heat_modes_sampled(dev):
    """65,536 decoupled heat modes, N = 4096, p_t = 1, mixed: the benchmark's
    configuration; 8 sampled instances (including the extreme lambdas)."""
    from paper_1409_5254_gb300 import tmg
    lam, amps, freqs = inputs.heat_modes_batch(2, 256, 4096, 1)
    n, N, p = lam.shape[0], 4096, 1
    f = inputs.sine_load_vectors(amps, freqs, 1.0, N, p, device=dev).reshape(-1)
    u0 = np.zeros(n)
    with tmg.Batch([p] * n, 1.0 / N, lam, N, precision="mixed", tol=1e-10, max_cycles=200) as B:
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        cyc, rel, mx = B.stats()
        assert (rel <= 1e-10).all()
        idx = [int(np.argmin(lam)), int(np.argmax(lam))] + list(np.random.default_rng(0).integers(0, n, 6))
        _sampled_check(B, None, u, idx, [p] * n, [N] * n, np.full(n, 1.0 / N), lam, u0, 1e-10, (amps, freqs, 1.0))


def test_full_size_uneven_batch_sampled(dev):
    """10,000 instances, N log-uniform in [2^6, 2^16], p_t in {0..3}, lambda tau
    log-uniform in [1e-3, 1e3], mixed; 12 sampled instances."""
    from paper_1409_5254_gb300 import tmg
    Nv, pv, z = inputs.uneven_batch(3, 10000)
    tau = 1.0 / Nv
    lam = z / tau
    A, K = inputs.sinusoid_batch_params(3, len(Nv))
    f = torch.cat([inputs.sine_load_vectors(A[i:i + 1], K[i:i + 1], 1.0, int(Nv[i]), int(pv[i]),
                                            device=dev).reshape(-1) for i in range(len(Nv))])
    u0 = np.ones(len(Nv))
    with tmg.Batch(pv, tau, lam, Nv, precision="mixed", tol=1e-10, max_cycles=300) as B:
        u = B.solve(f, torch.from_numpy(u0).to(dev))
        cyc, rel, mx = B.stats()
        assert (rel <= 1e-10).all()
        idx = [int(np.argmax(Nv)), int(np.argmin(Nv))] + list(np.random.default_rng(1).integers(0, len(Nv), 10))
        _sampled_check(B, None, u, idx, pv, Nv, tau, lam, u0, 1e-10, (A, K, 1.0))
