"""The time-slab partition (slabs.py) with the library's kernels, on one GPU.

Every run here uses one GPU: the ranks of the partition run in one process,
one after the other (slabs.run_in_process), exchanging the margin and the
coarse problem by copies -- the data the multi-GPU driver sends by
point-to-point messages and all_gather (that driver is tested with gloo ranks
on the CPU in test_slabs.py).  Each rank splits its cycle at the slab level
with tmg_cycle_down / tmg_cycle_up and every rank applies tmg_cycle to the
gathered coarse problem.  The FP64 iterates of the owned slabs must equal the
single-plan tmg_cycle iterates to 1e-12 relative (the same linear map in
another rounding order).
"""
import numpy as np
import pytest

import oracle as O
from paper_1409_5254_gb300 import inputs, slabs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5254_gb300 import build_ext
    build_ext.build()
    return torch.device("cuda:0")


def run(dev, R, p, nu, N, n_min, lam, cycles, precision="fp64"):
    from paper_1409_5254_gb300 import tmg
    prob = inputs.scalar_problem(R + p, N, p, lam=lam, T=1.0, u0=0.6)
    tau = prob["tau"]
    F = torch.from_numpy(prob["F"]).to(dev)
    _, _, _, b = O.blocks(p)
    bt = torch.from_numpy(b).to(dev)
    ranks, backends = [], []
    for r in range(R):
        lay = slabs.slab_layout(N, R, r, *nu, n_min=n_min, coarse_per_slab=64)
        be = slabs.GpuSlabBackend(lay, p, tau, lam, precision=precision, nu1=nu[0], nu2=nu[1], n_min=n_min)
        backends.append(be)
        ranks.append(slabs.SlabRank(lay, be, F[lay.start:lay.b].contiguous(), prob["u0"], bt))
    got, ref = [], []
    with tmg.Plan(p, tau, lam, N, precision=precision, nu1=nu[0], nu2=nu[1], n_min=n_min,
                  update_residual=False) as plan:
        u = torch.zeros_like(F)
        for _ in range(cycles):
            slabs.run_in_process(ranks, 1, backends[0].coarse_cycle)
            got.append(torch.cat([rk.own() for rk in ranks]).cpu().numpy())
            plan.cycle(F, prob["u0"], u)
            ref.append(u.cpu().numpy().copy())
    for be in backends:
        be.close()
    return got, ref, ranks[0].lay


@pytest.mark.parametrize("R,p,nu,N", [(2, 1, (1, 1), 1 << 15), (4, 2, (2, 2), 1 << 16), (3, 0, (2, 1), 3 << 14),
                                      (2, 10, (2, 2), 1 << 13), (8, 3, (1, 2), 1 << 16)])
def test_slab_cycles_match_single_plan_cycles(dev, R, p, nu, N):
    got, ref, lay = run(dev, R, p, nu, N, 64, 2.0, 3)
    assert lay.slab_levels >= 2
    for k in range(3):
        err = np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= 1e-12, (k, err)


def test_slab_cycles_mixed_precision(dev):
    """Mixed form: FP32 cycles inside FP64 residuals; the slab and single-plan
    iterates differ only by FP32 rounding in another order."""
    got, ref, _ = run(dev, 4, 1, (2, 2), 1 << 16, 64, 1.0, 4, precision="mixed")
    for k in range(4):
        err = np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= 1e-5, (k, err)


def test_split_cycle_entry_points_compose_to_tmg_cycle(dev):
    """tmg_cycle_down, then the coarsest level's own cycle from zero on its
    right-hand side (a plan of that level's problem), then tmg_cycle_up,
    applies the same cycle as tmg_cycle on a plan with the full hierarchy."""
    from paper_1409_5254_gb300 import tmg
    p, N, lam, s = 2, 1 << 14, 3.0, 4
    prob = inputs.scalar_problem(9, N, p, lam=lam, T=1.0, u0=0.2)
    F = torch.from_numpy(prob["F"]).to(dev)
    u_a = torch.from_numpy(np.random.default_rng(1).standard_normal((N, p + 1))).to(dev)
    u_b = u_a.clone()
    with tmg.Plan(p, prob["tau"], lam, N, s + 1, precision="fp64", n_min=1, tail_cap=1) as top, \
            tmg.Plan(p, prob["tau"] * 2 ** s, lam, N >> s, precision="fp64", n_min=16) as low, \
            tmg.Plan(p, prob["tau"], lam, N, precision="fp64", n_min=16) as full:
        fc = top.cycle_down(F, prob["u0"], u_a)
        uc = torch.zeros_like(fc)
        low.cycle(fc, 0.0, uc)
        top.cycle_up(uc, u_a)
        full.cycle(F, prob["u0"], u_b)
    a, b_ = u_a.cpu().numpy(), u_b.cpu().numpy()
    assert np.abs(a - b_).max() <= 1e-12 * np.abs(b_).max()


def test_split_cycle_rejects_plans_it_cannot_split(dev):
    from paper_1409_5254_gb300 import tmg
    N = 1 << 12
    F = torch.zeros((N, 2), dtype=torch.float64, device=dev)
    u = torch.zeros_like(F)
    for kw in ({"precision": "mixed"}, {"precision": "fp64", "gamma": 2}, {"precision": "fp64", "tail_cap": 2048}):
        with tmg.Plan(1, 1e-3, 1.0, N, 4, n_min=1, **kw) as plan:
            with pytest.raises(tmg.TmgError) as e:
                plan.cycle_down(F, 0.0, u)
            assert e.value.status == tmg.TMG_EUNSUPPORTED
