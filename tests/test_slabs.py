"""Time-slab partition of one long horizon (slabs.py) on CPU: gloo ranks, no GPU.

The per-rank arithmetic here is the oracle's textbook cycle cut at the slab
level (oracle.mg_cycle_down / mg_cycle_up, pinned below against the uncut
cycle), so these tests check the partition itself -- the margins, the
margin exchange, the all-gather of the coarse problem and the coarse cycle on
it -- against the single-rank textbook cycle: the iterates of every rank's own
slab equal the single-rank iterates to 1e-12 relative after each of several
cycles.  The GPU backend of the same driver is tested in test_gpu_slabs.py.
"""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1409_5254_gb300 import inputs, slabs

torch = pytest.importorskip("torch")


class OracleSlabBackend:
    """The four steps a slab rank needs, from the oracle (test only)."""

    def __init__(self, lay, p, z, nu1, nu2, n_min):
        self.lay, self.p, self.z, self.nu, self.n_min = lay, p, z, (nu1, nu2), n_min
        _, _, self.a, _ = O.blocks(p)

    def _fhat(self, F, e_before):
        Fh = F.numpy().copy()
        Fh[0] += self.a * e_before
        return Fh

    def down(self, F_ext, e_before, u_ext):
        self._e = e_before
        fc = O.mg_cycle_down(self.p, self.z, self._fhat(F_ext, e_before), u_ext.numpy(), self.lay.slab_levels,
                             n_min=1, max_levels=self.lay.slab_levels + 1, nu1=self.nu[0], nu2=self.nu[1])
        return torch.from_numpy(fc)

    def up(self, uc_ext, u_ext):
        u = O.mg_cycle_up(self.p, self.z, self._fhat(self._F, self._e), u_ext.numpy(), uc_ext.numpy(),
                          self.lay.slab_levels, n_min=1, max_levels=self.lay.slab_levels + 1, nu1=self.nu[0],
                          nu2=self.nu[1])
        u_ext.copy_(torch.from_numpy(u))

    def coarse_cycle(self, fc):
        zc = self.z * (1 << self.lay.slab_levels)
        uc = O.mg_one_cycle(self.p, zc, fc.numpy(), np.zeros(tuple(fc.shape)), n_min=self.n_min, nu1=self.nu[0],
                            nu2=self.nu[1])
        return torch.from_numpy(uc)


def make_rank(lay, prob, p, z, nu, n_min):
    be = OracleSlabBackend(lay, p, z, nu[0], nu[1], n_min)
    F_ext = torch.from_numpy(np.ascontiguousarray(prob["F"][lay.start:lay.b]))
    be._F = F_ext
    _, _, _, b = O.blocks(p)
    return slabs.SlabRank(lay, be, F_ext, prob["u0"], torch.from_numpy(b))


def reference_iterates(prob, p, z, nu, n_min, k):
    Fh = O.fold_u0(p, prob["F"], prob["u0"])
    u = np.zeros_like(prob["F"])
    out = []
    for _ in range(k):
        u = O.mg_one_cycle(p, z, Fh, u, n_min=n_min, nu1=nu[0], nu2=nu[1])
        out.append(u.copy())
    return out


def test_cut_cycle_composes_to_the_textbook_cycle():
    """The oracle's cut cycle (way down to level s, the level-s problem's own
    cycle from zero, way up) is the uncut cycle, bit for bit."""
    for p, N, s, nu in ((1, 4096, 3, (1, 1)), (2, 2048, 5, (2, 2)), (0, 8192, 1, (3, 1)), (3, 1024, 4, (0, 2))):
        prob = inputs.scalar_problem(3, N, p, lam=2.0, T=1.0, u0=0.3)
        z = 2.0 * prob["tau"]
        Fh = O.fold_u0(p, prob["F"], prob["u0"])
        u = np.random.default_rng(0).standard_normal((N, p + 1))
        ref = O.mg_one_cycle(p, z, Fh, u, n_min=16, nu1=nu[0], nu2=nu[1])
        fc = O.mg_cycle_down(p, z, Fh, u, s, n_min=16, nu1=nu[0], nu2=nu[1])
        uc = O.mg_one_cycle(p, z * 2 ** s, fc, np.zeros_like(fc), n_min=16, nu1=nu[0], nu2=nu[1])
        got = O.mg_cycle_up(p, z, Fh, u, uc, s, n_min=16, nu1=nu[0], nu2=nu[1])
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("R", [2, 4])
def test_layout(R):
    N = 1 << 16
    lays = [slabs.slab_layout(N, R, r, 2, 2) for r in range(R)]
    S = N // R
    for r, lay in enumerate(lays):
        assert (lay.a, lay.b) == (r * S, (r + 1) * S)
        assert lay.margin == (0 if r == 0 else slabs.margin_for(lay.slab_levels, 2, 2))
        assert lay.margin + 1 <= S and lay.start % (1 << lay.slab_levels) == 0
        assert (S >> lay.slab_levels) >= 256 and lay.slab_levels + 1 < slabs._levels(N, 64)
        assert lay.margin_of(r) == lay.margin


@pytest.mark.parametrize("R,p,nu", [(2, 1, (1, 1)), (4, 2, (2, 2)), (3, 0, (2, 1))])
def test_in_process_slabs_match_single_rank_iterates(R, p, nu):
    N = 3 * 4096 if R == 3 else 1 << 14
    n_min = 16
    prob = inputs.scalar_problem(5, N, p, lam=3.0, T=1.0, u0=0.7)
    z = 3.0 * prob["tau"]
    ranks = [make_rank(slabs.slab_layout(N, R, r, *nu, n_min=n_min, coarse_per_slab=64), prob, p, z, nu, n_min)
             for r in range(R)]
    ref = reference_iterates(prob, p, z, nu, n_min, 3)
    for k in range(3):
        slabs.run_in_process(ranks, 1, ranks[0].be.coarse_cycle)
        got = np.concatenate([rk.own().numpy() for rk in ranks])
        err = np.abs(got - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= 1e-12, (k, err)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str, p: int, nu, cycles: int):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N, n_min = 1 << 14, 16
        prob = inputs.scalar_problem(7, N, p, lam=1.5, T=1.0, u0=-0.4)
        z = 1.5 * prob["tau"]
        lay = slabs.slab_layout(N, world, rank, *nu, n_min=n_min, coarse_per_slab=64)
        rk = make_rank(lay, prob, p, z, nu, n_min)
        for k in range(cycles):
            slabs.run_distributed(rk, 1, dist)
            np.save(os.path.join(out_dir, f"rank{rank}_cycle{k}.npy"), rk.own().numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,p,nu", [(2, 1, (1, 1)), (2, 3, (2, 2))])
def test_gloo_ranks_reproduce_single_rank_iterates(tmp_path, world, p, nu):
    """World-size-2 gloo ranks: per cycle the margin goes left to right by
    point-to-point messages and the coarse right-hand sides by all_gather;
    every rank's own slab equals the single-rank iterate to 1e-12."""
    import torch.multiprocessing as mp
    cycles = 3
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path), p, nu, cycles), nprocs=world, join=True,
                       start_method="spawn")
    N, n_min = 1 << 14, 16
    prob = inputs.scalar_problem(7, N, p, lam=1.5, T=1.0, u0=-0.4)
    ref = reference_iterates(prob, p, 1.5 * prob["tau"], nu, n_min, cycles)
    for k in range(cycles):
        got = np.concatenate([np.load(os.path.join(tmp_path, f"rank{r}_cycle{k}.npy")) for r in range(world)])
        err = np.abs(got - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= 1e-12, (k, err)
