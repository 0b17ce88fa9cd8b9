"""Multi-rank host logic (replicas.py) on CPU: two gloo ranks, no GPU.

The long horizon runs one replica per rank and batches shard by instances;
ranks exchange only timings.  These tests check the max-over-ranks reduction,
the whole-job throughput, and that every rank derives the same balanced,
disjoint and complete instance shards on its own.
"""
import os
import socket

import numpy as np
import pytest

from paper_1409_5254_gb300 import inputs, replicas

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, local, w = replicas.rank_info()
        assert (r, local, w) == (rank, rank, world)
        # each rank "timed" a different value; all must see the slowest
        ms = replicas.max_over_ranks(10.0 + 3.0 * rank)
        # the uneven batch recipe: every rank computes the shards independently
        Nv, pv, _ = inputs.uneven_batch(3, 500)
        weights = Nv * (pv + 1)
        mine = replicas.partition_instances(weights, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine.tolist())
        value = replicas.aggregate_throughput([int(weights[mine].sum())], ms)
        vals = [None] * world
        dist.all_gather_object(vals, value)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([ms, value, len(mine)], dtype=np.float64))
        if rank == 0:
            import json
            with open(os.path.join(out_dir, "shards.json"), "w") as fh:
                json.dump({"shards": gathered, "vals": vals}, fh)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_timing_and_shards(tmp_path):
    import json

    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 13.0                      # max over ranks
    with open(tmp_path / "shards.json") as fh:
        d = json.load(fh)
    s0, s1 = (np.array(x) for x in d["shards"])
    Nv, pv, _ = inputs.uneven_batch(3, 500)
    weights = Nv * (pv + 1)
    assert len(np.intersect1d(s0, s1)) == 0
    assert np.array_equal(np.sort(np.concatenate([s0, s1])), np.arange(len(Nv)))
    # whole-job throughput: the sum of both ranks' units over the slowest time
    per_rank_units = [weights[s0].sum(), weights[s1].sum()]
    assert sum(d["vals"]) == pytest.approx(sum(per_rank_units) / (13.0e-3))


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_is_complete_disjoint_and_balanced(world):
    rng = np.random.default_rng(world)
    w = rng.integers(1, 10_000, 1000).astype(float)
    shards = replicas.partition_instances(w, world)
    allidx = np.concatenate(shards)
    assert np.array_equal(np.sort(allidx), np.arange(len(w)))
    loads = np.array([w[s].sum() for s in shards])
    assert loads.max() <= w.sum() / world + w.max()    # the LPT bound
    for s in shards:
        assert np.all(np.diff(s) > 0)                    # instance order kept within a rank


def test_single_process_defaults():
    assert replicas.max_over_ranks(4.25) == 4.25
    assert replicas.aggregate_throughput([100, 300], 2.0) == pytest.approx(200_000.0)
    with pytest.raises(ValueError):
        replicas.partition_instances([1.0], 0)
