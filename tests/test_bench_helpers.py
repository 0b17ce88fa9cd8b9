"""The benchmark's host-side arithmetic (CPU): the algorithmic byte model that
the roofline divides by, the hierarchy of the oracle runs, and the check that
reports ncu traffic only for the kernel source it was captured on."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_level0_bytes_are_32_per_dof():
    """k_updown0 moves the residual pair (6 + 6 B), the solution (8 + 8 B) and the
    level-1 correction and right-hand side (2 + 2 B per fine DoF): 32 B/DoF."""
    N, d = 1 << 24, 2
    cb = bench.cycle_bytes(N, d, 7)
    assert cb["updown0"] == 32 * N * d
    assert cb["start0"] == 16 * N * d          # read F, write the pair and f_1
    assert cb["confirm0"] == 24 * N * d
    # the coarse levels add 5 level-vector passes per fused pair on top of level 0
    assert cb["updown0"] < cb["cycle"] < 1.4 * cb["updown0"]


def test_coarse_bytes_follow_the_level_grouping():
    """Two levels per kernel move 1.25 + 2.25 level-l vectors, a single level
    1.5 + 2.5; the on-chip or scanned coarsest level reads f and writes u."""
    N, d = 1 << 10, 1
    nl = lambda l: (N >> l) * d * 4                       # noqa: E731
    pair = lambda l: nl(l) + nl(l) // 4 + nl(l) + nl(l) // 4 + nl(l)   # noqa: E731
    single = lambda l: nl(l) + nl(l) // 2 + nl(l) + nl(l) // 2 + nl(l)   # noqa: E731
    up0 = bench.cycle_bytes(N, d, 1)["updown0"]
    assert bench.cycle_bytes(N, d, 4)["cycle"] == up0 + pair(1) + single(3) + 2 * (N >> 4) * d * 4
    assert bench.cycle_bytes(N, d, 5)["cycle"] == up0 + pair(1) + pair(3) + 2 * (N >> 5) * d * 4


def test_oracle_samples_keep_the_hierarchy_depth():
    """The oracle runs on a sample of n intervals coarsen as deep as the GPU
    hierarchy of the full N (the coarsest level scaled with the sample)."""
    assert bench.n_min_for(bench.N_FULL) == bench.N_MIN
    assert bench.n_min_for(1 << 21) == bench.N_MIN >> 3
    assert bench.n_min_for(1 << 16) == max(64, bench.N_MIN >> 8)
    assert bench.n_min_for(64) == 64
    assert bench.n_min_p(1) == bench.N_MIN and bench.n_min_p(2) == 64


def test_traffic_is_reported_only_for_its_kernel_source(tmp_path, monkeypatch):
    """measured_traffic() returns the captured bytes when the kernel source
    hashes to the recorded prefix, and None for any other source."""
    src = os.path.join(ROOT, "paper_1409_5254_gb300", "csrc", "tmg_kernels.cuh")
    with open(src, "rb") as fh:
        h = hashlib.sha256(fh.read()).hexdigest()[:16]
    monkeypatch.setitem(bench.UPDOWN0_TRAFFIC, "kernels_sha256", h)
    assert bench.measured_traffic() == pytest.approx(bench.UPDOWN0_TRAFFIC["bytes_per_launch"])
    monkeypatch.setitem(bench.UPDOWN0_TRAFFIC, "kernels_sha256", "0" * 16)
    assert bench.measured_traffic() is None
