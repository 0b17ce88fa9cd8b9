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


def test_fp64_cycle_model_counts_level_vectors_and_operations():
    """The FP64 form's model: 28 + 28 B/DoF at level 0, four level vectors per
    coarse level, the coarsest level read and written (three passes when
    scanned); operations from fp64_ops_per_interval on every level."""
    N, d, nu = 1 << 12, 2, (1, 1)
    down, up, down0, up0 = bench.fp64_ops_per_interval(d, *nu)
    assert (down, up) == (2 * d * d + 5 * d, 2 * d * d + d + 4 * d)
    assert (down0, up0) == (down + 6 * d, up + d)
    b, ops = bench.fp64_cycle_model(N, d, nu, 3, False)
    nb = N * d * 8
    assert b["cycle"] == 56 * N * d + 4 * (nb >> 1) + 4 * (nb >> 2) + 2 * (nb >> 3)
    assert ops["cycle"] == down0 * N + up0 * N + (down + up) * (N // 2 + N // 4) + (d * d + 3 * d + 3) * (N >> 3)


def test_kernel_roofline_takes_the_larger_bound():
    """A kernel is bounded by the larger of its HBM time and its FP64 time."""
    hbm = bench.kernel_roofline("k", 1.0, 6.8e9, 0, 6800.0, "measured")
    assert hbm["bound"] == "hbm" and hbm["frac"] == pytest.approx(1.0)
    alu = bench.kernel_roofline("k", 2.0, 1e6, bench.FP64_PEAK_OPS * 1e-3, 6800.0, "measured")
    assert alu["bound"] == "alu" and alu["frac"] == pytest.approx(0.5)


def test_batched_model_uses_real_lengths_and_cycle_counts():
    """Mixed batched bytes: 16 + 16 B/DoF (start, confirmation) plus each
    instance's own cycles of its own hierarchy."""
    Nv, pv, cyc = [4096, 100], [1, 0], [3, 5]
    nbytes, ops = bench.batched_solve_model(Nv, pv, cyc, "mixed")
    exp = 32 * 4096 * 2 + 3 * bench.cycle_bytes(4096, 2, bench.oracle_levels(4096) - 1)["cycle"]
    exp += 32 * 100 + 5 * bench.cycle_bytes(100, 1, bench.oracle_levels(100) - 1)["cycle"]
    assert nbytes == exp and ops == 0
    assert bench.oracle_levels(4096) == 7 and bench.oracle_levels(100) == 2 and bench.oracle_levels(33) == 1
