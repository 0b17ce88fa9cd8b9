"""The plan's hierarchy on the host (tmg_plan_shape, the code tmg_setup runs):
level counts against the oracle's coarsening rule, and the choice between the
single-CTA coarse solver and the grid-wide scan.  No GPU."""
import pytest

import oracle as O
from paper_1409_5254_gb300 import tmg

TAIL_NMAX = 8192       # largest level the single-CTA solver takes
TAIL_LEVELS = 16       # most levels it holds
TAIL_DEFAULT_V = 64    # its default first level for V-cycles


@pytest.mark.parametrize("N", [1, 2, 3, 37, 64, 65, 100, 1024, 3 * 1024, 20002, 1 << 16, (1 << 20) + 2, 1 << 24])
@pytest.mark.parametrize("n_min", [1, 2, 64, 15000, 1 << 17])
@pytest.mark.parametrize("levels", [0, 1, 3])
def test_level_count_follows_the_coarsening_rule(N, n_min, levels):
    """Coarsen while the level has an even number of intervals, more than
    n_min of them, and the level cap allows (the nested meshes of Section 3),
    exactly as the oracle's textbook cycle does."""
    s = tmg.plan_shape(1, 1e-3, 1.0, N, levels, n_min=n_min)
    assert s["levels"] == O.num_levels(N, n_min, levels)
    assert 0 <= s["tail_level"] < s["levels"]
    assert s["tail_intervals"] == N >> s["tail_level"]


def test_benchmark_hierarchy():
    """The long-horizon benchmark: 2^24 intervals coarsened to 2^17, which is
    too large for one CTA and goes to the scan."""
    s = tmg.plan_shape(1, 1e-6, 1.0, 1 << 24, n_min=1 << 17)
    assert s == {"levels": 8, "tail_level": 7, "tail_intervals": 1 << 17, "scan_coarsest": True}


@pytest.mark.parametrize("p", [0, 1, 3, 5])
@pytest.mark.parametrize("N", [1 << 12, 1 << 20, 3 << 14])
def test_v_cycle_default_puts_the_on_chip_solver_at_64_intervals(p, N):
    s = tmg.plan_shape(p, 1e-3, 1.0, N)
    assert not s["scan_coarsest"]
    assert s["tail_intervals"] <= TAIL_DEFAULT_V
    # the first level at or below 64 intervals (the levels above it stream)
    assert s["tail_level"] == 0 or (N >> (s["tail_level"] - 1)) > TAIL_DEFAULT_V


@pytest.mark.parametrize("cap", [64, 128, 512, 1024])
def test_tail_cap_selects_the_first_level_within_it(cap):
    N = 1 << 14
    s = tmg.plan_shape(1, 1e-3, 1.0, N, gamma=2, tail_cap=cap)
    assert s["tail_intervals"] <= cap < 2 * s["tail_intervals"]


def test_w_cycles_take_the_largest_on_chip_level_within_the_limits():
    """W-cycles default to the largest level the single-CTA solver takes: at
    most 8192 intervals, at most 16 levels, and the level stack within its
    200 KB of shared memory (all of 8192 intervals at p_t = 0 in FP32, 4096 at
    p_t = 1)."""
    s = tmg.plan_shape(0, 1e-3, 1.0, 4096, gamma=2)
    assert s["tail_level"] == 0 and not s["scan_coarsest"]
    assert tmg.plan_shape(0, 1e-3, 1.0, 1 << 16, gamma=2)["tail_intervals"] == TAIL_NMAX
    assert tmg.plan_shape(1, 1e-3, 1.0, 1 << 16, gamma=2)["tail_intervals"] == TAIL_NMAX // 2
    s = tmg.plan_shape(1, 1e-3, 1.0, 1 << 24, gamma=2, n_min=1)
    assert s["levels"] == 25
    assert s["tail_intervals"] <= TAIL_NMAX and s["levels"] - s["tail_level"] <= TAIL_LEVELS


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("N", [37, 1 << 11, 1 << 24])
@pytest.mark.parametrize("p", [10, 20])
def test_wide_degrees_always_solve_their_coarsest_level_by_the_scan(p, prec, gamma, N):
    s = tmg.plan_shape(p, 1e-3, 1.0, N, precision=prec, gamma=gamma)
    assert s["scan_coarsest"] and s["tail_level"] == s["levels"] - 1


def test_status_codes_match_setup():
    def status(*args, **kw):
        with pytest.raises(tmg.TmgError) as e:
            tmg.plan_shape(*args, **kw)
        return e.value.status
    assert status(21, 1e-3, 1.0, 64) == tmg.TMG_EINVAL
    assert status(1, 0.0, 1.0, 64) == tmg.TMG_EINVAL
    assert status(1, 1e-3, 1.0, 0) == tmg.TMG_EINVAL
    assert status(1, 1e-3, 1.0, 64, 0, 2.5) == tmg.TMG_EINVAL
    assert status(1, 1e-3, 1.0, 64, gamma=3) == tmg.TMG_EINVAL
    for p in (6, 9, 11, 19):
        assert status(p, 1e-3, 1.0, 64) == tmg.TMG_EUNSUPPORTED
