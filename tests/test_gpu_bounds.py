"""The debug build with bounds checks (csrc/tmg_bounds.h, -DTMG_BOUNDS).

compute-sanitizer is closed on this machine, so the kernels check their own
indices instead: the level-vector loads and stores of the streaming kernels
(against their array extents where a kernel knows them, else q >= 0), the
shared-memory layouts of the on-chip solvers against the CTA's shared memory,
and every load and store of the space-time heat kernels against its
interval's arrays.  A violation is counted and the access skipped.

This test builds that library and runs parity tests against it in a child
process (TMG_BOUNDS=1): single problems (FP64 cycles over every hierarchy
kind, W-cycles), batches (both schedules, V and W, uneven lengths) and the
heat equation (every grid size class).  tests/conftest.py asserts after
every GPU test that no kernel met an out-of-range index; the parity
assertions themselves must also hold.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SELECTION = [
    "tests/test_gpu_parity.py::test_fp64_cycles_match_textbook_cycle",
    "tests/test_gpu_parity.py::test_w_cycles_over_streaming_levels_match_textbook_cycle",
    "tests/test_gpu_batched.py::test_batched_w_cycles_match_textbook_cycle",
    "tests/test_gpu_batched.py::test_schedules_match_oracle",
    "tests/test_gpu_heat.py::test_cycle_iterates",
    "tests/test_gpu_heat.py::test_mixed_cycle_within_fp32",
]


def test_parity_under_bounds_checks():
    subprocess.check_call([sys.executable, "-c",
                           "from paper_1409_5254_gb300 import build_ext; build_ext.build(bounds=True)"], cwd=ROOT)
    env = dict(os.environ, TMG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *SELECTION],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
