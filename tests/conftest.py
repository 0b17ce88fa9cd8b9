import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def load_golden(name):
    """Rows of a ';'-separated golden fixture (comments start with '#')."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([[float(x) for x in field.split()] for field in line.split(";")])
    return rows


@pytest.fixture(autouse=True)
def _bounds_clean(request):
    """Under the debug build with bounds checks (TMG_BOUNDS=1), every GPU test
    must leave no out-of-range index behind in any kernel it ran."""
    yield
    if os.environ.get("TMG_BOUNDS") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_1409_5254_gb300 import tmg
    res = tmg.debug_bounds()
    assert res is not None, "TMG_BOUNDS=1 but the loaded library has no bounds checks"
    count, first = res
    assert count == 0, f"{count} out-of-range indices; first: site {first >> 40}, index {first & ((1 << 40) - 1)}"
