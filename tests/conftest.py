import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer-running test")
    config.addinivalue_line("markers", "check_violations: makes the checked build's bounds "
                            "comparisons fail on purpose (test hook)")


@pytest.fixture(autouse=True)
def _bounds_record(request):
    """With PGEN_LIBRARY=checked (the bounds-checked library), every GPU test
    starts from zeroed check records and fails if any bounds comparison
    failed during it, unless it provokes failures on purpose."""
    if (os.environ.get("PGEN_LIBRARY") != "checked"
            or request.node.get_closest_marker("gpu") is None):
        yield
        return
    import torch
    import paper_1003_3684_gb300 as pg
    torch.cuda.synchronize()
    pg.pg_check_read(reset=True)
    yield
    torch.cuda.synchronize()
    rep = pg.pg_check_read(reset=True)
    if request.node.get_closest_marker("check_violations") is None:
        assert rep.count == 0, f"failed bounds comparisons in the checked build: {rep}"


def read_golden(name):
    """Parse a golden fixture: '#' lines are comments; returns list of token lists."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def golden():
    return read_golden
