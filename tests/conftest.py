import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: long CPU test")


def read_golden(name):
    """Parse a tests/golden/*.txt fixture: '#' comments, 'key: values' lines,
    ';' separating matrix rows; returns {key: list-of-rows or list}."""
    out = {}
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if ":" in line:
                k, v = line.split(":", 1)
                if ";" in v:
                    out[k.strip()] = [[float(t) for t in r.split()] for r in v.split(";")]
                else:
                    out[k.strip()] = [float(t) for t in v.split()]
            else:
                rows.append(line.split())
    if rows:
        out["rows"] = rows
    return out


@pytest.fixture(scope="session")
def oracle():
    import oracle as o
    o.build()
    return o


@pytest.fixture(autouse=True)
def _bounds_word(request):
    """In the index-checking build (HS_DEBUG_BOUNDS=1), every GPU test must
    leave the library's bounds words at zero."""
    yield
    if request.node.get_closest_marker("gpu") is None or os.environ.get("HS_DEBUG_BOUNDS", "") in ("", "0"):
        return
    import torch
    from paper_2606_16959_gb300 import hs
    torch.cuda.synchronize()
    w = hs.hs_debug_bounds(reset=True)
    assert w is not None, "HS_DEBUG_BOUNDS=1 but the loaded library has no index checks"
    assert w[0] == 0, f"{w[0]} out-of-range indices; first at site {w[1]}: index {w[2]}, extent {w[3]}"
