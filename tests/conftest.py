import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libthor")
    config.addinivalue_line("markers", "slow: long CPU test")


_GRIDS = {}


def oracle_grid(glevel, modified=True, max_iter=100000, tol=1e-5):
    """Session cache of oracle grids (their construction dominates test time)."""
    from oracle.grid import build_grid
    key = (glevel, modified, max_iter, tol)
    if key not in _GRIDS:
        _GRIDS[key] = build_grid(glevel, modified=modified, max_iter=max_iter, tol=tol)
    return _GRIDS[key]


def report_dir():
    """Folder for the measured reports some GPU tests write (JSON, text), from
    the THOR_REPORT_DIR environment variable; None (no report) when unset or
    not a folder."""
    import os
    d = os.environ.get("THOR_REPORT_DIR")
    return d if d and os.path.isdir(d) else None
