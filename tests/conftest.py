import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def load_fig2_table():
    """Rows of the Fig. 2 golden table as {name: list[int]}."""
    rows = {}
    with open(os.path.join(ROOT, "tests", "golden", "fig2_halfedges.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, *vals = line.split()
            rows[name] = [int(v) for v in vals]
    return rows


@pytest.fixture(scope="session")
def fig2_table():
    return load_fig2_table()
