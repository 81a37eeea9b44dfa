import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path through the C-ABI)")
    config.addinivalue_line("markers", "slow: longer CPU-only oracle checks")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_tables():
    """Rows of the paper's Tables 1-4 as dicts (see tests/golden/paper_iteration_tables.txt)."""
    rows = []
    with open(os.path.join(GOLDEN, "paper_iteration_tables.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t, d, beta, p, n, pwl, pmim, mim, cg = line.split()
            conv = lambda s: None if s == "-" else int(s)  # noqa: E731
            rows.append(dict(table=t, d=int(d), beta=float(beta), p=int(p), n=int(n),
                             pwl=conv(pwl), pmim=conv(pmim), mim=conv(mim), cg=conv(cg)))
    return rows
