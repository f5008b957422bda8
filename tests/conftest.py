import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def mechs():
    from paper_2510_10005_gb300 import inputs
    return {k: inputs.gen_mechanism(k) for k in ("h2", "ch4")}


@pytest.fixture(scope="session")
def ref(mechs):
    import oracle
    return {k: oracle.RefMech(m) for k, m in mechs.items()}


def pytest_sessionfinish(session, exitstatus):
    """With CHEMGB_PARITY_REPORT set, write the largest errors the parity
    checks measured (tests/parity.py) to that file as JSON."""
    path = os.environ.get("CHEMGB_PARITY_REPORT")
    if not path:
        return
    import json
    import parity
    if parity.REPORT:
        with open(path, "w") as f:
            json.dump(parity.REPORT, f, indent=1, sort_keys=True)
