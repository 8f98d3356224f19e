import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


_PARITY = []


@pytest.fixture(scope="session")
def parity_log():
    """Collects parity reports (counts of compared and excluded points and cells); written
    as JSON to $FUSEFLOW_PARITY_LOG at the end of the session when that is set."""
    def log(name, report):
        _PARITY.append({"case": name, **report})
        print(name, report)
    return log


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("FUSEFLOW_PARITY_LOG")
    if path and _PARITY:
        import json
        with open(path, "w") as f:
            json.dump(_PARITY, f, indent=1)
