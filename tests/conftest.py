import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long CPU run of the oracle")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_sessionfinish(session, exitstatus):
    """Write the parity errors of the session (both definitions, per case) where
    $CGKS_PARITY_REPORT says."""
    path = os.environ.get("CGKS_PARITY_REPORT")
    if not path:
        return
    try:
        import json
        import parity_util
    except Exception:
        return
    with open(path, "a") as f:
        for r in parity_util.REPORT:
            f.write(json.dumps(r) + "\n")
