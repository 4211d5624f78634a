import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "oracle: pins of the CPU oracle")
    config.addinivalue_line("markers", "abi: C-ABI library build and exports")


def load_golden(name):
    """Rows of a whitespace-separated golden file, '#' lines skipped, as strings."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def gpu():
    """The CUDA binding; GPU tests fail (not skip) when the library cannot load."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_04197_gb300 import gravity
    return gravity


def pytest_sessionfinish(session, exitstatus):
    """Write the parity figures the GPU tests recorded (tests/util.py) to $PARITY_LOG."""
    path = os.environ.get("PARITY_LOG")
    if not path:
        return
    try:
        from util import PARITY_RECORDS
    except ImportError:
        return
    if PARITY_RECORDS:
        import json
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(PARITY_RECORDS, f, indent=1, sort_keys=True)
