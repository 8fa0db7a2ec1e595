import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU physics check")


def pytest_collection_modifyitems(config, items):
    # GPU tests need a device; make the skip explicit instead of failing on CPU hosts.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device on this host")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_sessionfinish(session, exitstatus):
    """Write the worst parity errors the tests observed (helpers.observe) to
    the JSON file named by LB_PARITY_LOG, if set."""
    path = os.environ.get("LB_PARITY_LOG")
    if not path:
        return
    try:
        import helpers
    except Exception:  # pragma: no cover
        return
    import json
    rows = [{"test": t, "quantity": k, "max_error": v} for (t, k), v in sorted(helpers.OBSERVED.items())]
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    with open(path, "w") as fh:
        json.dump(rows, fh, indent=0)
