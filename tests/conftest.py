import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, built in-tree; GPU tests fail loudly if it is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu test selected but no CUDA device is visible")
    from paper_2503_11731_gb300 import gsr
    return gsr.lib()


def pytest_terminal_summary(terminalreporter):
    """Every parity check's errors and flagged fraction (tests/parity.py)."""
    try:
        import parity
    except ImportError:
        return
    if not parity.REPORTS:
        return
    tr = terminalreporter
    tr.section("parity against the FP64 oracle (flagged = excluded as FP32-flippable)")
    for r in parity.REPORTS:
        errs = ", ".join(f"{k} {r[k]:.2e}" for k in ("rgb", "normal", "alpha", "T", "depth", "intensity", "range",
                                                     "drop") if k in r)
        tr.write_line(f"{r['test']}: {r['kind']} n={r['n']} flagged {r['flagged']} "
                      f"({100 * r['flagged_frac']:.3f} %, cap {100 * r['cap']:.3f} %); max errors {errs}")
    path = os.environ.get("GSR_PARITY_LOG")
    if path:
        import json
        with open(path, "w") as f:
            json.dump(parity.REPORTS, f, indent=1)
