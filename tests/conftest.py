import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def lib():
    """The GPU library's Python binding; fails loudly when it is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    import paper_1008_0861_gb300 as P
    P.load()  # raises if libaniso.so is absent
    return P


def pytest_terminal_summary(terminalreporter):
    """List the FP32 cases whose tolerance was raised above 1e-4 by the
    problem's own FP32 noise floor (tests/gpu_util.py: fp32_tol)."""
    try:
        import gpu_util
    except Exception:
        return
    cases = getattr(gpu_util, "LOOSE_FP32_CASES", [])
    if cases:
        terminalreporter.section("FP32 cases with a tolerance above 1e-4 (noise floor)")
        for c in cases:
            terminalreporter.write_line(c)
