"""Shared pytest set-up: markers and the repository root on sys.path."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long CPU statistics test")


def pytest_terminal_summary(terminalreporter):
    """Report the largest element-wise differences the GPU parity comparisons saw."""
    try:
        from gpu_helpers import EW_SEEN
    except Exception:
        return
    if not EW_SEEN:
        return
    for prec in (64, 32):
        seen = [e for e in EW_SEEN if e[0] == prec]
        if seen:
            wv = max(seen, key=lambda e: e[1])
            ws = max(seen, key=lambda e: e[2])
            terminalreporter.write_line(
                f"element-wise FP{prec}: {len(seen)} comparisons; worst voxel {wv[1]:.3e} ({wv[3]}), "
                f"worst shell {ws[2]:.3e} ({ws[3]})")
