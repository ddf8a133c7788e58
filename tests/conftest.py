import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_terminal_summary(terminalreporter):
    """Worst error / tolerance ratio of each parity check that ran (1.0 is
    the tolerance itself)."""
    try:
        from helpers import MARGINS
    except ImportError:
        return
    if not MARGINS:
        return
    terminalreporter.write_sep("-", "parity margins (worst error / tolerance)")
    for (test, what), r in sorted(MARGINS.items(), key=lambda kv: -kv[1]):
        terminalreporter.write_line(f"{r:8.4f}  {what:14s} {test}")
