import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libmg")


def pytest_terminal_summary(terminalreporter):
    """Print the measured parity errors (in units of u = 2^-53) of the cycle-level GPU checks."""
    try:
        from tests.gpu_common import OBSERVED
    except Exception:
        return
    if not OBSERVED:
        return
    tr = terminalreporter
    tr.section("FP64 cycle parity: err / u against the bound u (C1 + C2 F)")
    worst = {}
    for name, err_u, amp, bound_u in OBSERVED:
        if name not in worst or err_u / bound_u > worst[name][0] / worst[name][2]:
            worst[name] = (err_u, amp, bound_u)
    tr.write_line(f"{'check':52s} {'err/u':>12s} {'F':>10s} {'bound/u':>12s} {'margin':>8s}")
    for name, (err_u, amp, bound_u) in sorted(worst.items()):
        tr.write_line(f"{name:52s} {err_u:12.1f} {amp:10.3g} {bound_u:12.1f} {bound_u / max(err_u, 1e-300):8.1f}")
