import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA library binding; skips when no GPU is present."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10058_gb300 import genga
    genga.load()
    return genga


def pytest_terminal_summary(terminalreporter):
    """Logs the measured parity margins and the candidate pairs found within
    1e-12 relative of their critical radius by the detection parity tests
    (their decisions were compared bit-exactly with the oracle's like all
    others)."""
    _print_numerics(terminalreporter)
    try:
        from tests import borderline
    except ImportError:
        return
    if not borderline.LOG:
        return
    tr = terminalreporter
    tr.section(f"encounter pairs within {borderline.REL:g} relative of r_crit")
    for case, ncand, found in borderline.LOG:
        tr.write_line(f"{case}: {len(found)} of {ncand} candidates")
        for tag, i, j, q in found[:20]:
            tr.write_line(f"    ({i}, {j}) {tag} |r/rc - 1| = {q:.3e}")
        if len(found) > 20:
            tr.write_line(f"    ... {len(found) - 20} more")


def _print_numerics(terminalreporter):
    try:
        from tests import numerics_log
    except ImportError:
        return
    if not numerics_log.LOG:
        return
    tr = terminalreporter
    tr.section("measured parity (largest relative error / tolerance)")
    for case, quantity, value, tol in numerics_log.LOG:
        tr.write_line(f"{case}: {quantity} {value:.3e} (tolerance {tol:.0e})")
