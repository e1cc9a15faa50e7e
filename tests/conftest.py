import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: larger CPU oracle runs")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Parity report: how many compared elements needed an FP32-ambiguity
    allowance or the widened scale, and how many meet the plain
    1e-5 * |oracle| + 1e-7 bound."""
    try:
        import _helpers
    except ImportError:
        return
    lines = _helpers.report_lines()
    if lines:
        terminalreporter.section("parity report")
        for ln in lines:
            terminalreporter.write_line(ln)
    path = os.environ.get("GSR_PARITY_REPORT")
    if path:
        _helpers.write_report(path)
