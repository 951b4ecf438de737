import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: paper-sized workloads (minutes)")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Counts of the GPU-vs-oracle comparisons of this session: queries
    compared, compared down to their output, survivor sets handed back to
    the oracle after a legitimate divergence, LM separations, ICP decisions
    at their threshold."""
    helpers = sys.modules.get("tests.helpers")
    if helpers is not None and helpers.SESSION["queries"]:
        terminalreporter.write_line(f"oracle comparisons: {helpers.SESSION}")
