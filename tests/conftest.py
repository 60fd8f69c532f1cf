import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def band_report(request):
    """Lines describing the contact band of each verdict-parity batch (edges
    whose oracle minimum clearance lies within 1e-4 m of the margin, and how
    the GPU decided them); printed in the terminal summary."""
    rep = []
    request.config._mrpop_band_report = rep
    return rep


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    rep = getattr(config, "_mrpop_band_report", None)
    if rep:
        terminalreporter.section("contact band: edges with |oracle min clearance - margin| <= 1e-4 m")
        for line in rep:
            terminalreporter.write_line(line)
