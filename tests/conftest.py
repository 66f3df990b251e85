import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libbmdca.so")


def pytest_terminal_summary(terminalreporter):
    import fliplog
    if fliplog.CHECKED[0]:
        terminalreporter.section("Boundary flips of the teacher-forced sweep checks")
        for line in fliplog.summary_lines():
            terminalreporter.write_line(line)


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def bm():
    """The CUDA binding; builds the library when it is missing or stale."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_18456_gb300 import _build, bmdca
    _build.build()
    bmdca.lib()
    return bmdca
