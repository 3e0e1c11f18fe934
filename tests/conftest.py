import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def inp():
    from paper_2407_09812_gb300 import inputs as I
    return I


def pytest_terminal_summary(terminalreporter):
    """Worst relative errors of the CUDA path against the oracle seen by the
    parity checks of this session."""
    try:
        from parity import WORST
    except ImportError:
        return
    if WORST:
        terminalreporter.write_line("worst relative errors vs oracle: " +
                                    ", ".join(f"{k} {v:.2e}" for k, v in sorted(WORST.items())))
