import os
import sys

import pytest

ROOT = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(ROOT)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# support-parity counts reported by the GPU parity tests (printed at the end of the session)
_PARITY_LOG = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture
def parity_log(request):
    """Record one line of counts for the end-of-session summary: support differences against the
    oracle split into in-band, L-explained and unexplained, and any other figure a test reports."""
    def log(**kw):
        _PARITY_LOG.append((request.node.nodeid.split("/")[-1], kw))
    return log


def pytest_terminal_summary(terminalreporter):
    if not _PARITY_LOG:
        return
    terminalreporter.write_sep("-", "parity against the oracle: support differences "
                                    "(inband / L_explained / unexplained) and errors")
    for name, kw in _PARITY_LOG:
        terminalreporter.write_line(name + ": " + " ".join(f"{k}={v}" for k, v in kw.items()))
