import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# every output buffer and workspace the binding allocates starts as NaN
# (0xFF bytes), so an entry a kernel never writes fails the parity checks
# instead of passing on a recycled buffer that holds an earlier call's result
os.environ.setdefault("PSSGP_NAN_FILL", "1")

# largest error of each parity check seen in this session, printed at the end
_REPORT = {}


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def report():
    """report(name, err, bound): keep the largest err (and its bound) per check."""
    def rec(name, err, bound):
        err = float(err)
        old = _REPORT.get(name)
        if old is None or err > old[0]:
            _REPORT[name] = (err, float(bound))
    return rec


def pytest_terminal_summary(terminalreporter):
    if not _REPORT:
        return
    terminalreporter.section("parity: largest error per check (error / bound)")
    for name in sorted(_REPORT):
        err, bound = _REPORT[name]
        terminalreporter.write_line(f"{name:60s} {err:10.3e} / {bound:8.1e}")
