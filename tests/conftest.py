import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


def pytest_terminal_summary(terminalreporter):
    """Integrator parity: how many compared cells left the contract tolerance and were accepted by
    the tight-oracle re-check (an accept/reject decision flipped by rounding near err = 1)."""
    gc = sys.modules.get("gpu_common")
    rows = getattr(gc, "BIFURCATIONS", None)
    if not rows:
        return
    tr = terminalreporter
    tr.write_sep("-", "integrator parity: bifurcated cells (re-checked against the tight oracle)")
    for test, n, nb in rows:
        tr.write_line(f"{nb:6d} of {n:7d} cells  {test}")
    tot = sum(r[1] for r in rows)
    totb = sum(r[2] for r in rows)
    tr.write_line(f"{totb:6d} of {tot:7d} cells  in total")


@pytest.fixture(scope="session")
def h2():
    from synth.mechanism import h2_mechanism
    return h2_mechanism()


@pytest.fixture(scope="session")
def ch4():
    from synth.mechanism import ch4_mechanism
    return ch4_mechanism()


@pytest.fixture(scope="session")
def om_h2(h2):
    import oracle
    return oracle.OracleMech(h2)


@pytest.fixture(scope="session")
def om_ch4(ch4):
    import oracle
    return oracle.OracleMech(ch4)
