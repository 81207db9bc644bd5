import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


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
