"""GPU parity of the integrator beyond 64 unknowns (row A6).  Groups of several warps factor and
solve systems of at most 64 unknowns with the panel LU and the register-held triangular sweeps;
larger systems take the shared-memory LU (two barriers per pivot step) and the shared-memory
sweeps.  The CH4 mechanism with 11 inert species appended has N = 65: its cells run that path,
in 128-thread groups (the default for this size) and in 64-thread groups, against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2312_13513_gb300 as cg  # noqa: E402
from synth.states import les_field, load_table  # noqa: E402

from gpu_common import assert_parity, to_dev  # noqa: E402
from helpers import with_inert_species  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wide(ch4):
    m = with_inert_species(ch4, 11)
    assert m.ns + 1 == 65
    return m, oracle.OracleMech(m), cg.Mechanism(m)


def _states(mech, base_ns, n, seed):
    f = les_field(load_table("ch4_flamelet.npz"), n=n, seed=seed)
    rng = np.random.default_rng(seed)
    Y = np.zeros((mech.ns, n))
    Y[:base_ns] = f["Y"]
    Y[base_ns:] = rng.uniform(0.0, 2e-3, (mech.ns - base_ns, n))
    Y /= Y.sum(axis=0, keepdims=True)
    return np.ascontiguousarray(f["T"]), np.ascontiguousarray(f["p"]), Y


@pytest.mark.parametrize("group", [0, 64])
def test_parity_beyond_64_unknowns(wide, ch4, group):
    mech, om, dm = wide
    T, p, Y = _states(mech, ch4.ns, 37, 4321)
    Td, pd, Yd = to_dev(T, p, Y)
    st = torch.full((T.size,), -1, dtype=torch.int8, device="cuda")
    ns = torch.zeros(T.size, dtype=torch.int32, device="cuda")
    opts = cg.options(group_threads=group) if group else None
    cg.advance(dm, Td, pd, Yd, 1e-6, 1e-6, 1e-10, status=st, nsub=ns, opts=opts)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    assert ns.cpu().numpy().min() >= 1
    out = assert_parity(om, T, p, Y, Td.cpu().numpy(), Yd.cpu().numpy(), 1e-6, 1e-6, 1e-10)
    assert out <= 2
