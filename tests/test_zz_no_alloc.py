"""The allocation-free integrator entry point (chem_advance_noalloc) gives bitwise the same
results and step counts as chem_advance_ex, on two calls in a row, for both group shapes.

This file is collected last so that a run stopping at the first failure has already run every
other test.  It also passes when run alone in a fresh process: the first call performs the
per-device look-up of the library's static scratch array.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_13513_gb300 import _lib  # noqa: E402
import paper_2312_13513_gb300 as cg  # noqa: E402
from synth.mechanism import ch4_mechanism, h2_mechanism  # noqa: E402
from synth.states import les_field, load_table, quasi_dns_field  # noqa: E402

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _run_both(L, dm, f, dt, call):
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    T0 = torch.tensor(f["T"], device=dev)
    p = torch.tensor(f["p"], device=dev)
    Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device=dev)
    n = T0.numel()
    Ta, Ya = T0.clone(), Y0.clone()
    Tb, Yb = T0.clone(), Y0.clone()
    sa = torch.full((n,), -1, dtype=torch.int8, device=dev)
    sb = torch.full((n,), -1, dtype=torch.int8, device=dev)
    na = torch.zeros(n, dtype=torch.int32, device=dev)
    nb = torch.zeros(n, dtype=torch.int32, device=dev)
    ra = torch.full((n,), -1, dtype=torch.int32, device=dev)
    rb = torch.full((n,), -1, dtype=torch.int32, device=dev)
    rc = L.chem_advance_ex(dm.handle, _p(Ta), _p(p), _p(Ya), n, dt, n, 1e-6, 1e-10, None,
                           _p(sa), _p(na), _p(ra), None, ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, L.chem_last_error()
    rc = L.chem_advance_noalloc(dm.handle, _p(Tb), _p(p), _p(Yb), n, dt, n, 1e-6, 1e-10,
                                _p(sb), _p(nb), _p(rb), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, L.chem_last_error()
    torch.cuda.synchronize()
    assert np.all(sa.cpu().numpy() == 0) and np.all(sb.cpu().numpy() == 0), call
    # the same kernel in the same launch shape: bitwise the same results and step counts
    assert torch.equal(Ta, Tb) and torch.equal(Ya, Yb), call
    assert torch.equal(na, nb) and torch.equal(ra, rb), call
    # every cell was advanced once (the shared queue counter was reset for this call)
    assert np.all(nb.cpu().numpy() >= 1), call


def test_noalloc_matches_regular_entry_point_twice():
    """H2 mechanism: sub-warp groups, two cells per queue entry."""
    L = _lib.load()
    dm = cg.Mechanism(h2_mechanism())
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=5000 + 3, seed=4242)
    for call in range(2):
        _run_both(L, dm, f, 5e-7, call)


def test_noalloc_ch4_one_cta_per_cell_twice():
    """CH4 mechanism: one 128-thread group per cell, one cell per queue entry."""
    L = _lib.load()
    dm = cg.Mechanism(ch4_mechanism())
    f = les_field(load_table("ch4_flamelet.npz"), n=37, seed=4243)
    for call in range(2):
        _run_both(L, dm, f, 1e-6, call)
