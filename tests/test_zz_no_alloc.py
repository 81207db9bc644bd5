"""The allocation-free integrator entry point (chem_advance_noalloc) gives the same results as
chem_advance_ex, on two calls in a row.

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
from synth.mechanism import h2_mechanism  # noqa: E402
from synth.states import load_table, quasi_dns_field  # noqa: E402

from gpu_common import within  # noqa: E402

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def test_noalloc_matches_regular_entry_point_twice():
    L = _lib.load()
    mech = h2_mechanism()
    dm = cg.Mechanism(mech)
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=5000 + 3, seed=4242)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    for call in range(2):
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
        rc = L.chem_advance_ex(dm.handle, _p(Ta), _p(p), _p(Ya), n, 5e-7, n, 1e-6, 1e-10, None,
                               _p(sa), _p(na), None, None, ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.chem_last_error()
        rc = L.chem_advance_noalloc(dm.handle, _p(Tb), _p(p), _p(Yb), n, 5e-7, n, 1e-6, 1e-10,
                                    _p(sb), _p(nb), None, ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.chem_last_error()
        torch.cuda.synchronize()
        assert np.all(sa.cpu().numpy() == 0) and np.all(sb.cpu().numpy() == 0), call
        Tan, Yan = Ta.cpu().numpy(), Ya.cpu().numpy()
        Tbn, Ybn = Tb.cpu().numpy(), Yb.cpu().numpy()
        assert np.all(within(Tan, Yan, Tbn, Ybn)), call
        assert np.array_equal(na.cpu().numpy(), nb.cpu().numpy()), call
        # every cell was advanced (the shared queue counter was reset for this call)
        assert np.all(nb.cpu().numpy() >= 1), call
