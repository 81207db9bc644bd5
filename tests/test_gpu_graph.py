"""A whole chemistry step captured into a CUDA graph and replayed: the entry points are pure
stream work (stream-ordered temporaries, device-side fallback count), so capture works and a
replay gives bitwise the result of the direct call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2312_13513_gb300 as cg  # noqa: E402
from synth.states import load_table, quasi_dns_field  # noqa: E402

from gpu_common import to_dev  # noqa: E402
from test_gpu_serve import _identity_model  # noqa: E402

pytestmark = pytest.mark.gpu


def _field(n, seed):
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=n, seed=seed)
    return f["T"], f["p"], f["Y"]


def _capture(fn):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn(s)                                  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn(s)
    return g


def test_integrator_step_replays_bitwise(h2):
    dm = cg.Mechanism(h2)
    T0, p0, Y0 = to_dev(*_field(20000, 71))
    T, p, Y = T0.clone(), p0.clone(), Y0.clone()
    g = _capture(lambda s: cg.advance(dm, T, p, Y, 5e-7, stream=s))
    Tr, Yr = T0.clone(), Y0.clone()
    cg.advance(dm, Tr, p0, Yr, 5e-7)
    for _ in range(2):                         # replays start from the same state each time
        T.copy_(T0); Y.copy_(Y0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(T, Tr) and torch.equal(Y, Yr)


def test_surrogate_step_with_fallback_replays_bitwise(h2):
    dm = cg.Mechanism(h2)
    Th, ph, Yh = _field(20000, 72)
    model = _identity_model(dm, h2, Th, ph, Yh)
    Th = Th.copy()
    Th[::7] = 2500.0                           # outside the training box: FP64 fallback cells
    T0, p0, Y0 = to_dev(Th, ph, Yh)
    T, p, Y = T0.clone(), p0.clone(), Y0.clone()
    route = torch.empty(T.numel(), dtype=torch.int8, device="cuda")
    g = _capture(lambda s: cg.surrogate_advance(model, T, p, Y, 5e-7, route=route, stream=s))
    Tr, Yr = T0.clone(), Y0.clone()
    rr = torch.empty_like(route)
    cg.surrogate_advance(model, Tr, p0, Yr, 5e-7, route=rr)
    T.copy_(T0); Y.copy_(Y0)
    g.replay()
    torch.cuda.synchronize()
    assert int(rr.sum()) == int(np.ceil(20000 / 7))
    assert torch.equal(route, rr)
    assert torch.equal(T, Tr) and torch.equal(Y, Yr)
