"""The "chemistry + thermo" step (chem_step_*): its stages give bitwise the results of the
individual entry points, a captured CUDA graph replays bitwise, and the Thermo stage recovers
the chemistry's temperature from the conserved enthalpy (§3.1, Fig. 1; graphs: §3.2)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2312_13513_gb300 as cg  # noqa: E402
from synth.states import load_table, quasi_dns_field  # noqa: E402
from synth.transport import generate_transport  # noqa: E402

from gpu_common import to_dev  # noqa: E402

pytestmark = pytest.mark.gpu

DT = 5e-7
MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2312_13513_gb300",
                     "models", "h2_quasi_dns.chemsur")


def _buffers(n, ns):
    f64 = lambda *s: torch.empty(*s, dtype=torch.float64, device="cuda")
    return {"h0": f64(n), "cp0": f64(n), "q": f64(n), "mu": f64(n), "lam": f64(n), "D": f64(ns, n),
            "thermo_status": torch.empty(n, dtype=torch.int8, device="cuda")}


def _step(dm, tr, T, p, Y, b, model=None, route=None, status=None, nsub=None):
    return cg.Step(dm, T, p, Y, DT, model=model, transport=tr, h0=b["h0"], cp0=b["cp0"], q=b["q"], route=route,
                   status=status, nsub=nsub, thermo_status=b["thermo_status"], mu=b["mu"], lam=b["lam"],
                   D=b["D"])


@pytest.mark.parametrize("route", ["fp64", "surrogate"])
def test_step_stages_match_entry_points_and_graph_replays_bitwise(h2, route):
    if route == "surrogate" and not os.path.exists(MODEL):
        pytest.skip("no trained model in the package")
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=20000 + 7, seed=81)
    dm = cg.Mechanism(h2)
    tr = cg.Transport(dm, generate_transport(h2))
    model = cg.Surrogate(dm, path=MODEL) if route == "surrogate" else None
    T0, p, Y0 = to_dev(f["T"], f["p"], f["Y"])
    n = T0.numel()
    # the stages one by one
    h0 = torch.empty(n, dtype=torch.float64, device="cuda"); cp0 = torch.empty_like(h0)
    cg.mixture_thermo(dm, T0, Y0, h0, cp0)
    T1, Y1 = T0.clone(), Y0.clone()
    if model is not None:
        cg.surrogate_advance(model, T1, p, Y1, DT)
    else:
        cg.advance(dm, T1, p, Y1, DT)
    q = cg.heat_release(dm, T0, p, Y0, Y1, DT)
    Tc = T1.clone()
    ts = torch.empty(n, dtype=torch.int8, device="cuda")
    cg.temperature_from_enthalpy(dm, h0, Y1, T1, status=ts)
    mu = torch.empty_like(h0); lam = torch.empty_like(h0); D = torch.empty_like(Y0)
    tr(T1, p, Y1, mu, lam, D)
    torch.cuda.synchronize()
    # the Thermo stage recovers the chemistry's temperature from the conserved enthalpy: to the
    # Newton tolerance after the surrogate's own enthalpy-conserving post-processing, to the
    # integrator's tolerance (rtol 1e-6 on T) after the FP64 step, which conserves h only as well
    # as it integrates the energy equation
    assert int(ts.abs().sum()) == 0
    tol = 1e-8 if model is not None else 5e-6
    assert float(((T1 - Tc).abs() / Tc).max()) <= tol
    # the step, direct, then twice as a graph from the same start state
    T, Y = T0.clone(), Y0.clone()
    b = _buffers(n, h2.ns)
    st = _step(dm, tr, T, p, Y, b, model=model)
    for use_graph in (False, True, True):
        T.copy_(T0); Y.copy_(Y0)
        st.run(graph=use_graph)
        torch.cuda.synchronize()
        assert torch.equal(T, T1) and torch.equal(Y, Y1), use_graph
        assert torch.equal(b["h0"], h0) and torch.equal(b["cp0"], cp0) and torch.equal(b["q"], q)
        assert torch.equal(b["mu"], mu) and torch.equal(b["lam"], lam) and torch.equal(b["D"], D)
        assert torch.equal(b["thermo_status"], ts)
    st.run(graph=False)
    ms = st.stage_ms()
    assert len(ms) == 4 and all(m > 0.0 for m in ms)
    st.close()


def test_step_rejects_bad_descriptions(h2):
    dm = cg.Mechanism(h2)
    T, p, Y = to_dev(*[np.asarray(a) for a in (np.full(4, 1500.0), np.full(4, 1.01325e6), np.full((h2.ns, 4), 1.0 / h2.ns))])
    with pytest.raises(cg.ChemError):
        cg.Step(dm, T, p, Y, DT)                         # no h0
    h0 = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(cg.ChemError):
        cg.Step(dm, T, p, Y, -1.0, h0=h0)
    tr = cg.Transport(dm, generate_transport(h2))
    with pytest.raises(cg.ChemError):
        cg.Step(dm, T, p, Y, DT, h0=h0, transport=tr)    # transport without an output
