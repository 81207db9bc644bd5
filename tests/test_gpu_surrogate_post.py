"""GPU parity of the surrogate's post-processing, element by element (rows S3 and S4).

The network's output Y' is taken from the device (chem_surrogate_forward); the oracle then
applies its own element-conservation projection and its Newton iteration for T from the
enthalpy (the paper's Thermo Newton, §3.1) to that Y', cell by cell, and decides the route of
each cell: the network's result when the cell is inside the training box, the projection
conserves the elements after clipping and the Newton iteration converges inside [200, 6000] K;
the FP64 integrator otherwise.  chem_surrogate_advance must take the same decision for every
cell, return the oracle's composition and temperature on the network route, and return
chem_advance's result bitwise on the fallback route.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2312_13513_gb300 as cg  # noqa: E402
from oracle import surrogate as osur  # noqa: E402

from gpu_common import to_dev  # noqa: E402
from helpers import random_states  # noqa: E402

pytestmark = pytest.mark.gpu

DT = 5e-7
Y_ATOL = 1e-12        # network route: |Y''_gpu - Y''_oracle| (both from the same Y')
T_RTOL = 1e-11        # network route: |T_gpu - T_oracle| / T_oracle


def _params(mech, x, seed, out_scale, y_std):
    """A random 4 x 512 GELU network with statistics and a wide box around the features x."""
    rng = np.random.default_rng(seed)
    nin, ns = mech.ns + 2, mech.ns
    dims = [nin, 512, 512, 512, 512, ns]
    W = [rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]) for i in range(5)]
    W[4] *= out_scale
    b = [0.1 * rng.standard_normal(dims[i + 1]) for i in range(5)]
    sd = x.std(axis=0)
    sd = np.where(sd > 1e-6 * np.maximum(1.0, np.abs(x.mean(axis=0))), sd, 1.0)
    return {"W": W, "b": b, "dt": DT, "x_mean": x.mean(axis=0), "x_std": sd,
            "y_mean": np.zeros(ns), "y_std": np.full(ns, y_std),
            "box_lo": x.min(axis=0) - 1.0, "box_hi": x.max(axis=0) + 1.0}


def _oracle_post(mech, om, T0, Y0, ynet, box):
    """Route, Y'' and T of every cell from the oracle's projection and Newton on the device's Y';
    also flags the cells whose decision sits within rounding of a threshold (residual within a
    factor of 10 of 1e-9, or a Newton iterate within 1e-6 of the temperature bounds)."""
    n = T0.size
    A = osur.element_mass_matrix(mech)
    route = np.zeros(n, np.int8)
    Yo = np.array(Y0, copy=True)
    To = np.array(T0, copy=True)
    near = np.zeros(n, bool)
    why = {"box": 0, "nonfinite": 0, "conservation": 0, "newton": 0}
    for i in range(n):
        if box[i]:
            route[i] = 1; why["box"] += 1
            continue
        yp = ynet[:, i]
        if not np.all(np.isfinite(yp)):
            route[i] = 1; why["nonfinite"] += 1
            continue
        ypp, ok = osur.project(mech, Y0[:, i], yp)
        res = max(np.max(np.abs(A @ ypp - A @ Y0[:, i])), abs(ypp.sum() - Y0[:, i].sum()))
        if 1e-10 <= res <= 1e-8:
            near[i] = True
        if not ok:
            route[i] = 1; why["conservation"] += 1
            continue
        h0 = om.enthalpy_mass(T0[i], Y0[:, i])
        Tn, okn = osur.temperature_from_enthalpy(om, h0, ypp, T0[i])
        if abs(Tn - 200.0) <= 1e-6 * 200.0 or abs(Tn - 6000.0) <= 1e-6 * 6000.0:
            near[i] = True
        if not okn:
            route[i] = 1; why["newton"] += 1
            continue
        Yo[:, i] = ypp
        To[i] = Tn
    return route, To, Yo, near, why


def _compare(h2, om_h2, prm, T, p, Y):
    dm = cg.Mechanism(h2)
    model = cg.Surrogate(dm, prm)
    Td, pd, Yd = to_dev(T, p, Y)
    ynet, _, box = cg.surrogate_forward(model, Td, pd, Yd)
    route_d = torch.full((T.size,), -1, dtype=torch.int8, device="cuda")
    cg.surrogate_advance(model, Td, pd, Yd, DT, route=route_d)
    Tf, pf, Yf = to_dev(T, p, Y)
    cg.advance(dm, Tf, pf, Yf, DT)
    torch.cuda.synchronize()
    yn = ynet.cpu().numpy().astype(np.float64)
    bx = box.cpu().numpy().astype(bool)
    r_gpu = route_d.cpu().numpy()
    Tg, Yg = Td.cpu().numpy(), Yd.cpu().numpy()
    Tfb, Yfb = Tf.cpu().numpy(), Yf.cpu().numpy()
    r_or, To, Yo, near, why = _oracle_post(h2, om_h2, T, Y, yn, bx)
    # the route of every cell whose decision is not within rounding of a threshold
    sure = ~near
    assert np.array_equal(r_gpu[sure], r_or[sure]), np.nonzero((r_gpu != r_or) & sure)[0][:10]
    assert set(np.unique(r_gpu).tolist()) <= {0, 1}
    net = (r_gpu == 0) & (r_or == 0)
    fb = r_gpu == 1
    # network route: the oracle's projection and Newton on the device's network output
    dY = np.abs(Yg[:, net] - Yo[:, net])
    assert np.all(dY <= Y_ATOL), dY.max()
    dT = np.abs(Tg[net] - To[net]) / To[net]
    assert np.all(dT <= T_RTOL), dT.max()
    # fallback route: the FP64 integrator's result, bitwise
    assert np.array_equal(Tg[fb], Tfb[fb]) and np.array_equal(Yg[:, fb], Yfb[:, fb])
    return why, int(net.sum()), int(near.sum())


def test_projection_and_newton_elementwise_vs_oracle(h2, om_h2):
    """A non-trivial random network over 2000 H2 states: Y'' and T of the network route match the
    oracle's projection and Newton applied to the device's Y', element by element."""
    T, p, Y = random_states(h2, 2000, 51, "H2", Tlo=600.0, Thi=2400.0)
    prm = _params(h2, osur.features(T, p, Y), 61, out_scale=1.0, y_std=0.05)
    why, n_net, n_near = _compare(h2, om_h2, prm, T, p, Y)
    assert n_net >= 1900, (why, n_net)
    assert n_near <= 5


def test_conservation_and_newton_failures_fall_back(h2, om_h2):
    """A network whose Box-Cox increments are large (composition changes by large factors) and
    states outside the Newton range (150 K and 6500 K, inside a widened box): cells fail the
    conservation test after clipping and the Newton test; each such cell takes the FP64 route,
    as the oracle decides, and matches chem_advance bitwise."""
    T, p, Y = random_states(h2, 1500, 52, "H2", Tlo=800.0, Thi=2400.0)
    T[:6] = 150.0
    T[6:12] = 6500.0
    x = osur.features(T, p, Y)
    prm = _params(h2, x, 62, out_scale=3.0, y_std=3.0)
    prm["box_lo"][0] = 100.0
    prm["box_hi"][0] = 7000.0
    why, n_net, _ = _compare(h2, om_h2, prm, T, p, Y)
    assert why["conservation"] >= 20, why
    assert why["newton"] >= 6, why
    assert n_net >= 20, (why, n_net)
