"""GPU parity of the BF16 surrogate path (tcgen05 GEMM, fused forward, projection, fallback)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2312_13513_gb300 as cg  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from oracle import surrogate as osur  # noqa: E402

from gpu_common import to_dev  # noqa: E402
from helpers import random_states  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(300, 200, 192), (128, 128, 64), (1024, 512, 512), (4096, 128, 512)])
def test_gemm_bf16_matches_torch(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    C = cg.gemm_bf16(A, B, bias)
    ref = A.double() @ B.double().T + bias.double()
    err = (C.double() - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item(), err


def _random_params(ns, seed, dt=5e-7):
    rng = np.random.default_rng(seed)
    nin = ns + 2
    dims = [nin, 512, 512, 512, 512, ns]
    W = [rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]) for i in range(5)]
    b = [0.1 * rng.standard_normal(dims[i + 1]) for i in range(5)]
    return {"W": W, "b": b, "dt": dt}


def _std(x):
    """Feature scale; a constant feature (ln p at fixed pressure) gets scale 1, because its
    standard deviation is rounding noise."""
    sd = x.std(axis=0)
    return np.where(sd > 1e-6 * np.maximum(1.0, np.abs(x.mean(axis=0))), sd, 1.0)


def _oracle_z(params, T, p, Y):
    x = osur.features(T, p, Y)
    xz = (x - params["x_mean"]) / params["x_std"]
    Wr = [omlp.bf16_round(w) for w in params["W"]]
    br = [np.asarray(bb, np.float32).astype(np.float64) for bb in params["b"]]
    out, _ = omlp.forward(Wr, br, xz, emulate_bf16=True)
    return out.T      # [ns, n]


def test_forward_matches_oracle_mlp(h2):
    dm = cg.Mechanism(h2)
    T, p, Y = random_states(h2, 1000, 9, "H2", Tlo=300.0, Thi=2500.0)
    x = osur.features(T, p, Y)
    prm = _random_params(h2.ns, 3)
    prm["x_mean"] = x.mean(axis=0)
    prm["x_std"] = _std(x)
    prm["y_mean"] = 0.01 * np.arange(h2.ns)
    prm["y_std"] = 0.05 + 0.01 * np.arange(h2.ns)
    prm["box_lo"] = x.min(axis=0) - 1.0
    prm["box_hi"] = x.max(axis=0) + 1.0
    prm["box_hi"][0] = 2000.0           # cells hotter than 2000 K leave the box
    model = cg.Surrogate(dm, prm)
    Td, pd, Yd = to_dev(T, p, Y)
    ynet, z, box = cg.surrogate_forward(model, Td, pd, Yd, with_z=True)
    torch.cuda.synchronize()
    z = z.cpu().numpy().astype(np.float64)
    zr = _oracle_z(prm, T, p, Y)
    dz = np.abs(z - zr)
    tol = 1e-2 * np.maximum(1.0, np.abs(zr))
    assert np.all(dz <= tol), (dz.max(), np.unravel_index(np.argmax(dz - tol), dz.shape))
    assert np.array_equal(box.cpu().numpy().astype(bool), T > 2000.0)
    # inverse transform: Y' = BC^-1(BC(Y0) + z sd + mu)
    yr = osur.boxcox_inv(osur.boxcox(Y) + zr * prm["y_std"][:, None] + prm["y_mean"][:, None])
    yg = ynet.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(yg - yr) <= 0.05 * np.abs(yr) + 1e-6)


def _identity_params(mech, x):
    prm = _random_params(mech.ns, 1)
    prm["W"][4] = np.zeros_like(prm["W"][4])
    prm["b"][4] = np.zeros(mech.ns)
    prm["x_mean"] = x.mean(axis=0)
    prm["x_std"] = _std(x)
    prm["y_mean"] = np.zeros(mech.ns)
    prm["y_std"] = np.ones(mech.ns)
    prm["box_lo"] = x.min(axis=0) - 1.0
    prm["box_hi"] = x.max(axis=0) + 1.0
    return prm


def test_identity_network_through_projection_and_newton(h2, om_h2):
    """A network that predicts no change: every cell takes the network route, conserves
    elements to 1e-9, keeps its enthalpy and stays at its temperature."""
    dm = cg.Mechanism(h2)
    T, p, Y = random_states(h2, 777, 12, "H2", Tlo=400.0, Thi=2400.0)
    prm = _identity_params(h2, osur.features(T, p, Y))
    model = cg.Surrogate(dm, prm)
    Td, pd, Yd = to_dev(T, p, Y)
    route = torch.full((T.size,), -1, dtype=torch.int8, device="cuda")
    cg.surrogate_advance(model, Td, pd, Yd, prm["dt"], route=route)
    torch.cuda.synchronize()
    route = route.cpu().numpy(); Tg = Td.cpu().numpy(); Yg = Yd.cpu().numpy()
    assert np.all(route == 0)
    A = osur.element_mass_matrix(h2)
    assert np.max(np.abs(A @ Yg - A @ Y)) <= 1e-9
    assert np.max(np.abs(Tg - T) / T) <= 1e-5
    for i in range(0, T.size, 97):
        h0 = om_h2.enthalpy_mass(T[i], Y[:, i])
        h1 = om_h2.enthalpy_mass(Tg[i], Yg[:, i])
        assert abs(h1 - h0) <= 1e-9 * om_h2.cp_mass(T[i], Y[:, i]) * T[i]


def test_out_of_box_cells_fall_back_to_the_fp64_integrator(h2):
    """Cells outside the training box take the FP64 route and match chem_advance bitwise."""
    dm = cg.Mechanism(h2)
    T, p, Y = random_states(h2, 1500, 13, "H2", Tlo=900.0, Thi=2200.0)
    prm = _identity_params(h2, osur.features(T, p, Y))
    prm["box_hi"][0] = 1500.0
    model = cg.Surrogate(dm, prm)
    Ts, ps, Ys = to_dev(T, p, Y)
    route = torch.full((T.size,), -1, dtype=torch.int8, device="cuda")
    cg.surrogate_advance(model, Ts, ps, Ys, prm["dt"], route=route)
    Ti, pi, Yi = to_dev(T, p, Y)
    cg.advance(dm, Ti, pi, Yi, prm["dt"])
    torch.cuda.synchronize()
    route = route.cpu().numpy()
    hot = T > 1500.0
    assert np.array_equal(route == 1, hot)
    assert np.array_equal(Ts.cpu().numpy()[hot], Ti.cpu().numpy()[hot])
    assert np.array_equal(Ys.cpu().numpy()[:, hot], Yi.cpu().numpy()[:, hot])


def test_surrogate_rejects_wrong_dt(h2):
    dm = cg.Mechanism(h2)
    T, p, Y = random_states(h2, 10, 14, "H2")
    prm = _identity_params(h2, osur.features(T, p, Y))
    model = cg.Surrogate(dm, prm)
    with pytest.raises(cg.ChemError):
        cg.surrogate_advance(model, *to_dev(T, p, Y), 1e-6)


# ---------------------------------------------------------------------------------------------
# training kernels
# ---------------------------------------------------------------------------------------------
def _small_problem(seed, B=256, nin=11, nout=9):
    rng = np.random.default_rng(seed)
    dims = [nin, 512, 512, 512, 512, nout]
    W = [omlp.bf16_round(rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i])) for i in range(5)]
    b = [np.float32(0.1 * rng.standard_normal(dims[i + 1])).astype(np.float64) for i in range(5)]
    X = omlp.bf16_round(rng.standard_normal((B, nin)))
    T = rng.standard_normal((B, nout))
    return W, b, X, T


def test_trainer_forward_backward_match_oracle():
    from paper_2312_13513_gb300.train import PAD, Trainer
    W, b, X, T = _small_problem(1)
    B, nin = X.shape
    nout = T.shape[1]
    tr = Trainer(nin, nout, B, W=W, b=b)
    Xd = torch.zeros((B, PAD), dtype=torch.bfloat16, device="cuda")
    Xd[:, :nin] = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16)
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    out = torch.empty((B, nout), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    tr.forward(Xd, out)
    tr.backward(Td, loss)
    dW, db = tr.get(1)
    o_out, cache = omlp.forward(W, b, X, emulate_bf16=True)
    assert np.max(np.abs(out.cpu().numpy() - o_out)) <= 1e-2 * max(1.0, np.max(np.abs(o_out)))
    assert abs(loss.item() - omlp.mse_loss(o_out, T)) <= 1e-3 * omlp.mse_loss(o_out, T)
    gW, gb = omlp.backward(W, b, cache, o_out, T)
    for l in range(5):
        rel = np.linalg.norm(dW[l] - gW[l]) / np.linalg.norm(gW[l])
        relb = np.linalg.norm(db[l] - gb[l]) / np.linalg.norm(gb[l])
        assert rel < 2e-2 and relb < 2e-2, (l, rel, relb)


def test_adam_step_matches_oracle():
    from paper_2312_13513_gb300.train import PAD, Trainer
    W, b, X, T = _small_problem(2)
    B, nin = X.shape
    tr = Trainer(nin, T.shape[1], B, W=W, b=b)
    Xd = torch.zeros((B, PAD), dtype=torch.bfloat16, device="cuda")
    Xd[:, :nin] = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16)
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    tr.forward(Xd)
    tr.backward(Td)
    dW, db = tr.get(1)
    tr.adam(1e-3)
    W1, b1 = tr.get(0)
    params = [np.asarray(w, np.float64) for w in W] + [np.asarray(x, np.float64) for x in b]
    grads = [np.asarray(g, np.float64) for g in dW] + [np.asarray(g, np.float64) for g in db]
    m = [np.zeros_like(x) for x in params]
    v = [np.zeros_like(x) for x in params]
    ref, _, _ = omlp.adam_step(params, grads, m, v, 1, lr=1e-3)
    got = [np.asarray(w, np.float64) for w in W1] + [np.asarray(x, np.float64) for x in b1]
    for r, g in zip(ref, got):
        assert np.max(np.abs(r - g)) <= 2e-6


def test_training_reduces_loss():
    """Fit the outputs of a fixed random teacher network: loss must fall by 10x."""
    from paper_2312_13513_gb300.train import PAD, Trainer
    Wt, bt, _, _ = _small_problem(3, nout=9)
    rng = np.random.default_rng(4)
    n, B = 8192, 512
    X = omlp.bf16_round(rng.standard_normal((n, 11)))
    Y, _ = omlp.forward(Wt, bt, X, emulate_bf16=False)
    Xd = torch.zeros((n, PAD), dtype=torch.bfloat16, device="cuda")
    Xd[:, :11] = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16)
    Yd = torch.tensor(Y, dtype=torch.float32, device="cuda")
    tr = Trainer(11, 9, B, seed=5)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    first = None
    for step in range(300):
        i = (step * B) % n
        tr.forward(Xd[i:i + B])
        tr.backward(Yd[i:i + B], loss)
        if first is None:
            first = loss.item()
        tr.adam(1e-3)
    assert loss.item() < 0.1 * first, (first, loss.item())
