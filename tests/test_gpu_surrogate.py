"""GPU parity of the BF16 surrogate path (tcgen05 GEMM, fused forward, projection, fallback)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2312_13513_gb300 as cg  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from oracle import surrogate as osur  # noqa: E402

from synth.states import load_table, quasi_dns_field  # noqa: E402

from gpu_common import to_dev  # noqa: E402
from helpers import random_states  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(300, 200, 192), (128, 128, 64), (1024, 512, 512), (4096, 128, 512),
                                   (16384, 800, 1600), (1000, 400, 800), (2048, 1600, 64), (640, 256, 136)])
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
    # the device receives FP32 weights: the oracle rounds (layers 2-5) or splits (layer 1) those
    W32 = [np.asarray(w, np.float32).astype(np.float64) for w in params["W"]]
    br = [np.asarray(bb, np.float32).astype(np.float64) for bb in params["b"]]
    out, _ = omlp.forward(W32, br, xz, emulate_bf16=True)
    return out.T      # [ns, n]


def _inverse_boxcox_fp32_bound(Y0, z, ysd, ymu, lam=0.1):
    """First-order bound of the FP32 kernel's error in Y' = (1 + lam b1)^(1/lam),
    b1 = BC(Y0) + z sd + mu, against the same formula in FP64 on the same z.  The kernel's steps and
    their rounding: Y0 to FP32 (relative u = 2^-24), u = powf(y, lam) (library powf, within 4 ulp
    = 2^-21 relative), BC = (u - 1) / lam, d = z sd + mu, b1 = BC + d, w = 1 + lam b1, Y' = powf(w,
    1 / lam), each operation rounded (u); the FP32 constants lam = 0.1f and 1 / 0.1f differ from
    0.1 and 10 by 1.5e-8 relative.  Doubled for safety."""
    u32, ulp4 = 2.0 ** -24, 2.0 ** -21
    y = np.maximum(np.asarray(Y0, np.float64), 0.0)
    pw = np.power(y, lam)
    bc0 = (pw - 1.0) / lam
    d = z * ysd + ymu
    b1 = bc0 + d
    w = 1.0 + lam * b1
    lny = np.log(np.where(y > 0.0, y, 1.0))
    # error of b1: powf and the FP32 input (through d BC / d y = y^lam / y), the subtraction and
    # division, the FP32 lambda inside the power, then the two sums
    e_b1 = ((ulp4 + lam * u32) * pw + u32 * np.abs(pw - 1.0)) / lam + u32 * np.abs(pw - 1.0) / lam \
        + 1.5e-8 * pw * np.abs(lny) / lam + u32 * (np.abs(bc0) + np.abs(d) + np.abs(b1) + np.abs(z * ysd))
    e_w = lam * e_b1 + u32 * np.abs(w) + 1.5e-8 * np.abs(b1) * lam
    wp = np.maximum(w, 1e-300)
    # powf(w, 1 / 0.1f): 1 / 0.1f is 10 - 1.5e-7, which changes w^10 by 1.5e-7 |ln w| relative
    rel = (1.0 / lam) * e_w / wp + ulp4 + 1.5e-7 * np.abs(np.log(wp))
    yr = np.power(np.maximum(w, 0.0), 1.0 / lam)
    return 2.0 * (rel * yr) + 1e-30


@pytest.mark.parametrize("n", [1000, 2 * 152 * 128 + 77])
def test_forward_matches_oracle_mlp(h2, n):
    """n = 1000: eight tiles, one per CTA; 2 * 152 * 128 + 77: every CTA of the persistent grid
    takes two or three tiles in turn (the barriers' phases carry from tile to tile), the last
    one ragged."""
    check_forward_against_oracle(h2, n)


def check_forward_against_oracle(mech, n):
    """The forward pass on n random states of mech against the oracle's BF16 emulation: z to
    1e-2, the trust-box flags exactly, the inverse Box-Cox on the device's own z to FP32 rounding."""
    dm = cg.Mechanism(mech)
    T, p, Y = random_states(mech, n, 9, "H2", Tlo=300.0, Thi=2500.0)
    x = osur.features(T, p, Y)
    prm = _random_params(mech.ns, 3)
    prm["x_mean"] = x.mean(axis=0)
    prm["x_std"] = _std(x)
    prm["y_mean"] = 0.01 * np.arange(mech.ns)
    prm["y_std"] = 0.05 + 0.01 * np.arange(mech.ns)
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
    # the compensated first layer: a plain BF16 one would sit much farther from the oracle
    xz = (osur.features(T, p, Y) - prm["x_mean"]) / prm["x_std"]
    W32 = [np.asarray(w, np.float32).astype(np.float64) for w in prm["W"]]
    b32 = [np.asarray(bb, np.float32).astype(np.float64) for bb in prm["b"]]
    zp, _ = omlp.forward([omlp.bf16_round(W32[0])] + W32[1:], b32, omlp.bf16_round(xz), emulate_bf16=True)
    assert np.sqrt(np.mean(dz ** 2)) < 0.5 * np.sqrt(np.mean((zp.T - zr) ** 2))
    assert np.array_equal(box.cpu().numpy().astype(bool), T > 2000.0)
    # inverse transform on the device's own network output z: Y' = BC^-1(BC(Y0) + z sd + mu),
    # within the FP32 rounding of the kernel's arithmetic
    ysd = np.float32(prm["y_std"]).astype(np.float64)[:, None]
    ymu = np.float32(prm["y_mean"]).astype(np.float64)[:, None]
    yr = osur.boxcox_inv(osur.boxcox(Y) + z * ysd + ymu)
    yg = ynet.cpu().numpy().astype(np.float64)
    tol = _inverse_boxcox_fp32_bound(Y, z, ysd, ymu)
    assert np.all(np.abs(yg - yr) <= tol), np.max(np.abs(yg - yr) / tol)


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
        assert rel < 1e-2 and relb < 1e-2, (l, rel, relb)


def _split_rows(x, pad):
    """[x_hi | x_lo | x_hi | 0] BF16 rows (the trainer's compensated input layout)."""
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    xh = xt.to(torch.bfloat16)
    xl = (xt - xh.float()).to(torch.bfloat16)
    n, c = x.shape
    X = torch.zeros((n, pad), dtype=torch.bfloat16, device="cuda")
    X[:, :c], X[:, c:2 * c], X[:, 2 * c:3 * c] = xh, xl, xh
    return X


def test_normalize_writes_compensated_rows():
    from paper_2312_13513_gb300 import _lib
    from paper_2312_13513_gb300.train import PAD
    rng = np.random.default_rng(21)
    n, c = 1000, 11
    x = (rng.standard_normal((n, c)) * 300.0 + 1000.0).astype(np.float32)
    mean = np.float32(rng.standard_normal(c) * 10.0 + 1000.0)
    sd = np.float32(np.abs(rng.standard_normal(c)) * 100.0 + 1.0)
    xd = torch.tensor(x, device="cuda")
    md, sdd = torch.tensor(mean, device="cuda"), torch.tensor(sd, device="cuda")
    X = torch.full((n, PAD), 7.0, dtype=torch.bfloat16, device="cuda")
    cg.check(_lib.load().chem_train_normalize(cg._ptr(xd), n, c, cg._ptr(md), cg._ptr(sdd), cg._ptr(X), PAD,
                                              None, 0, None, None, None, None))
    torch.cuda.synchronize()
    v = (xd - md) / sdd
    want = _split_rows(v.cpu().numpy(), PAD)
    assert torch.equal(X, want)


def test_trainer_compensated_first_layer_matches_oracle():
    """Unrounded FP32 weights and inputs: the trainer's first layer is the compensated product."""
    from paper_2312_13513_gb300.train import PAD, Trainer
    rng = np.random.default_rng(23)
    B, nin, nout = 256, 11, 9
    dims = [nin, 512, 512, 512, 512, nout]
    W = [np.float32(rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i])).astype(np.float64)
         for i in range(5)]
    b = [np.float32(0.1 * rng.standard_normal(dims[i + 1])).astype(np.float64) for i in range(5)]
    X = np.float32(rng.standard_normal((B, nin)) * 2.0).astype(np.float64)
    T = rng.standard_normal((B, nout))
    tr = Trainer(nin, nout, B, W=W, b=b)
    Xd = _split_rows(X, PAD)
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    out = torch.empty((B, nout), dtype=torch.float32, device="cuda")
    tr.forward(Xd, out)
    tr.backward(Td)
    dW, _ = tr.get(1)
    o_out, cache = omlp.forward(W, b, X, emulate_bf16=True)
    got = out.cpu().numpy()
    assert np.max(np.abs(got - o_out)) <= 1e-2 * max(1.0, np.max(np.abs(o_out)))
    # a plain BF16 first layer would sit much farther from the compensated oracle
    o_plain, _ = omlp.forward([omlp.bf16_round(W[0])] + W[1:], b, omlp.bf16_round(X), emulate_bf16=True)
    e_gpu = np.sqrt(np.mean((got - o_out) ** 2))
    e_plain = np.sqrt(np.mean((o_plain - o_out) ** 2))
    assert e_gpu < 0.5 * e_plain, (e_gpu, e_plain)
    gW, _ = omlp.backward(W, b, cache, o_out, T)
    rel = np.linalg.norm(dW[0] - gW[0]) / np.linalg.norm(gW[0])
    assert rel < 2e-2, rel


def test_adam_step_matches_oracle():
    """Three Adam steps on three different batches: after each step the device's FP32 master
    weights match the oracle's Adam (FP64 moments carried across the steps) applied to the
    device's own gradients of that step, so the moment buffers and the step counter of the
    bias correction are checked beyond the first step."""
    from paper_2312_13513_gb300.train import PAD, Trainer
    W, b, X, T = _small_problem(2)
    B, nin = X.shape
    tr = Trainer(nin, T.shape[1], B, W=W, b=b)
    params = [np.asarray(w, np.float64) for w in W] + [np.asarray(x, np.float64) for x in b]
    m = [np.zeros_like(x) for x in params]
    v = [np.zeros_like(x) for x in params]
    rng = np.random.default_rng(12)
    for step in (1, 2, 3):
        Xs = X if step == 1 else omlp.bf16_round(rng.standard_normal(X.shape))
        Ts = T if step == 1 else rng.standard_normal(T.shape)
        Xd = torch.zeros((B, PAD), dtype=torch.bfloat16, device="cuda")
        Xd[:, :nin] = torch.tensor(Xs, dtype=torch.float32).to(torch.bfloat16)
        Td = torch.tensor(Ts, dtype=torch.float32, device="cuda")
        tr.forward(Xd)
        tr.backward(Td)
        dW, db = tr.get(1)
        tr.adam(1e-3)
        W1, b1 = tr.get(0)
        grads = [np.asarray(g, np.float64) for g in dW] + [np.asarray(g, np.float64) for g in db]
        params, m, v = omlp.adam_step(params, grads, m, v, step, lr=1e-3)
        got = [np.asarray(w, np.float64) for w in W1] + [np.asarray(x, np.float64) for x in b1]
        for r, g in zip(params, got):
            assert np.max(np.abs(r - g)) <= 2e-6, step
        # the next step starts from the device's weights (FP32 master copies)
        params = got


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


# ---------------------------------------------------------------------------------------------
# the trained model shipped with the package
# ---------------------------------------------------------------------------------------------
MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2312_13513_gb300",
                     "models", "h2_quasi_dns.chemsur")


@pytest.mark.skipif(not os.path.exists(MODEL), reason="no trained model in the package")
def test_trained_surrogate_heat_release_error_vs_oracle(h2, om_h2):
    """The shipped H2 model on a sample of a quasi-DNS-shaped field it was not trained on: field
    L1 heat-release error of the surrogate step against the FP64 oracle <= 1 %, every cell
    conserves the elements and its enthalpy."""
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=1 << 21, seed=4242)
    rng = np.random.default_rng(5)
    s = np.sort(rng.choice(f["T"].size, 20000, replace=False))
    T0, p, Y0 = f["T"][s], f["p"][s], f["Y"][:, s]
    dm = cg.Mechanism(h2)
    model = cg.Surrogate(dm, path=MODEL)
    Td, pd, Yd = to_dev(T0, p, Y0)
    route = torch.empty(T0.size, dtype=torch.int8, device="cuda")
    cg.surrogate_advance(model, Td, pd, Yd, 5e-7, route=route)
    torch.cuda.synchronize()
    Ys = Yd.cpu().numpy()
    T1, Y1 = om_h2.advance(T0, p, Y0, 5e-7, 1e-6, 1e-10)[:2]
    q_ref = np.array([osur.heat_release(om_h2, T0[i], p[i], Y0[:, i], Y1[:, i], 5e-7) for i in range(T0.size)])
    q_sur = np.array([osur.heat_release(om_h2, T0[i], p[i], Y0[:, i], Ys[:, i], 5e-7) for i in range(T0.size)])
    err = osur.hrr_error(q_sur, q_ref)
    assert err <= 0.01, err
    A = osur.element_mass_matrix(h2)
    assert np.max(np.abs(A @ Ys - A @ Y0)) <= 1e-9
    # network-route cells: temperature from enthalpy conservation (Newton to 1e-9)
    net = np.where(route.cpu().numpy() == 0)[0][::50]
    assert net.size > 0
    h0 = np.array([om_h2.enthalpy_mass(T0[i], Y0[:, i]) for i in net])
    Tn = Td.cpu().numpy()
    h1 = np.array([om_h2.enthalpy_mass(Tn[i], Ys[:, i]) for i in net])
    assert np.max(np.abs(h1 - h0) / np.abs(h0).max()) <= 1e-8


def test_trained_network_gains_over_frozen_chemistry_and_an_untrained_network(h2, om_h2):
    """What the training buys: on held-out quasi-DNS cells the shipped model's heat-release error
    is <= 1 %, frozen chemistry (no change over the step) is off by 100 % by construction, and a
    network with the same shape, statistics and trust box but untrained weights is at least ten
    times worse than the trained one."""
    from paper_2312_13513_gb300 import train as trn
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=1 << 21, seed=4343)
    rng = np.random.default_rng(6)
    s = np.sort(rng.choice(f["T"].size, 5000, replace=False))
    T0, p, Y0 = f["T"][s], f["p"][s], f["Y"][:, s]
    dm = cg.Mechanism(h2)
    T1, Y1 = om_h2.advance(T0, p, Y0, 5e-7, 1e-6, 1e-10)[:2]
    q_ref = np.array([osur.heat_release(om_h2, T0[i], p[i], Y0[:, i], Y1[:, i], 5e-7) for i in range(T0.size)])

    def err_of(model):
        Td, pd, Yd = to_dev(T0, p, Y0)
        cg.surrogate_advance(model, Td, pd, Yd, 5e-7)
        torch.cuda.synchronize()
        Ys = Yd.cpu().numpy()
        q = np.array([osur.heat_release(om_h2, T0[i], p[i], Y0[:, i], Ys[:, i], 5e-7) for i in range(T0.size)])
        return osur.hrr_error(q, q_ref)

    trained = err_of(cg.Surrogate(dm, path=MODEL))
    prm = trn.load_model_params(MODEL)
    r = np.random.default_rng(7)
    prm["W"] = [r.standard_normal(w.shape) / np.sqrt(w.shape[1]) for w in prm["W"]]
    prm["b"] = [np.zeros_like(b) for b in prm["b"]]
    untrained = err_of(cg.Surrogate(dm, prm))
    frozen = osur.hrr_error(np.zeros_like(q_ref), q_ref)
    assert trained <= 0.01, trained
    assert frozen == pytest.approx(1.0)
    assert untrained >= 10.0 * trained, (untrained, trained)
