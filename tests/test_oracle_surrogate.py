"""Pins of the oracle's MLP (forward, backward, Adam) and surrogate post-processing."""
import numpy as np
import pytest

from oracle import mlp
from oracle import surrogate as sur
from synth.states import PATM

from helpers import random_states


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1.00390625, 1.01171875, 1.0078125 + 2 ** -8 + 2 ** -20, -2.5, 3.14159265, 0.0,
                  65504.0, 1e-40])
    want = np.array([1.0, 1.0, 1.015625, 1.015625, -2.5, 3.140625, 0.0, 65536.0, 0.0])
    got = mlp.bf16_round(x)
    assert np.array_equal(got[:8], want[:8])
    assert abs(got[8]) < 1e-38


def test_gelu_closed_forms():
    x = np.linspace(-6, 6, 101)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15, rtol=0)
    assert mlp.gelu(np.array([40.0]))[0] == 40.0
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_compensated_first_layer_error_bound():
    """hi + lo represents v to 2^-16 relative (two 8-bit significands); the dropped lo*lo term and
    the rounding of lo bound the product error by 3 * 2^-17 * sum |x_j| |W_ij|, against about
    2^-9 for a plain BF16 product.  BF16-representable operands give the exact product."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal((400, 11)) * np.exp(rng.uniform(-3, 3, (400, 11)))
    W = rng.standard_normal((64, 11))
    exact = x @ W.T
    scale = np.abs(x) @ np.abs(W).T
    err = np.abs(mlp.first_layer(W, x) - exact)
    assert np.all(err <= 3 * 2.0 ** -17 * scale)
    plain = np.abs(mlp.bf16_round(x) @ mlp.bf16_round(W).T - exact)
    assert np.median(plain / scale) > 30 * np.median(err / scale)
    xb, Wb = mlp.bf16_round(x), mlp.bf16_round(W)
    assert np.array_equal(mlp.first_layer(Wb, xb), xb @ Wb.T)
    hi, lo = mlp.split_bf16(x)
    assert np.all(np.abs(hi + lo - x) <= 2.0 ** -16 * np.abs(x))


def _net(rng, dims):
    Ws = [rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]) for i in range(len(dims) - 1)]
    bs = [0.1 * rng.standard_normal(dims[i + 1]) for i in range(len(dims) - 1)]
    return Ws, bs


def test_forward_and_backward_match_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    dims = [11, 16, 16, 16, 9]
    Ws, bs = _net(rng, dims)
    x = rng.standard_normal((7, 11))
    t = rng.standard_normal((7, 9))
    out, cache = mlp.forward(Ws, bs, x, emulate_bf16=False)
    dW, db = mlp.backward(Ws, bs, cache, out, t)
    Wt = [torch.tensor(W, requires_grad=True) for W in Ws]
    bt = [torch.tensor(b, requires_grad=True) for b in bs]
    a = torch.tensor(x)
    for l in range(len(Ws)):
        a = a @ Wt[l].T + bt[l]
        if l < len(Ws) - 1:
            a = torch.nn.functional.gelu(a, approximate="none")
    loss = ((a - torch.tensor(t)) ** 2).mean()
    loss.backward()
    assert np.allclose(out, a.detach().numpy(), rtol=1e-13, atol=1e-13)
    for l in range(len(Ws)):
        assert np.allclose(dW[l], Wt[l].grad.numpy(), rtol=1e-11, atol=1e-14)
        assert np.allclose(db[l], bt[l].grad.numpy(), rtol=1e-11, atol=1e-14)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    Ws, bs = _net(rng, [3, 5, 4, 2])
    x = rng.standard_normal((6, 3))
    t = rng.standard_normal((6, 2))
    out, cache = mlp.forward(Ws, bs, x, emulate_bf16=False)
    dW, db = mlp.backward(Ws, bs, cache, out, t)
    h = 1e-6
    for l in range(3):
        for idx in [(0, 0), (1, 2), (Ws[l].shape[0] - 1, Ws[l].shape[1] - 1)]:
            Wp = [W.copy() for W in Ws]; Wp[l][idx] += h
            Wm = [W.copy() for W in Ws]; Wm[l][idx] -= h
            lp = mlp.mse_loss(mlp.forward(Wp, bs, x, False)[0], t)
            lm = mlp.mse_loss(mlp.forward(Wm, bs, x, False)[0], t)
            assert abs(dW[l][idx] - (lp - lm) / (2 * h)) < 1e-7


def test_adam_first_step_is_signed_lr():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -1e-3, 2.0])]
    m = [np.zeros(3)]; v = [np.zeros(3)]
    p1, _, _ = mlp.adam_step([p[0].copy()], g, m, v, 1, lr=1e-2, eps=0.0)
    assert np.allclose(p1[0] - p[0], -1e-2 * np.sign(g[0]), rtol=1e-12)


def test_adam_constant_gradient_three_steps():
    """Kingma & Ba's Adam with a constant gradient g: the moments are geometric sums,
    m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so the bias-corrected ratio is g / |g| and every
    step moves each parameter by -lr sign(g) (eps = 0).  Checked after each of three steps, with
    the moments themselves."""
    b1, b2, lr = 0.9, 0.999, 1e-2
    p0 = np.array([1.0, -2.0, 3.0, 0.25])
    g = np.array([0.5, -1e-3, 2.0, -7.0])
    p = [p0.copy()]; m = [np.zeros(4)]; v = [np.zeros(4)]
    for t in (1, 2, 3):
        p, m, v = mlp.adam_step(p, [g.copy()], m, v, t, lr=lr, beta1=b1, beta2=b2, eps=0.0)
        assert np.allclose(m[0], (1.0 - b1 ** t) * g, rtol=1e-14, atol=0)
        assert np.allclose(v[0], (1.0 - b2 ** t) * g * g, rtol=1e-13, atol=0)
        assert np.allclose(p[0] - p0, -t * lr * np.sign(g), rtol=1e-12, atol=0)


def test_adam_alternating_gradient_three_steps():
    """Gradients g, -g, g: expanding the moment recursion by hand,
    m_1 = (1 - b1) g, m_2 = -(1 - b1)^2 g, m_3 = (1 - b1)(1 - b1 (1 - b1)) g, while v_t stays
    (1 - b2^t) g^2; the three steps are therefore -lr s, lr (1 - b1) / (1 + b1) s and
    -lr (1 - b1 + b1^2) / (1 + b1 + b1^2) s with s = sign(g) (eps = 0)."""
    b1, b2, lr = 0.9, 0.999, 1e-2
    g = np.array([0.3, -4.0, 1e-2])
    s = np.sign(g)
    want_m = [(1 - b1) * g, -(1 - b1) ** 2 * g, (1 - b1) * (1 - b1 * (1 - b1)) * g]
    want_step = [-lr * s, lr * (1 - b1) / (1 + b1) * s, -lr * (1 - b1 + b1 * b1) / (1 + b1 + b1 * b1) * s]
    p = [np.zeros(3)]; m = [np.zeros(3)]; v = [np.zeros(3)]
    for t in (1, 2, 3):
        before = p[0].copy()
        gt = g if t != 2 else -g
        p, m, v = mlp.adam_step(p, [gt.copy()], m, v, t, lr=lr, beta1=b1, beta2=b2, eps=0.0)
        assert np.allclose(m[0], want_m[t - 1], rtol=1e-13, atol=0)
        assert np.allclose(v[0], (1.0 - b2 ** t) * g * g, rtol=1e-13, atol=0)
        assert np.allclose(p[0] - before, want_step[t - 1], rtol=1e-11, atol=0)


def test_boxcox_roundtrip_and_log_limit():
    y = np.logspace(-30, 0, 61)
    assert np.allclose(sur.boxcox_inv(sur.boxcox(y)), y, rtol=1e-9, atol=0)
    assert np.allclose(sur.boxcox(y, lam=1e-9), np.log(y), rtol=1e-6)
    assert sur.boxcox(np.array([-1e-3]))[0] == -1.0 / sur.LAMBDA
    assert sur.boxcox_inv(np.array([-20.0]))[0] == 0.0


def test_projection_conserves_and_is_weighted_least_squares(h2, om_h2):
    T, p, Y = random_states(h2, 5, 3, "H2")
    rng = np.random.default_rng(0)
    A = sur.element_mass_matrix(h2)
    assert np.allclose(A.sum(axis=0), 1.0, rtol=1e-14)
    for i in range(T.size):
        Y0 = Y[:, i]
        Yp = Y0 * (1.0 + 0.02 * rng.standard_normal(Y0.size))
        Ypp, ok = sur.project(h2, Y0, Yp)
        assert ok
        assert np.max(np.abs(A @ Ypp - A @ Y0)) < 1e-13
        # KKT: D^{-1} (Y'' - Y') lies in the row space of A
        D = Yp + 1e-12
        r = (Ypp - Yp) / D
        lam, *_ = np.linalg.lstsq(A.T, r, rcond=None)
        assert np.max(np.abs(A.T @ lam - r)) < 1e-9 * max(1.0, np.max(np.abs(r)))
        Yq, ok = sur.project(h2, Y0, Y0)
        assert ok and np.max(np.abs(Yq - Y0)) < 1e-15


def test_temperature_from_enthalpy(h2, om_h2):
    T, p, Y = random_states(h2, 4, 8, "H2", Tlo=300.0, Thi=2500.0)
    for i in range(T.size):
        h0 = om_h2.enthalpy_mass(T[i], Y[:, i])
        Tn, ok = sur.temperature_from_enthalpy(om_h2, h0, Y[:, i], 1000.0)
        assert ok and abs(Tn - T[i]) < 1e-8 * T[i]


def test_heat_release_matches_energy_equation(h2, om_h2):
    """For a tiny step, -rho sum h_k dY_k/(W_k dt) equals rho cp dT/dt."""
    T, p, Y = random_states(h2, 4, 9, "H2")
    for i in range(T.size):
        y0 = np.r_[T[i], Y[:, i]]
        qs = []
        for dt in (2e-14, 1e-14):      # Richardson: remove the O(dt) truncation of the quotient
            y1, st, _, _ = om_h2.rodas4(p[i], y0, dt, 1e-12, 1e-22)
            qs.append(sur.heat_release(om_h2, T[i], p[i], Y[:, i], y1[1:], dt))
        q = 2.0 * qs[1] - qs[0]
        f = om_h2.rhs(p[i], y0)
        q_ref = om_h2.density(T[i], p[i], Y[:, i]) * om_h2.cp_mass(T[i], Y[:, i]) * f[0]
        assert abs(q - q_ref) <= 1e-5 * abs(q_ref)


def test_features_are_T_log_p_and_boxcox():
    """The feature row [T, ln p, BC(Y_1..Y_ns)]: the pressure feature of p^2 is twice that of p
    (a logarithm), T passes through, and the composition columns are the Box-Cox transforms
    checked above."""
    rng = np.random.default_rng(4)
    n, ns = 5, 4
    T = rng.uniform(300, 2500, n)
    p = rng.uniform(2.0, 50.0, n)
    Y = rng.dirichlet(np.ones(ns), n).T
    x1, x2 = sur.features(T, p, Y), sur.features(T, p * p, Y)
    assert x1.shape == (n, ns + 2)
    assert np.array_equal(x1[:, 0], T)
    assert np.allclose(x2[:, 1], 2.0 * x1[:, 1], rtol=1e-14, atol=0)
    assert np.array_equal(x1[:, 2:], sur.boxcox(Y).T)


def test_bf16_emulation_rounds_where_the_gpu_holds_bf16():
    """With BF16 emulation, every hidden activation is a BF16 value (a fixed point of the
    rounding), the weights of layers 2-5 enter rounded (rounding them beforehand changes
    nothing), and the first layer is compensated (rounding its weights beforehand does change
    the output)."""
    rng = np.random.default_rng(6)
    Ws, bs = _net(rng, [11, 32, 32, 32, 32, 9])
    x = rng.standard_normal((8, 11)) * 3.0
    out, cache = mlp.forward(Ws, bs, x, emulate_bf16=True)
    for a in cache["a"][1:]:
        assert np.array_equal(mlp.bf16_round(a), a)
    pre = [Ws[0]] + [mlp.bf16_round(W) for W in Ws[1:]]
    assert np.array_equal(mlp.forward(pre, bs, x, emulate_bf16=True)[0], out)
    pre0 = [mlp.bf16_round(Ws[0])] + Ws[1:]
    assert not np.array_equal(mlp.forward(pre0, bs, x, emulate_bf16=True)[0], out)


def test_heat_release_error_closed_forms():
    """The field L1-relative heat-release error sum |q - q_ref| / sum |q_ref|: zero for the
    reference itself, exactly 1 for twice the reference and for a zero field, 2 for its negation
    (a sign flip counts in full), and 1/2 against a reference twice the field: it normalises by
    the reference, not by the surrogate."""
    q_ref = np.array([3.0, -1.0, 0.5, 8.0])
    assert sur.hrr_error(q_ref, q_ref) == 0.0
    assert sur.hrr_error(2.0 * q_ref, q_ref) == pytest.approx(1.0, rel=1e-15)
    assert sur.hrr_error(np.zeros(4), q_ref) == pytest.approx(1.0, rel=1e-15)
    assert sur.hrr_error(-q_ref, q_ref) == pytest.approx(2.0, rel=1e-15)
    assert sur.hrr_error(q_ref, 2.0 * q_ref) == pytest.approx(0.5, rel=1e-15)
