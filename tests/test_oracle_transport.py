"""Pins of the oracle's mixture-averaged transport properties and of the synthetic transport data."""
import numpy as np
import pytest

from oracle import transport as ot
from synth.mechanism import ch4_mechanism, h2_mechanism
from synth.transport import T_FIT, TransportData, generate_transport, omega22

PATM = 1.01325e6


@pytest.fixture(scope="module")
def h2_tr():
    m = h2_mechanism()
    return m, generate_transport(m)


def test_fits_reproduce_kinetic_theory_viscosity(h2_tr):
    """The cubic fits in ln T stay within 1 % of the Chapman-Enskog values they were fitted to."""
    m, tr = h2_tr
    rng = np.random.default_rng(2024)
    W = np.asarray(m.W)
    sigma = 2.5 + 1.1 * np.log1p(W / 4.0) * rng.uniform(0.85, 1.15, m.ns)
    eps = 60.0 + 55.0 * np.log1p(W / 4.0) ** 1.5 * rng.uniform(0.8, 1.25, m.ns)
    for T in (300.0, 800.0, 1500.0, 2900.0):
        mu_fit, _, _ = ot.pure_species(tr, T, PATM)
        mu_ce = 2.6693e-5 * np.sqrt(W * T) / (sigma ** 2 * omega22(T / eps))
        assert np.all(np.abs(mu_fit / mu_ce - 1.0) < 0.01)


def test_pure_species_limit(h2_tr):
    """A cell holding one species has that species' viscosity and conductivity, and its
    diffusion coefficient is the self-diffusion fit."""
    m, tr = h2_tr
    for k in range(m.ns):
        Y = np.zeros(m.ns)
        Y[k] = 1.0
        mu, lam, D = ot.mixture(tr, m.W, 1234.0, PATM, Y)
        mu_k, lam_k, Djk = ot.pure_species(tr, 1234.0, PATM)
        assert mu == pytest.approx(mu_k[k], rel=1e-14)
        assert lam == pytest.approx(lam_k[k], rel=1e-14)
        assert D[k] == pytest.approx(Djk[k, k], rel=1e-14)


def test_wilke_reduces_to_pure_value_for_identical_species():
    """Two species with the same molar mass and viscosity: every Phi_kj = 1, so the mixture
    viscosity is that viscosity at any composition."""
    c = np.array([-10.0, 0.6, 0.01, -0.001])
    tr = TransportData(mu_poly=np.stack([c, c]), lambda_poly=np.stack([c, c]) + [20.0, 0, 0, 0],
                       diff_poly=np.tile(np.array([-5.0, 1.5, 0.0, 0.0]), (2, 2, 1)))
    W = np.array([28.0, 28.0])
    for y0 in (0.1, 0.5, 0.93):
        mu, lam, _ = ot.mixture(tr, W, 1500.0, PATM, np.array([y0, 1.0 - y0]))
        assert mu == pytest.approx(np.exp(ot._poly(c, np.log(1500.0))), rel=1e-14)
        assert lam == pytest.approx(np.exp(ot._poly(c, np.log(1500.0)) + 20.0), rel=1e-14)


def test_mathur_average_lies_between_pure_values():
    m = ch4_mechanism()
    tr = generate_transport(m)
    rng = np.random.default_rng(3)
    for _ in range(20):
        Y = rng.dirichlet(np.ones(m.ns) * 0.3)
        T = rng.uniform(300.0, 2500.0)
        _, lam, _ = ot.mixture(tr, m.W, T, PATM, Y)
        _, lam_k, _ = ot.pure_species(tr, T, PATM)
        present = Y > 0
        assert lam_k[present].min() * (1 - 1e-12) <= lam <= lam_k[present].max() * (1 + 1e-12)


def test_binary_mixture_diffusion_identity(h2_tr):
    """For two species, 1 - Y_1 = Y_2 = X_2 W_2 / W_mix, so D_1m = D_12 W_2 / W_mix and
    D_2m = D_12 W_1 / W_mix."""
    m, tr = h2_tr
    i, j = 0, 1
    W = np.asarray(m.W)
    Y = np.zeros(m.ns)
    Y[i], Y[j] = 0.3, 0.7
    _, _, D = ot.mixture(tr, m.W, 1700.0, PATM, Y)
    _, _, Djk = ot.pure_species(tr, 1700.0, PATM)
    Wmix = 1.0 / (Y[i] / W[i] + Y[j] / W[j])
    assert D[i] == pytest.approx(Djk[i, j] * W[j] / Wmix, rel=1e-13)
    assert D[j] == pytest.approx(Djk[i, j] * W[i] / Wmix, rel=1e-13)


def test_diffusion_scales_inversely_with_pressure_and_viscosity_does_not(h2_tr):
    m, tr = h2_tr
    Y = np.full(m.ns, 1.0 / m.ns)
    mu1, lam1, D1 = ot.mixture(tr, m.W, 1500.0, PATM, Y)
    mu4, lam4, D4 = ot.mixture(tr, m.W, 1500.0, 4 * PATM, Y)
    assert mu4 == mu1 and lam4 == lam1
    assert np.allclose(D4 * 4, D1, rtol=1e-14, atol=0)


def test_trace_species_continuity(h2_tr):
    """Removing a species continuously: the properties at a tiny mass fraction tend to those
    without it."""
    m, tr = h2_tr
    Y = np.full(m.ns, 1.0 / (m.ns - 1))
    Y[3] = 0.0
    base = ot.mixture(tr, m.W, 1500.0, PATM, Y)
    Y2 = Y.copy()
    Y2[3] = 1e-12
    near = ot.mixture(tr, m.W, 1500.0, PATM, Y2 / Y2.sum())
    assert near[0] == pytest.approx(base[0], rel=1e-9)
    assert near[1] == pytest.approx(base[1], rel=1e-9)


def test_wilke_interaction_factors_obey_reciprocity(h2_tr):
    """Wilke's interaction factors satisfy Phi_jk / Phi_kj = (mu_j / mu_k)(W_k / W_j), a property of
    their form (1 + (mu_k/mu_j)^(1/2) (W_j/W_k)^(1/4))^2 / (8 (1 + W_k/W_j))^(1/2).  For a binary
    mixture the rule mu = X1 mu1 / (X1 + X2 Phi12) + X2 mu2 / (X1 Phi21 + X2) at three compositions
    determines Phi12 and Phi21; fitted to the oracle's mixture viscosities of H2 with N2 (molar
    masses 14 times apart), they obey the identity."""
    from scipy.optimize import least_squares
    m, tr = h2_tr
    W = np.asarray(m.W)
    i, j = m.species.index("H2"), m.species.index("N2")
    T = 1500.0
    mu_k, _, _ = ot.pure_species(tr, T, PATM)
    data = []
    for y2 in (0.2, 0.5, 0.8):
        Y = np.zeros(m.ns)
        Y[i], Y[j] = 1.0 - y2, y2
        X = (Y / W) / np.sum(Y / W)
        data.append((X[i], X[j], ot.mixture(tr, W, T, PATM, Y)[0]))

    def resid(v):
        a, b = v
        return [(x1 * mu_k[i] / (x1 + x2 * a) + x2 * mu_k[j] / (x1 * b + x2)) / mu - 1.0 for x1, x2, mu in data]

    fit = least_squares(resid, [1.0, 1.0], bounds=([1e-3, 1e-3], [1e3, 1e3]), xtol=1e-15, ftol=1e-15, gtol=1e-15)
    assert np.max(np.abs(resid(fit.x))) < 1e-12
    a, b = fit.x
    assert b / a == pytest.approx((mu_k[j] / mu_k[i]) * (W[i] / W[j]), rel=1e-8)
