"""The seeded input generators hold to the recipes the workloads state (no arithmetic of the
method lives here): the Gaussian random field's statistics, the quasi-DNS field's perturbation
amplitudes and normalisation, and the LES field's mixture-fraction distribution."""
import numpy as np
import pytest

from synth.states import gaussian_random_field, les_field, load_table, quasi_dns_field


def test_gaussian_random_field_statistics():
    """Zero mean, unit variance, periodic, and the correlation of a Gaussian spectral filter
    exp(-k^2 l^2 / 2) on white noise: exp(-r^2 / (4 l^2)) at lag r."""
    rng = np.random.default_rng(3)
    ell = 4.0
    g = gaussian_random_field((128, 128, 128), ell, rng)    # ~4000 correlation volumes
    assert abs(g.mean()) < 1e-12 and g.std() == pytest.approx(1.0, rel=1e-12)
    for r in (2, 4, 8):
        rho = np.mean([np.mean(g * np.roll(g, r, axis=a)) for a in range(3)])
        assert rho == pytest.approx(np.exp(-r * r / (4 * ell * ell)), abs=0.03), r


def test_quasi_dns_field_recipe():
    """Mass fractions non-negative and summing to one; T perturbed by 5 % (relative standard
    deviation of T over the unperturbed profile), p at one atmosphere; deterministic per seed."""
    tab = load_table("h2_flamelet.npz")
    f = quasi_dns_field(tab, n=32 * 32 * 32, seed=5, grid=32, period=32)
    assert f["Y"].shape[1] == f["T"].size == 32 ** 3
    assert np.all(f["Y"] >= 0.0) and np.allclose(f["Y"].sum(axis=0), 1.0, rtol=0, atol=1e-14)
    base = np.interp(f["c"], tab["c"], tab["T"])
    assert np.std(f["T"] / base - 1.0) == pytest.approx(0.05, rel=0.1)
    assert np.all(f["p"] == 1.01325e6)
    g = quasi_dns_field(tab, n=32 * 32 * 32, seed=5, grid=32, period=32)
    assert np.array_equal(f["T"], g["T"]) and np.array_equal(f["Y"], g["Y"])


def test_les_field_mixture_fraction_is_beta_distributed():
    """Mixture fraction Beta-distributed with the stated mean 0.3 and variance 0.05; T clipped to
    [300, 2200] K; mass fractions normalised."""
    f = les_field(load_table("ch4_flamelet.npz"), n=200000, seed=7)
    assert f["Z"].mean() == pytest.approx(0.3, abs=0.005)
    assert f["Z"].var() == pytest.approx(0.05, abs=0.002)
    assert f["T"].min() >= 300.0 and f["T"].max() <= 2200.0
    assert np.allclose(f["Y"].sum(axis=0), 1.0, rtol=0, atol=1e-14) and np.all(f["Y"] >= 0.0)


@pytest.mark.parametrize("which,ns,nr,n3,ntroe,elements", [
    ("h2", 9, 25, 4, 1, ["H", "O", "N"]),
    ("ch4", 53, 325, 30, 25, ["C", "H", "O", "N"])])
def test_synthetic_mechanisms_have_the_stated_shapes(which, ns, nr, n3, ntroe, elements, request):
    """Species, reaction, third-body and fall-off counts and elements of the H2/air- and
    CH4/air-shaped mechanisms; log10 A in [8, 14], b in [-1, 1], Ea in [0, 40] kcal/mol,
    collision efficiencies other than 1 in [0.5, 12]."""
    m = request.getfixturevalue(which)
    rt = np.asarray(m.rtype)
    assert (m.ns, m.nr) == (ns, nr) and list(m.elements) == elements
    assert int(np.sum(rt == 1)) == n3 and int(np.sum(rt == 2)) == ntroe
    lA = np.log10(np.asarray(m.A))
    assert lA.min() >= 8.0 and lA.max() <= 14.0
    assert np.all(np.abs(m.b) <= 1.0) and np.all((np.asarray(m.Ea) >= 0.0) & (np.asarray(m.Ea) <= 40000.0))
    e = np.asarray(m.eff)[rt != 0]
    e = e[e != 1.0]
    assert e.size and e.min() >= 0.5 and e.max() <= 12.0
