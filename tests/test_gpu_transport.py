"""GPU parity of the thermophysical and transport property kernels against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2312_13513_gb300 as cg  # noqa: E402
from oracle import transport as ot  # noqa: E402
from synth.states import les_field, load_table, quasi_dns_field  # noqa: E402
from synth.transport import generate_transport  # noqa: E402

from gpu_common import to_dev  # noqa: E402
from helpers import random_states  # noqa: E402

pytestmark = pytest.mark.gpu


def _states(kind, mech, n, seed):
    if kind == "h2":
        f = quasi_dns_field(load_table("h2_flamelet.npz"), n=n, seed=seed)
    else:
        f = les_field(load_table("ch4_flamelet.npz"), n=n, seed=seed)
    return f["T"], f["p"], f["Y"]


@pytest.mark.parametrize("kind", ["h2", "ch4"])
def test_transport_matches_oracle(kind, h2, ch4):
    mech = h2 if kind == "h2" else ch4
    tr = generate_transport(mech)
    T, p, Y = _states(kind, mech, 700, 41)
    p = p * np.linspace(0.5, 3.0, p.size)              # pressure varies across cells
    dm = cg.Mechanism(mech)
    gt = cg.Transport(dm, tr)
    Td, pd, Yd = to_dev(T, p, Y)
    mu = torch.empty_like(Td); lam = torch.empty_like(Td); D = torch.empty_like(Yd)
    gt(Td, pd, Yd, mu, lam, D)
    torch.cuda.synchronize()
    mu_r, lam_r, D_r = ot.mixture_cells(tr, mech.W, T, p, Y)
    assert np.allclose(mu.cpu().numpy(), mu_r, rtol=1e-11, atol=0)
    assert np.allclose(lam.cpu().numpy(), lam_r, rtol=1e-11, atol=0)
    assert np.allclose(D.cpu().numpy(), D_r, rtol=1e-11, atol=0)


def test_transport_pure_species_and_optional_outputs(h2):
    tr = generate_transport(h2)
    n = h2.ns
    Y = np.eye(n)                                      # cell k holds species k alone
    T = np.linspace(400.0, 2800.0, n)
    p = np.full(n, 1.01325e6)
    dm = cg.Mechanism(h2)
    gt = cg.Transport(dm, tr)
    Td, pd, Yd = to_dev(T, p, Y)
    D = torch.empty_like(Yd)
    gt(Td, pd, Yd, D=D)                                # viscosity and conductivity not requested
    torch.cuda.synchronize()
    for k in range(n):
        _, _, Djk = ot.pure_species(tr, T[k], p[k])
        assert D[k, k].item() == pytest.approx(Djk[k, k], rel=1e-12)


def test_mixture_thermo_matches_oracle(h2, om_h2):
    T, p, Y = random_states(h2, 500, 43, "H2", Tlo=300.0, Thi=2900.0)
    dm = cg.Mechanism(h2)
    Td, _, Yd = to_dev(T, p, Y)
    h = torch.empty_like(Td); cp = torch.empty_like(Td)
    cg.mixture_thermo(dm, Td, Yd, h, cp)
    torch.cuda.synchronize()
    h_r = np.array([om_h2.enthalpy_mass(T[i], Y[:, i]) for i in range(T.size)])
    cp_r = np.array([om_h2.cp_mass(T[i], Y[:, i]) for i in range(T.size)])
    assert np.allclose(h.cpu().numpy(), h_r, rtol=1e-12, atol=1e-6 * np.abs(h_r).max())
    assert np.allclose(cp.cpu().numpy(), cp_r, rtol=1e-12, atol=0)


def test_temperature_from_enthalpy_recovers_temperature(ch4, om_ch4):
    T, p, Y = _states("ch4", ch4, 400, 44)
    h0 = np.array([om_ch4.enthalpy_mass(T[i], Y[:, i]) for i in range(T.size)])
    dm = cg.Mechanism(ch4)
    guess = T + np.where(np.arange(T.size) % 2 == 0, 250.0, -150.0)
    guess = np.clip(guess, 250.0, 3000.0)
    Td, _, Yd = to_dev(guess, p, Y)
    hd = torch.tensor(h0, device="cuda")
    st = torch.full((T.size,), 7, dtype=torch.int8, device="cuda")
    cg.temperature_from_enthalpy(dm, hd, Yd, Td, st)
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    assert np.allclose(Td.cpu().numpy(), T, rtol=1e-9, atol=0)


def test_temperature_from_enthalpy_flags_failures(h2):
    dm = cg.Mechanism(h2)
    T, p, Y = random_states(h2, 4, 45, "H2", Tlo=800.0, Thi=1200.0)
    Td, _, Yd = to_dev(T, p, Y)
    h = torch.tensor([np.nan, 1e30, -1e30, 0.0], device="cuda", dtype=torch.float64)
    st = torch.zeros(4, dtype=torch.int8, device="cuda")
    before = Td.clone()
    cg.temperature_from_enthalpy(dm, h, Yd, Td, st)
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert s[0] == 1 and s[1] == 1 and s[2] == 1
    assert torch.equal(Td[:3], before[:3])             # unconverged cells keep their temperature
