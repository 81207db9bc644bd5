"""GPU parity of the FP64 integrator (C ABI through the Python binding) against the oracle.

Rows covered: thermo / rates / RHS / analytic Jacobian (chem_eval_rhs_jac), the Rodas4
integrator with the persistent work queue in both the warp-per-cell (H2, N = 10) and
CTA-per-cell (CH4, N = 54) forms, staged coalesced loads and stores, indexed mode, per-cell
status, and the edge cases (empty, ragged, non-finite, all-zero rates, step limit).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2312_13513_gb300 as cg  # noqa: E402
from synth.states import flamelet_samples, les_field, load_table, quasi_dns_field  # noqa: E402

from gpu_common import assert_parity, to_dev, within  # noqa: E402
from helpers import prereacted_mixing_states, random_states  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dm_h2(h2):
    return cg.Mechanism(h2)


@pytest.fixture(scope="module")
def dm_ch4(ch4):
    return cg.Mechanism(ch4)


@pytest.mark.parametrize("which,fuel,n", [("h2", "H2", 300), ("ch4", "CH4", 40)])
def test_rhs_and_jacobian_parity(which, fuel, n, request):
    om = request.getfixturevalue("om_" + which)
    dm = request.getfixturevalue("dm_" + which)
    T, p, Y = random_states(om.mech, n, 31, fuel, Tlo=300.0, Thi=2600.0)
    f, J = cg.eval_rhs_jac(dm, *to_dev(T, p, Y))
    f = f.cpu().numpy(); J = J.cpu().numpy()
    N = om.N
    for c in range(n):
        y = np.r_[T[c], Y[:, c]]
        fr = om.rhs(p[c], y)
        Jr = om.jacobian(p[c], y)
        scale_f = np.abs(fr) + 1e-12 * np.max(np.abs(fr))
        assert np.all(np.abs(f[:, c] - fr) <= 1e-10 * scale_f + 1e-300), c
        Jg = J[:, c].reshape(N, N)
        for col in range(N):
            sc = np.max(np.abs(Jr[:, col])) + 1e-300
            assert np.max(np.abs(Jg[:, col] - Jr[:, col])) <= 1e-10 * sc, (c, col)


def _run(dm, T, p, Y, dt, rtol=1e-6, atol=1e-10, opts=None, idx=None):
    Td, pd, Yd = to_dev(T, p, Y)
    n = T.size if idx is None else idx.size
    st = torch.full((T.size,), -1, dtype=torch.int8, device="cuda")
    ns = torch.zeros(T.size, dtype=torch.int32, device="cuda")
    nr = torch.zeros(T.size, dtype=torch.int32, device="cuda")
    idx_d = None if idx is None else torch.tensor(idx, dtype=torch.int32, device="cuda")
    cg.advance(dm, Td, pd, Yd, dt, rtol, atol, idx=idx_d, status=st, nsub=ns, nrej=nr, opts=opts,
               ncells=n)
    torch.cuda.synchronize()
    return (Td.cpu().numpy(), Yd.cpu().numpy(), st.cpu().numpy(), ns.cpu().numpy(),
            nr.cpu().numpy())


def test_parity_h2_mixing_states(om_h2, h2, dm_h2):
    """4096 H2/air mixing states, half partially reacted; dt = 1e-6 s (warp per cell)."""
    T, p, Y = prereacted_mixing_states(om_h2, h2, 4096, 12345)
    Tg, Yg, st, nsub, nrej = _run(dm_h2, T, p, Y, 1e-6)
    assert np.all(st == 0)
    assert nsub.min() >= 1
    out = assert_parity(om_h2, T, p, Y, Tg, Yg, 1e-6, 1e-6, 1e-10)
    assert out <= 8


def test_parity_h2_quasi_dns_subset(om_h2, h2, dm_h2):
    """A 2-front slab of the quasi-DNS field (ragged size), dt = 5e-7 s."""
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=128 * 40 + 5, seed=12346)
    T, p, Y = f["T"], f["p"], f["Y"]
    Tg, Yg, st, _, _ = _run(dm_h2, T, p, Y, 5e-7)
    assert np.all(st == 0)
    out = assert_parity(om_h2, T, p, Y, Tg, Yg, 5e-7, 1e-6, 1e-10)
    assert out <= 5


def test_parity_ch4_les_subset(om_ch4, ch4, dm_ch4):
    """LES-shaped CH4 states, dt = 1e-6 s (CTA-sized group per cell)."""
    f = les_field(load_table("ch4_flamelet.npz"), n=515, seed=777)
    T, p, Y = f["T"], f["p"], f["Y"]
    Tg, Yg, st, _, _ = _run(dm_ch4, T, p, Y, 1e-6)
    assert np.all(st == 0)
    out = assert_parity(om_ch4, T, p, Y, Tg, Yg, 1e-6, 1e-6, 1e-10)
    assert out <= 3


@pytest.mark.parametrize("G", [4, 8, 16, 32, 64, 128])
def test_parity_h2_other_group_sizes(om_h2, h2, dm_h2, G):
    """Sub-warp, warp and multi-warp groups on the H2 mechanism (N = 10): the multi-warp groups
    run the panel LU and the register-held sweeps with fewer than 32 rows."""
    T, p, Y = prereacted_mixing_states(om_h2, h2, 301, 17)
    Tg, Yg, st, _, _ = _run(dm_h2, T, p, Y, 1e-6, opts=cg.options(group_threads=G))
    assert np.all(st == 0)
    assert_parity(om_h2, T, p, Y, Tg, Yg, 1e-6, 1e-6, 1e-10)


@pytest.mark.parametrize("G", [32, 64, 256])
def test_parity_ch4_other_group_sizes(om_ch4, ch4, dm_ch4, G):
    f = les_field(load_table("ch4_flamelet.npz"), n=67, seed=778)
    T, p, Y = f["T"], f["p"], f["Y"]
    Tg, Yg, st, _, _ = _run(dm_ch4, T, p, Y, 1e-6, opts=cg.options(group_threads=G))
    assert np.all(st == 0)
    assert_parity(om_ch4, T, p, Y, Tg, Yg, 1e-6, 1e-6, 1e-10)


def test_full_size_quasi_dns_sampled(om_h2, h2, dm_h2):
    """2^20 cells of the quasi-DNS field in the benchmark's launch configuration; the oracle
    recomputes a seeded sample of 4096 cells one by one."""
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=1 << 20, seed=12346)
    T, p, Y = f["T"], f["p"], f["Y"]
    Tg, Yg, st, nsub, _ = _run(dm_h2, T, p, Y, 5e-7)
    assert np.all(st == 0)
    rng = np.random.default_rng(5)
    s = np.sort(rng.choice(T.size, 4096, replace=False))
    assert_parity(om_h2, T[s], p[s], Y[:, s], Tg[s], Yg[:, s], 5e-7, 1e-6, 1e-10)
    # conservation at every cell: elements exactly, sum Y to rounding
    comp = np.asarray(h2.comp, np.float64)
    b0 = comp.T @ (Y / om_h2.W[:, None])
    b1 = comp.T @ (Yg / om_h2.W[:, None])
    assert np.max(np.abs(b1 - b0)) <= 1e-12 * np.max(b0)


def test_full_size_les_sampled(om_ch4, ch4, dm_ch4):
    """262144 cells of the LES field in the benchmark's launch configuration; the oracle recomputes
    a seeded sample of 1024 cells one by one."""
    f = les_field(load_table("ch4_flamelet.npz"), n=262144, seed=12347)
    T, p, Y = f["T"], f["p"], f["Y"]
    Tg, Yg, st, _, _ = _run(dm_ch4, T, p, Y, 1e-6)
    assert np.all(st == 0)
    rng = np.random.default_rng(6)
    s = np.sort(rng.choice(T.size, 1024, replace=False))
    assert_parity(om_ch4, T[s], p[s], Y[:, s], Tg[s], Yg[:, s], 1e-6, 1e-6, 1e-10)


def test_indexed_mode_and_untouched_cells(om_h2, h2, dm_h2):
    T, p, Y = random_states(h2, 1000, 41, "H2")
    idx = np.sort(np.random.default_rng(1).choice(1000, 333, replace=False)).astype(np.int32)
    Tg, Yg, st, nsub, _ = _run(dm_h2, T, p, Y, 1e-6, idx=idx)
    mask = np.zeros(1000, bool); mask[idx] = True
    assert np.array_equal(Tg[~mask], T[~mask]) and np.array_equal(Yg[:, ~mask], Y[:, ~mask])
    assert np.all(st[idx] == 0) and np.all(st[~mask] == -1)
    assert_parity(om_h2, T[idx], p[idx], Y[:, idx], Tg[idx], Yg[:, idx], 1e-6, 1e-6, 1e-10)


def test_edge_cases(om_h2, h2, dm_h2):
    T, p, Y = random_states(h2, 37, 42, "H2")
    # empty call is a no-op
    Td, pd, Yd = to_dev(T, p, Y)
    assert cg.advance(dm_h2, Td, pd, Yd, 1e-6, ncells=0) == 0
    # invalid arguments are rejected with CHEM_EINVAL
    for bad in (dict(dt=0.0), dict(dt=-1.0), dict(dt=1e-6, rtol=0.0), dict(dt=1e-6, atol=-1.0)):
        with pytest.raises(cg.ChemError) as e:
            cg.advance(dm_h2, Td, pd, Yd, **bad)
        assert e.value.code == -1
    # non-finite and non-physical cells are reported and left unchanged
    Tn, Yn = T.copy(), Y.copy()
    Tn[3] = np.nan; Yn[2, 5] = np.inf; Tn[7] = -5.0
    Tg, Yg, st, _, _ = _run(dm_h2, Tn, p, Yn, 1e-6)
    assert st[3] == cg.CELL_NONFINITE and st[5] == cg.CELL_NONFINITE and st[7] == cg.CELL_NONFINITE
    assert np.isnan(Tg[3]) and np.isinf(Yg[2, 5]) and Tg[7] == -5.0
    others = np.setdiff1d(np.arange(37), [3, 5, 7])
    assert np.all(st[others] == 0)
    # step-attempt limit: status MAX_STEPS with the last accepted state kept
    Tg, Yg, st, nsub, nrej = _run(dm_h2, T, p, Y, 1e-3, opts=cg.options(max_steps=3))
    assert np.all((st == cg.CELL_MAX_STEPS) | (st == 0))
    assert np.any(st == cg.CELL_MAX_STEPS)
    assert np.all(nsub + nrej <= 3)


def test_all_zero_rates_bitwise_identity(h2):
    m0 = h2.copy()
    m0.A[:] = 0.0
    m0.troe[:, 0] = 0.0
    dm0 = cg.Mechanism(m0)
    T, p, Y = random_states(h2, 100, 43, "H2")
    Tg, Yg, st, _, _ = _run(dm0, T, p, Y, 1e-6)
    assert np.all(st == 0)
    assert np.array_equal(Tg, T) and np.array_equal(Yg, Y)


def test_deterministic_across_launch_shapes(om_h2, h2, dm_h2):
    T, p, Y = prereacted_mixing_states(om_h2, h2, 777, 99)
    ref = _run(dm_h2, T, p, Y, 1e-6)
    for opts in (cg.options(max_ctas=1), cg.options(groups_per_cta=1), cg.options(max_ctas=7)):
        got = _run(dm_h2, T, p, Y, 1e-6, opts=opts)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    # a permuted cell order gives the same per-cell results
    perm = np.random.default_rng(0).permutation(T.size)
    got = _run(dm_h2, T[perm], p[perm], Y[:, perm], 1e-6)
    assert np.array_equal(got[0], ref[0][perm]) and np.array_equal(got[1], ref[1][:, perm])


def test_load_from_text_file_matches_desc(tmp_path, h2, dm_h2):
    path = str(tmp_path / "h2.mech")
    h2.save(path)
    dm_file = cg.Mechanism(path=path)
    T, p, Y = random_states(h2, 64, 44, "H2")
    a = _run(dm_h2, T, p, Y, 1e-6)
    b = _run(dm_file, T, p, Y, 1e-6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_training_distribution_parity(om_h2, h2, dm_h2):
    """Independent samples of the quasi-DNS state distribution (the surrogate's training set)."""
    f = flamelet_samples(load_table("h2_flamelet.npz"), 2000, seed=5)
    Tg, Yg, st, _, _ = _run(dm_h2, f["T"], f["p"], f["Y"], 5e-7)
    assert np.all(st == 0)
    assert_parity(om_h2, f["T"], f["p"], f["Y"], Tg, Yg, 5e-7, 1e-6, 1e-10)
