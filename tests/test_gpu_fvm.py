"""GPU parity of the finite-volume species-equation assembly (Alg. 1 and the other terms, ldu and
CSR forms) and of the PaSR factor against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2312_13513_gb300 as cg  # noqa: E402
from oracle import fvm  # noqa: E402
from synth.mesh import box_mesh  # noqa: E402

pytestmark = pytest.mark.gpu


def _terms(m, seed, closed=False):
    rng = np.random.default_rng(seed)
    n, nf, nb = m.n_cells, m.owner.size, m.b_cell.size
    kw = dict(dt=2e-4, rho=rng.uniform(0.3, 1.5, n), rho_old=rng.uniform(0.3, 1.5, n), Y_old=rng.uniform(0, 0.3, n),
              phi=rng.standard_normal(nf) * 1e-3, phi_b=np.zeros(nb) if closed else rng.standard_normal(nb) * 1e-3,
              gamma=rng.uniform(1e-5, 5e-4, n), gamma_b=rng.uniform(1e-5, 5e-4, nb), Y_b=rng.uniform(0, 0.3, nb),
              S=rng.standard_normal(n), kappa=rng.uniform(0, 1, n))
    return kw


def _dev(kw):
    return {k: (torch.tensor(v, device="cuda") if isinstance(v, np.ndarray) else v) for k, v in kw.items()}


@pytest.mark.parametrize("shape,permute", [((6, 5, 4), True), ((7, 1, 1), False), ((1, 1, 1), False),
                                           ((9, 8, 3), True)])
def test_assembly_matches_the_oracle_matrix(shape, permute):
    m = box_mesh(*shape, seed=11, stretch=2.5, permute=permute)
    kw = _terms(m, 12)
    A, s = fvm.species_matrix(m, **kw)
    lo_r, up_r, dg_r = fvm.ldu(m, A)
    gm = cg.FvMesh(m)
    lo, up, dg, src = gm.assemble(**_dev(kw))
    torch.cuda.synchronize()
    sc = np.max(np.abs(A))
    for got, ref in ((lo, lo_r), (up, up_r), (dg, dg_r)):
        assert np.allclose(got.cpu().numpy(), ref, rtol=1e-13, atol=1e-15 * sc)
    assert np.allclose(src.cpu().numpy(), s, rtol=1e-13, atol=1e-15 * np.max(np.abs(s)))
    # CSR form: the same matrix, columns ascending, diagonal stored
    vals = gm.to_csr(lo, up, dg).cpu().numpy()
    rp, ci = gm.csr_pattern()
    B = np.zeros_like(A)
    for r in range(m.n_cells):
        cols = ci[rp[r]:rp[r + 1]]
        assert np.all(np.diff(cols) > 0) and r in cols
        B[r, cols] = vals[rp[r]:rp[r + 1]]
    assert np.allclose(B, A, rtol=1e-13, atol=1e-15 * sc)


def test_each_term_alone():
    """Every term switched on alone (the others' inputs NULL) against the oracle."""
    m = box_mesh(5, 4, 3, seed=13, stretch=2.0, permute=True)
    kw = _terms(m, 14)
    gm = cg.FvMesh(m)
    groups = [dict(dt=kw["dt"], rho=kw["rho"], rho_old=kw["rho_old"], Y_old=kw["Y_old"]),
              dict(phi=kw["phi"], phi_b=kw["phi_b"], Y_b=kw["Y_b"]),
              dict(gamma=kw["gamma"], gamma_b=kw["gamma_b"], Y_b=kw["Y_b"]),
              dict(S=kw["S"]), dict(S=kw["S"], kappa=kw["kappa"])]
    for g in groups:
        A, s = fvm.species_matrix(m, **g)
        lo, up, dg, src = gm.assemble(**_dev(g))
        torch.cuda.synchronize()
        lo_r, up_r, dg_r = fvm.ldu(m, A)
        assert np.allclose(lo.cpu().numpy(), lo_r, rtol=1e-13, atol=0)
        assert np.allclose(up.cpu().numpy(), up_r, rtol=1e-13, atol=0)
        assert np.allclose(dg.cpu().numpy(), dg_r, rtol=1e-13, atol=0)
        assert np.allclose(src.cpu().numpy(), s, rtol=1e-13, atol=0)


def test_large_mesh_sampled_rows_conservation_and_reproducibility():
    """64^3 permuted stretched mesh: sampled rows against the oracle's row form, the closed-box
    conservation identity 1^T A Y = sum rho V Y / dt for random Y, and bitwise repeat."""
    m = box_mesh(64, 64, 64, seed=15, stretch=2.0, permute=True)
    m.b_type[:] = 0
    kw = _terms(m, 16, closed=True)
    gm = cg.FvMesh(m)
    d = _dev(kw)
    lo, up, dg, src = gm.assemble(**d)
    lo2, up2, dg2, src2 = gm.assemble(**d)
    torch.cuda.synchronize()
    assert torch.equal(lo, lo2) and torch.equal(up, up2) and torch.equal(dg, dg2) and torch.equal(src, src2)
    rng = np.random.default_rng(17)
    cells = rng.choice(m.n_cells, 40, replace=False)
    rows = fvm.species_rows(m, cells, **kw)
    lo_h, up_h, dg_h = lo.cpu().numpy(), up.cpu().numpy(), dg.cpu().numpy()
    for P, (row, sp) in rows.items():
        assert dg_h[P] == pytest.approx(row[P], rel=1e-13)
        for f in np.nonzero(m.owner == P)[0]:
            assert up_h[f] == pytest.approx(row[int(m.neighbour[f])], rel=1e-13, abs=1e-300)
        for f in np.nonzero(m.neighbour == P)[0]:
            assert lo_h[f] == pytest.approx(row[int(m.owner[f])], rel=1e-13, abs=1e-300)
        assert src.cpu().numpy()[P] == pytest.approx(sp, rel=1e-13)
    Y = torch.tensor(rng.uniform(0, 1, m.n_cells), device="cuda")
    own = torch.tensor(m.owner.astype(np.int64), device="cuda")
    nei = torch.tensor(m.neighbour.astype(np.int64), device="cuda")
    r = dg * Y
    r.index_add_(0, own, up * Y[nei])
    r.index_add_(0, nei, lo * Y[own])
    total = float(r.sum())
    want = float((d["rho"] * torch.tensor(m.volume, device="cuda") * Y).sum()) / kw["dt"]
    assert total == pytest.approx(want, rel=1e-11)


def test_pasr_kappa_matches_the_oracle():
    rng = np.random.default_rng(18)
    n = 100000
    tau_c = 10.0 ** rng.uniform(-7, -2, n)
    rho = rng.uniform(0.2, 1.5, n)
    mu = rng.uniform(1e-5, 6e-5, n)
    strain = np.where(rng.uniform(size=n) < 0.05, 0.0, 10.0 ** rng.uniform(1, 5, n))
    delta = rng.uniform(2e-4, 2e-3, n)
    ref = fvm.pasr_kappa(tau_c, rho, mu, strain, delta, 0.17, 0.5)
    t = [torch.tensor(a, device="cuda") for a in (tau_c, rho, mu, strain, delta)]
    k = cg.pasr_kappa(*t, c_s=0.17, c_mix=0.5)
    torch.cuda.synchronize()
    got = k.cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-14, atol=0)
    assert np.all(got[strain == 0.0] == 1.0) and np.all((got >= 0.0) & (got <= 1.0))
