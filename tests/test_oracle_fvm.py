"""Pins of the oracle's finite-volume species-equation assembly (Alg. 1 and the other terms) and of
its PaSR factor."""
import numpy as np
import pytest

from oracle import fvm
from synth.mesh import box_mesh


def test_uniform_diffusion_is_the_seven_point_stencil():
    """Unit box, n cells per side, h = 1/n: a_f = gamma h^2 / h = gamma h on internal faces and
    gamma h^2 / (h/2) = 2 gamma h on the fixed-value x sides."""
    n, g = 4, 0.7
    m = box_mesh(n, n, n)
    A, s = fvm.species_matrix(m, gamma=np.full(m.n_cells, g), gamma_b=np.full(m.b_cell.size, g),
                              Y_b=np.zeros(m.b_cell.size))
    h = 1.0 / n
    for P in range(m.n_cells):
        i, j, k = P % n, (P // n) % n, P // (n * n)
        nbrs = [(i + di, j + dj, k + dk) for di, dj, dk in
                ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]
        inside = [c for c in nbrs if all(0 <= x < n for x in c)]
        d = g * h * len(inside) + (2 * g * h if i in (0, n - 1) else 0.0) * (2 if n == 1 else 1)
        assert A[P, P] == pytest.approx(d, rel=1e-14)
        for (a, b, c) in inside:
            assert A[P, a + n * b + n * n * c] == pytest.approx(-g * h, rel=1e-14)
        assert np.count_nonzero(A[P]) == 1 + len(inside)


def test_linear_field_has_zero_laplacian_on_a_stretched_permuted_mesh():
    """psi = x with exact fixed values on the x sides and zero gradient elsewhere: the two-point
    fluxes are exact on an orthogonal mesh, so A psi = s to rounding."""
    m = box_mesh(5, 4, 3, seed=3, stretch=3.0, permute=True)
    g = np.full(m.n_cells, 1.3)
    psi = m.centre[:, 0]
    A, s = fvm.species_matrix(m, gamma=g, gamma_b=np.full(m.b_cell.size, 1.3), Y_b=m.b_centre[:, 0])
    assert np.max(np.abs(A @ psi - s)) <= 1e-12 * np.max(np.abs(s))


def test_closed_box_conserves_the_species_mass():
    """Zero-gradient walls and no boundary flux: every face flux (convective and diffusive)
    enters two rows with opposite signs, so 1^T A Y = sum rho V Y / dt for any Y and phi."""
    m = box_mesh(4, 3, 3, seed=4, stretch=2.0, permute=True)
    rng = np.random.default_rng(5)
    m.b_type[:] = 0
    nb = m.b_cell.size
    rho = rng.uniform(0.5, 2.0, m.n_cells)
    dt = 1e-3
    A, s = fvm.species_matrix(m, dt=dt, rho=rho, rho_old=rho, Y_old=np.zeros(m.n_cells),
                              phi=rng.standard_normal(m.owner.size), phi_b=np.zeros(nb),
                              gamma=rng.uniform(0.1, 1.0, m.n_cells), gamma_b=np.ones(nb), Y_b=np.zeros(nb))
    Y = rng.uniform(0.0, 1.0, m.n_cells)
    assert np.sum(A @ Y) == pytest.approx(np.sum(rho * m.volume * Y / dt), rel=1e-12)


def test_upwind_convection_of_a_uniform_field_through_a_uniform_flow():
    """A uniform flow along x through a box with inflow at x = 0 (boundary value c) and outflow
    at x = 1: the uniform field Y = c is steady (A Y = s without the time term).  c is not 1, so
    that an inflow face that convected the cell's value instead of the boundary value fails."""
    n = 4
    m = box_mesh(n, 3, 2, seed=6, stretch=2.0, permute=True)
    u = 2.5
    # face flux u |S| on x-normal faces, oriented owner -> neighbour
    d = m.centre[m.neighbour] - m.centre[m.owner]
    xface = np.abs(d[:, 0]) > 0
    phi = np.where(xface, u * m.mag_sf * np.sign(d[:, 0]), 0.0)
    out = m.b_centre[:, 0] > 1.0 - 1e-12
    inl = m.b_centre[:, 0] < 1e-12
    phi_b = np.where(out, u * m.b_mag_sf, np.where(inl, -u * m.b_mag_sf, 0.0))
    c = 0.37
    A, s = fvm.species_matrix(m, phi=phi, phi_b=phi_b, Y_b=np.full(m.b_cell.size, c))
    assert np.max(np.abs(A @ np.full(m.n_cells, c) - s)) <= 1e-13 * u
    assert np.all(A - np.diag(np.diag(A)) <= 0.0)         # upwind: non-positive off-diagonals


def test_ldu_round_trip_and_source_term():
    """lower_f = A[neighbour, owner] and upper_f = A[owner, neighbour] rebuild A; the round trip
    runs on a convective (unsymmetric) matrix so that exchanging lower and upper fails."""
    m = box_mesh(3, 3, 2, seed=7, permute=True)
    rng = np.random.default_rng(8)
    S = rng.standard_normal(m.n_cells)
    kap = rng.uniform(0.0, 1.0, m.n_cells)
    nb = m.b_cell.size
    A, s = fvm.species_matrix(m, gamma=np.ones(m.n_cells), gamma_b=np.ones(nb), Y_b=np.zeros(nb), S=S, kappa=kap,
                              phi=rng.standard_normal(m.owner.size), phi_b=np.zeros(nb))
    assert np.allclose(s, m.volume * kap * S, rtol=1e-15, atol=0)
    assert not np.array_equal(A, A.T)
    lo, up, dg = fvm.ldu(m, A)
    B = np.diag(dg)
    B[m.neighbour, m.owner] = lo
    B[m.owner, m.neighbour] = up
    assert np.array_equal(A, B)
    Ad, _ = fvm.species_matrix(m, gamma=np.ones(m.n_cells), gamma_b=np.ones(nb), Y_b=np.zeros(nb))
    lo, up, _ = fvm.ldu(m, Ad)
    assert np.array_equal(lo, up)                           # diffusion alone is symmetric


def test_linear_diffusivity_is_interpolated_exactly_to_the_faces():
    """Alg. 1 interpolates gamma linearly to each face: for gamma linear in space, sampled at the
    cell centres of a stretched mesh, the face value is gamma at the face itself, which lies half
    the owner's width (its volume over the face area) from the owner's centre."""
    m = box_mesh(6, 5, 4, seed=31, stretch=3.0, permute=True)
    lin = lambda x: 0.5 + 2.0 * x[..., 0] + 0.7 * x[..., 1] - 0.3 * x[..., 2]
    nb = m.b_cell.size
    A, _ = fvm.species_matrix(m, gamma=lin(m.centre), gamma_b=np.ones(nb), Y_b=np.zeros(nb))
    d = m.centre[m.neighbour] - m.centre[m.owner]
    ax = np.argmax(np.abs(d), axis=1)
    xf = m.centre[m.owner].copy()
    f = np.arange(ax.size)
    xf[f, ax] += np.sign(d[f, ax]) * 0.5 * m.volume[m.owner] / m.mag_sf
    want = -lin(xf) * m.mag_sf * m.delta
    assert np.allclose(A[m.owner, m.neighbour], want, rtol=1e-13, atol=0)
    assert np.allclose(A[m.neighbour, m.owner], want, rtol=1e-13, atol=0)
    assert np.max(np.abs(m.weight - 0.5)) > 0.1             # the mesh really is stretched


def test_time_term_alone_carries_each_cells_species_mass():
    """With the time derivative alone, A Y = s gives rho Y = rho_old Y_old in every cell."""
    m = box_mesh(4, 3, 2, seed=32, stretch=2.0, permute=True)
    rng = np.random.default_rng(33)
    rho, rho_old = rng.uniform(0.3, 1.5, m.n_cells), rng.uniform(0.3, 1.5, m.n_cells)
    Y_old = rng.uniform(0.0, 0.3, m.n_cells)
    A, s = fvm.species_matrix(m, dt=2e-4, rho=rho, rho_old=rho_old, Y_old=Y_old)
    Y = np.linalg.solve(A, s)
    assert np.allclose(rho * Y, rho_old * Y_old, rtol=1e-14, atol=0)


def test_open_box_species_budget():
    """Over the whole box, storage plus the net convective outflow through the boundary equals
    the source, whatever the flux field: sum V (rho Y - rho_old Y_old) / dt + sum_b phi_b Y_b' =
    sum V kappa S, where a boundary face carries its cell's value out (phi_b >= 0) and the boundary
    value in (phi_b < 0); internal faces, convective and diffusive, cancel.  Zero-gradient walls,
    so that no diffusive flux crosses the boundary."""
    m = box_mesh(5, 4, 3, seed=34, stretch=2.0, permute=True)
    rng = np.random.default_rng(35)
    m.b_type[:] = 0
    n, nf, nb = m.n_cells, m.owner.size, m.b_cell.size
    kw = dict(dt=1e-3, rho=rng.uniform(0.5, 2, n), rho_old=rng.uniform(0.5, 2, n), Y_old=rng.uniform(0, 1, n),
              phi=rng.standard_normal(nf), phi_b=rng.standard_normal(nb), gamma=rng.uniform(0.1, 1, n),
              gamma_b=np.ones(nb), Y_b=rng.uniform(0, 1, nb), S=rng.standard_normal(n), kappa=rng.uniform(0, 1, n))
    A, s = fvm.species_matrix(m, **kw)
    Y = np.linalg.solve(A, s)
    face = np.where(kw["phi_b"] >= 0.0, Y[m.b_cell], kw["Y_b"])
    terms = np.r_[m.volume * (kw["rho"] * Y - kw["rho_old"] * kw["Y_old"]) / kw["dt"], kw["phi_b"] * face,
                  -m.volume * kw["kappa"] * kw["S"]]
    assert abs(terms.sum()) <= 1e-11 * np.abs(terms).sum()


def test_pasr_limits():
    rho, mu, strain, delta = 1.2, 1.8e-4, 500.0, 1e-3
    nu = (0.17 * delta) ** 2 * strain
    tmix = 1.0 * np.sqrt((mu + rho * nu) / (rho * nu * strain ** 2))
    k = fvm.pasr_kappa(np.array([tmix, 1e-30, 1e30]), np.full(3, rho), np.full(3, mu), np.full(3, strain),
                       np.full(3, delta), 0.17, 1.0)
    assert k[0] == pytest.approx(0.5, rel=1e-14)
    assert k[1] < 1e-20 and k[2] == pytest.approx(1.0, rel=1e-12)
    assert fvm.pasr_kappa(np.array([1e-4]), np.array([rho]), np.array([mu]), np.array([0.0]),
                          np.array([delta]), 0.17, 1.0)[0] == 1.0


def test_row_form_matches_the_dense_matrix():
    m = box_mesh(4, 3, 3, seed=9, stretch=2.0, permute=True)
    rng = np.random.default_rng(10)
    nb = m.b_cell.size
    kw = dict(dt=1e-3, rho=rng.uniform(0.5, 2, m.n_cells), rho_old=rng.uniform(0.5, 2, m.n_cells),
              Y_old=rng.uniform(0, 1, m.n_cells), phi=rng.standard_normal(m.owner.size),
              phi_b=rng.standard_normal(nb), gamma=rng.uniform(0.1, 1, m.n_cells), gamma_b=rng.uniform(0.1, 1, nb),
              Y_b=rng.uniform(0, 1, nb), S=rng.standard_normal(m.n_cells), kappa=rng.uniform(0, 1, m.n_cells))
    A, s = fvm.species_matrix(m, **kw)
    rows = fvm.species_rows(m, range(m.n_cells), **kw)
    for P, (row, sp) in rows.items():
        dense = np.zeros(m.n_cells)
        for c, v in row.items():
            dense[c] = v
        assert np.allclose(dense, A[P], rtol=1e-13, atol=1e-300) and sp == pytest.approx(s[P], rel=1e-13)


@pytest.mark.parametrize("shape,permute", [((5, 4, 3), True), ((1, 1, 1), False), ((8, 1, 1), True)])
def test_mesh_generator_geometry(shape, permute):
    """Face counts, owner < neighbour in upper-triangular order, interpolation weights in (0, 1)
    that reproduce the face position, volumes and boundary areas of the unit box."""
    nx, ny, nz = shape
    m = box_mesh(nx, ny, nz, seed=21, stretch=3.0, permute=permute)
    n = nx * ny * nz
    assert m.n_cells == n
    assert m.owner.size == (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert m.b_cell.size == 2 * (ny * nz + nx * nz + nx * ny)
    assert np.all(m.owner < m.neighbour)
    assert np.all(np.diff(m.owner) >= 0)
    assert np.all((m.weight > 0.0) & (m.weight < 1.0))
    assert m.volume.sum() == pytest.approx(1.0, rel=1e-13)
    assert m.b_mag_sf.sum() == pytest.approx(6.0, rel=1e-13)
    d = m.centre[m.neighbour] - m.centre[m.owner]
    assert np.allclose(1.0 / np.linalg.norm(d, axis=1), m.delta, rtol=1e-13)
    # w x_owner + (1 - w) x_neighbour lies on the face between them (along the connecting axis)
    xf = m.weight[:, None] * m.centre[m.owner] + (1.0 - m.weight[:, None]) * m.centre[m.neighbour]
    ax = np.argmax(np.abs(d), axis=1)
    lo = np.minimum(m.centre[m.owner, ax], m.centre[m.neighbour, ax])
    hi = np.maximum(m.centre[m.owner, ax], m.centre[m.neighbour, ax])
    assert np.all((xf[np.arange(ax.size), ax] > lo) & (xf[np.arange(ax.size), ax] < hi))
