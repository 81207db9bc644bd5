"""Seeded synthetic finite-volume meshes in face-addressed form (input generation only).

The paper's solver stores its mesh the OpenFOAM way (§3.1, Fig. 2): cells, internal faces with an
owner and a neighbour cell (owner < neighbour), boundary faces in patches, and per face the
interpolation weight, the inverse centre-to-centre distance ("delta coefficient") and the face
area.  The paper's meshes (the 128^3 Taylor-Green box, the burner's unstructured grid) are not
available; this module builds a stretched, optionally permuted hexahedral box in that form:

* nodes x_i = cumulative sums of seeded spacings (varying by up to a factor `stretch`),
  likewise in y and z, scaled to the unit box; cell centres midway between nodes;
* an internal face between cells P and N: |S| = its area, delta = 1 / |x_N - x_P| along the
  face normal, owner weight w = (x_N - x_f) / (x_N - x_P) (linear interpolation to the face);
* a boundary face: |S|, delta = 1 / |x_f - x_P|; its patch type is fixed-value on the x = 0 and
  x = L sides and zero-gradient elsewhere (callers may change it);
* cell and face numbering: natural (x fastest) or a seeded permutation, so that the assembly
  sees unstructured addressing; internal faces are sorted by owner then neighbour, as in the
  paper's ldu (upper-triangular order) convention.

Only geometry is computed here; no term of any equation.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    n_cells: int
    owner: np.ndarray          # [nf] int32, owner < neighbour
    neighbour: np.ndarray      # [nf] int32
    weight: np.ndarray         # [nf] owner interpolation weight
    delta: np.ndarray          # [nf] 1 / centre distance
    mag_sf: np.ndarray         # [nf] face area
    b_cell: np.ndarray         # [nb] int32 cell of each boundary face
    b_type: np.ndarray         # [nb] int8: 0 zero-gradient, 1 fixed-value
    b_delta: np.ndarray        # [nb] 1 / (face - cell centre) distance
    b_mag_sf: np.ndarray       # [nb]
    volume: np.ndarray         # [n_cells]
    centre: np.ndarray         # [n_cells, 3] cell centres (for tests)
    b_centre: np.ndarray       # [nb, 3] boundary face centres


def _nodes(n, rng, stretch):
    h = np.exp(rng.uniform(-np.log(stretch) / 2, np.log(stretch) / 2, n))
    x = np.concatenate([[0.0], np.cumsum(h)])
    return x / x[-1]                                 # unit box


def box_mesh(nx, ny, nz, seed=0, stretch=1.0, permute=False):
    rng = np.random.default_rng(seed)
    xs = [_nodes(m, rng, stretch) for m in (nx, ny, nz)]
    cs = [0.5 * (x[1:] + x[:-1]) for x in xs]
    hs = [np.diff(x) for x in xs]
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)          # natural numbering, x fastest
    perm = rng.permutation(n) if permute else np.arange(n)
    cid = perm[idx]                                  # cell number of grid cell (k, j, i)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    centre = np.empty((n, 3))
    centre[cid.ravel(), 0] = cs[0][I.ravel()]
    centre[cid.ravel(), 1] = cs[1][J.ravel()]
    centre[cid.ravel(), 2] = cs[2][K.ravel()]
    volume = np.empty(n)
    volume[cid.ravel()] = (hs[0][I] * hs[1][J] * hs[2][K]).ravel()
    own, nei, w, dlt, area = [], [], [], [], []
    bc, bt, bd, ba, bx = [], [], [], [], []
    for ax in range(3):
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        grid_ax = 2 - ax                           # arrays are [k, j, i]
        sl_lo[grid_ax] = slice(0, -1)
        sl_hi[grid_ax] = slice(1, None)
        a = cid[tuple(sl_lo)].ravel()
        b = cid[tuple(sl_hi)].ravel()
        # face positions along the axis and areas
        G = [K, J, I]
        pos = [g[tuple(sl_lo)].ravel() for g in G]   # grid indices of the lower cell
        i_ax = pos[grid_ax]
        xf = xs[ax][i_ax + 1]
        xp, xn = cs[ax][i_ax], cs[ax][i_ax + 1]
        other = [d for d in range(3) if d != ax]
        ar = hs[other[0]][pos[2 - other[0]]] * hs[other[1]][pos[2 - other[1]]]
        wf = (xn - xf) / (xn - xp)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        # the owner is the lower-numbered cell; its weight is the one of its own side
        w_own = np.where(a < b, wf, 1.0 - wf)
        own.append(lo); nei.append(hi); w.append(w_own); dlt.append(1.0 / (xn - xp)); area.append(ar)
        for side in (0, 1):
            slb = [slice(None)] * 3
            slb[grid_ax] = 0 if side == 0 else -1
            cells = cid[tuple(slb)].ravel()
            gp = [g[tuple(slb)].ravel() for g in G]
            ia = gp[grid_ax]
            xfb = xs[ax][0] if side == 0 else xs[ax][-1]
            d = np.abs(cs[ax][ia] - xfb)
            arb = hs[other[0]][gp[2 - other[0]]] * hs[other[1]][gp[2 - other[1]]]
            bc.append(cells); bd.append(1.0 / d); ba.append(arb)
            bt.append(np.full(cells.size, 1 if ax == 0 else 0, np.int8))
            fc = np.empty((cells.size, 3))
            for dd in range(3):
                fc[:, dd] = centre[cells, dd]
            fc[:, ax] = xfb
            bx.append(fc)
    owner = np.concatenate(own).astype(np.int32)
    neighbour = np.concatenate(nei).astype(np.int32)
    order = np.lexsort((neighbour, owner))
    return Mesh(n_cells=n, owner=owner[order], neighbour=neighbour[order],
                weight=np.concatenate(w)[order], delta=np.concatenate(dlt)[order],
                mag_sf=np.concatenate(area)[order], b_cell=np.concatenate(bc).astype(np.int32),
                b_type=np.concatenate(bt), b_delta=np.concatenate(bd), b_mag_sf=np.concatenate(ba),
                volume=volume, centre=centre, b_centre=np.concatenate(bx))
