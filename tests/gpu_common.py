"""Helpers for the GPU parity tests (CUDA path vs the oracle on the same seeded inputs)."""
import os

import numpy as np
import torch

T_RTOL = 1e-6          # relative tolerance on T
Y_RTOL = 1e-6          # times max_k Y_k, plus Y_ATOL
Y_ATOL = 1e-12


def to_dev(T, p, Y):
    d = torch.device("cuda:0")
    return (torch.tensor(T, dtype=torch.float64, device=d),
            torch.tensor(p, dtype=torch.float64, device=d),
            torch.tensor(np.ascontiguousarray(Y), dtype=torch.float64, device=d))


def within(T_ref, Y_ref, T_got, Y_got):
    """Per-cell boolean mask of the contract tolerance."""
    okT = np.abs(T_got - T_ref) <= T_RTOL * np.abs(T_ref)
    scale = Y_RTOL * np.max(np.abs(Y_ref), axis=0) + Y_ATOL
    okY = np.all(np.abs(Y_got - Y_ref) <= scale[None, :], axis=0)
    return okT & okY


def cell_error(T_ref, Y_ref, T_got, Y_got):
    """max(|dT| / (rtol T), |dY| / (rtol max Y + atol)) per cell: <= 1 means within tolerance."""
    eT = np.abs(T_got - T_ref) / (T_RTOL * np.abs(T_ref))
    scale = Y_RTOL * np.max(np.abs(Y_ref), axis=0) + Y_ATOL
    eY = np.max(np.abs(Y_got - Y_ref) / scale[None, :], axis=0)
    return np.maximum(eT, eY)


# (test, cells compared, cells outside the contract tolerance that the tight-oracle re-check
# accepted): printed at the end of the session by tests/conftest.py
BIFURCATIONS = []


def assert_parity(om, T0, p, Y0, T_gpu, Y_gpu, dt, rtol, atol, max_bifurcations=None):
    """Compare GPU results with the same-tolerance oracle.  Cells outside the tolerance are
    re-checked against a tight oracle run (rtol 1e-12): they pass if the GPU's distance to the
    tight answer is no larger than the oracle's own distance plus the tolerance (an accept /
    reject decision flipped by rounding near err = 1).  Such bifurcations are counted, recorded
    for the session summary and bounded: at most max(2, 0.5 % of the cells) unless the caller
    gives its own bound.  Returns their number."""
    T_or, Y_or, st, _ = om.advance(T0, p, Y0, dt, rtol, atol)
    assert np.all(st == 0)
    ok = within(T_or, Y_or, T_gpu, Y_gpu)
    bad = np.nonzero(~ok)[0]
    if bad.size:
        Tt, Yt, st2, _ = om.advance(T0[bad], p[bad], Y0[:, bad], dt, 1e-12, 1e-18)
        e_gpu = cell_error(Tt, Yt, T_gpu[bad], Y_gpu[:, bad])
        e_or = cell_error(Tt, Yt, T_or[bad], Y_or[:, bad])
        still = e_gpu > e_or + 1.0
        assert not np.any(still), (
            f"{int(still.sum())} cells outside tolerance even against the tight oracle; "
            f"worst gpu/oracle error {e_gpu.max():.3g}/{e_or.max():.3g}")
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    BIFURCATIONS.append((test, int(T0.size), int(bad.size)))
    cap = max(2, int(0.005 * T0.size)) if max_bifurcations is None else max_bifurcations
    assert bad.size <= cap, f"{bad.size} bifurcated cells of {T0.size} (at most {cap} expected)"
    return int(bad.size)
