"""GB300-native per-cell chemistry: FP64 Rodas4 integrator, BF16 MLP surrogate, serving loop.

Python entry points mirror the C ABI in include/chem.h one to one; they only marshal torch
tensors (device memory and streams) into pointers.  All arithmetic runs in libchem.so.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (CELL_H_UNDERFLOW, CELL_MAX_STEPS, CELL_NONFINITE, CELL_OK,  # noqa: F401
                   CELL_SINGULAR_LU, ChemError, check)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require(t, dtype, name):
    import torch
    if t is None:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Mechanism:
    """A mechanism uploaded to the current device (chem_load_mechanism[_desc])."""

    def __init__(self, mech=None, path=None):
        L = _lib.load()
        h = ctypes.c_void_p()
        if path is not None:
            check(L.chem_load_mechanism(path.encode(), ctypes.byref(h)))
        else:
            self._keep = [np.ascontiguousarray(a, dtype=t) for a, t in (
                (mech.elem_mass, np.float64), (mech.comp, np.int32), (mech.nasa_lo, np.float64),
                (mech.nasa_hi, np.float64), (mech.rtype, np.int32), (mech.reac, np.int32),
                (mech.prod, np.int32), (mech.A, np.float64), (mech.b, np.float64),
                (mech.Ea, np.float64), (mech.troe, np.float64), (mech.has_t2, np.int32),
                (mech.eff, np.float64))]
            d = _lib.MechDesc(mech.ns, mech.ne, mech.nr,
                              *[a.ctypes.data_as(ctypes.c_void_p) for a in self._keep])
            check(L.chem_load_mechanism_desc(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        ns, nr, ne = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(L.chem_mechanism_info(h, ctypes.byref(ns), ctypes.byref(nr), ctypes.byref(ne)))
        self.ns, self.nr, self.ne = ns.value, nr.value, ne.value

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().chem_free_mechanism(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def options(max_steps=0, group_threads=0, groups_per_cta=0, max_ctas=0):
    return _lib.Options(max_steps, group_threads, groups_per_cta, max_ctas)


def advance(mech, T, p, Y, dt, rtol=1e-6, atol=1e-10, idx=None, status=None, nsub=None,
            nrej=None, opts=None, stream=None, ncells=None):
    """chem_advance_ex: advance cells in place.  Y is [ns, ld] (species-major)."""
    import torch
    _require(T, torch.float64, "T"); _require(p, torch.float64, "p"); _require(Y, torch.float64, "Y")
    _require(idx, torch.int32, "idx"); _require(status, torch.int8, "status")
    _require(nsub, torch.int32, "nsub"); _require(nrej, torch.int32, "nrej")
    ld = Y.shape[1]
    if ncells is None:
        ncells = idx.numel() if idx is not None else T.numel()
    return check(_lib.load().chem_advance_ex(
        mech.handle, _ptr(T), _ptr(p), _ptr(Y), ld, float(dt), int(ncells), float(rtol),
        float(atol), _ptr(idx), _ptr(status), _ptr(nsub), _ptr(nrej),
        ctypes.byref(opts) if opts is not None else None, _stream_ptr(stream)))


def advance_simple(mech, T, p, Y, dt, rtol=1e-6, atol=1e-10, stream=None):
    """chem_advance: ld = ncells = T.numel()."""
    import torch
    _require(T, torch.float64, "T"); _require(p, torch.float64, "p"); _require(Y, torch.float64, "Y")
    return check(_lib.load().chem_advance(mech.handle, _ptr(T), _ptr(p), _ptr(Y), float(dt),
                                          T.numel(), float(rtol), float(atol), _stream_ptr(stream)))


def eval_rhs_jac(mech, T, p, Y, with_jacobian=True, stream=None):
    """chem_eval_rhs_jac: returns f [N, n] and J [N*N, n] (or None)."""
    import torch
    n = T.numel()
    N = mech.ns + 1
    f = torch.empty((N, n), dtype=torch.float64, device=T.device)
    J = torch.empty((N * N, n), dtype=torch.float64, device=T.device) if with_jacobian else None
    check(_lib.load().chem_eval_rhs_jac(mech.handle, _ptr(T), _ptr(p), _ptr(Y), Y.shape[1], n,
                                        _ptr(f), _ptr(J), _stream_ptr(stream)))
    return f, J


# ---------------------------------------------------------------------------------------------
# thermophysical and transport properties
# ---------------------------------------------------------------------------------------------
def mixture_thermo(mech, T, Y, h=None, cp=None, stream=None):
    """chem_mixture_thermo: mixture h (erg/g) and cp (erg/(g K)) per cell."""
    import torch
    _require(T, torch.float64, "T"); _require(Y, torch.float64, "Y")
    _require(h, torch.float64, "h"); _require(cp, torch.float64, "cp")
    check(_lib.load().chem_mixture_thermo(mech.handle, _ptr(T), _ptr(Y), Y.shape[1], T.numel(), _ptr(h), _ptr(cp),
                                          _stream_ptr(stream)))


def temperature_from_enthalpy(mech, h, Y, T, status=None, stream=None):
    """chem_temperature_from_enthalpy: Newton on h(T, Y) = h from the guess in T (in place)."""
    import torch
    _require(h, torch.float64, "h"); _require(Y, torch.float64, "Y"); _require(T, torch.float64, "T")
    _require(status, torch.int8, "status")
    check(_lib.load().chem_temperature_from_enthalpy(mech.handle, _ptr(h), _ptr(Y), Y.shape[1], T.numel(), _ptr(T),
                                                     _ptr(status), _stream_ptr(stream)))


class Step:
    """chem_step_*: one "chemistry + thermo" step (start-state thermo, chemistry, heat release and
    T from h, transport) over the caller's device arrays, direct or as a replayed CUDA graph."""

    def __init__(self, mech, T, p, Y, dt, rtol=1e-6, atol=1e-10, model=None, transport=None, h0=None,
                 cp0=None, q=None, route=None, status=None, nsub=None, thermo_status=None, mu=None,
                 lam=None, D=None):
        import torch
        for a, nm in ((T, "T"), (p, "p"), (Y, "Y"), (h0, "h0"), (cp0, "cp0"), (q, "q"), (mu, "mu"),
                      (lam, "lambda"), (D, "D")):
            _require(a, torch.float64, nm)
        _require(route, torch.int8, "route"); _require(status, torch.int8, "status")
        _require(nsub, torch.int32, "nsub"); _require(thermo_status, torch.int8, "thermo_status")
        self.mech, self.model, self.transport = mech, model, transport
        # the graph replays on these pointers: keep the tensors alive with the step
        self._keep = (T, p, Y, h0, cp0, q, route, status, nsub, thermo_status, mu, lam, D)
        d = _lib.StepDesc(mech.handle, model.handle if model is not None else None,
                          transport.handle if transport is not None else None, _ptr(T), _ptr(p), _ptr(Y),
                          Y.shape[1], T.numel(), float(dt), float(rtol), float(atol), _ptr(h0), _ptr(cp0),
                          _ptr(q), _ptr(route), _ptr(status), _ptr(nsub), _ptr(thermo_status), _ptr(mu),
                          _ptr(lam), _ptr(D))
        h = ctypes.c_void_p()
        check(_lib.load().chem_step_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def run(self, graph=False, stream=None):
        check(_lib.load().chem_step_run(self.handle, 1 if graph else 0, _stream_ptr(stream)))

    def stage_ms(self):
        """Device ms of (start-state thermo, chemistry, heat release + T from h, transport) of the
        last direct run."""
        ms = (ctypes.c_float * 4)()
        check(_lib.load().chem_step_stage_ms(self.handle, ms))
        return list(ms)

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().chem_step_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Transport:
    """chem_transport_*: mixture-averaged transport properties from fitted pure-species data."""

    def __init__(self, mech, data):
        self.mech = mech
        self._arrays = [np.ascontiguousarray(a, np.float64) for a in (data.mu_poly, data.lambda_poly, data.diff_poly)]
        d = _lib.TransportDesc(int(data.mu_poly.shape[0]), *[a.ctypes.data for a in self._arrays])
        h = ctypes.c_void_p()
        check(_lib.load().chem_transport_create(mech.handle, ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def __call__(self, T, p, Y, mu=None, lam=None, D=None, stream=None):
        import torch
        for a, nm in ((T, "T"), (p, "p"), (Y, "Y"), (mu, "mu"), (lam, "lambda"), (D, "D")):
            _require(a, torch.float64, nm)
        check(_lib.load().chem_transport_eval(self.handle, _ptr(T), _ptr(p), _ptr(Y), Y.shape[1], T.numel(), _ptr(mu),
                                              _ptr(lam), _ptr(D), _stream_ptr(stream)))

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().chem_transport_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FvMesh:
    """chem_fvmesh_*: a face-addressed finite-volume mesh on the device (fields of a
    synth.mesh.Mesh-like object: owner, neighbour, weight, delta, mag_sf, b_cell, b_type,
    b_delta, b_mag_sf, volume, n_cells)."""

    def __init__(self, mesh):
        import torch
        keep = [np.ascontiguousarray(mesh.owner, np.int32), np.ascontiguousarray(mesh.neighbour, np.int32),
                np.ascontiguousarray(mesh.weight, np.float64), np.ascontiguousarray(mesh.delta, np.float64),
                np.ascontiguousarray(mesh.mag_sf, np.float64), np.ascontiguousarray(mesh.b_cell, np.int32),
                np.ascontiguousarray(mesh.b_type, np.int8), np.ascontiguousarray(mesh.b_delta, np.float64),
                np.ascontiguousarray(mesh.b_mag_sf, np.float64), np.ascontiguousarray(mesh.volume, np.float64)]
        d = _lib.FvMeshDesc(int(mesh.n_cells), keep[0].size, keep[5].size,
                            *[a.ctypes.data_as(ctypes.c_void_p) for a in keep])
        h = ctypes.c_void_p()
        check(_lib.load().chem_fvmesh_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.n_cells, self.n_faces, self.n_bfaces = int(mesh.n_cells), keep[0].size, keep[5].size
        nnz = ctypes.c_int64()
        rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
        check(_lib.load().chem_fvmesh_csr(h, ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)))
        self.nnz = nnz.value

    def assemble(self, dt=0.0, rho=None, rho_old=None, Y_old=None, phi=None, phi_b=None, gamma=None,
                 gamma_b=None, Y_b=None, S=None, kappa=None, stream=None):
        """chem_fvm_assemble: returns (lower, upper, diag, source) device tensors."""
        import torch
        for a, nm in ((rho, "rho"), (rho_old, "rho_old"), (Y_old, "Y_old"), (phi, "phi"), (phi_b, "phi_b"),
                      (gamma, "gamma"), (gamma_b, "gamma_b"), (Y_b, "Y_b"), (S, "S"), (kappa, "kappa")):
            _require(a, torch.float64, nm)
        t = _lib.FvmTerms(float(dt), *[_ptr(a) for a in (rho, rho_old, Y_old, phi, phi_b, gamma, gamma_b, Y_b,
                                                          S, kappa)])
        dev = torch.device("cuda")
        lower = torch.empty(self.n_faces, dtype=torch.float64, device=dev)
        upper = torch.empty_like(lower)
        diag = torch.empty(self.n_cells, dtype=torch.float64, device=dev)
        source = torch.empty_like(diag)
        check(_lib.load().chem_fvm_assemble(self.handle, ctypes.byref(t), _ptr(lower), _ptr(upper), _ptr(diag),
                                            _ptr(source), _stream_ptr(stream)))
        return lower, upper, diag, source

    def to_csr(self, lower, upper, diag, stream=None):
        """chem_fvm_to_csr: CSR values [nnz] on the mesh's pattern."""
        import torch
        vals = torch.empty(self.nnz, dtype=torch.float64, device=diag.device)
        check(_lib.load().chem_fvm_to_csr(self.handle, _ptr(lower), _ptr(upper), _ptr(diag), _ptr(vals),
                                          _stream_ptr(stream)))
        return vals

    def csr_pattern(self):
        """(row_ptr, col_idx) of the mesh's CSR pattern, copied to host numpy arrays."""
        import torch
        nnz = ctypes.c_int64()
        rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
        check(_lib.load().chem_fvmesh_csr(self.handle, ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)))
        row_ptr = torch.as_tensor(_DeviceArray(rp.value, self.n_cells + 1, "<i4"), device="cuda")
        col = torch.as_tensor(_DeviceArray(ci.value, nnz.value, "<i4"), device="cuda")
        return row_ptr.cpu().numpy(), col.cpu().numpy()

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().chem_fvmesh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A library-owned device array exposed through __cuda_array_interface__ (to be copied, not written)."""

    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def pasr_kappa(tau_c, rho, mu, strain, delta, c_s=0.17, c_mix=1.0, kappa=None, stream=None):
    """chem_pasr_kappa: PaSR factor per cell (device tensors)."""
    import torch
    for a, nm in ((tau_c, "tau_c"), (rho, "rho"), (mu, "mu"), (strain, "strain"), (delta, "delta")):
        _require(a, torch.float64, nm)
    if kappa is None:
        kappa = torch.empty_like(tau_c)
    check(_lib.load().chem_pasr_kappa(tau_c.numel(), _ptr(tau_c), _ptr(rho), _ptr(mu), _ptr(strain), _ptr(delta),
                                      float(c_s), float(c_mix), _ptr(kappa), _stream_ptr(stream)))
    return kappa


def fast_exp(x, y, stream=None):
    """chem_fast_exp: y = exp(x) elementwise with the integrator's table-driven exponential."""
    import torch
    _require(x, torch.float64, "x"); _require(y, torch.float64, "y")
    if x.numel() != y.numel() or not x.is_contiguous() or not y.is_contiguous():
        raise ValueError("x and y must be contiguous and of the same size")
    check(_lib.load().chem_fast_exp(_ptr(x), _ptr(y), x.numel(), _stream_ptr(stream)))


def fp64_fma_peak():
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s."""
    v = ctypes.c_double()
    check(_lib.load().chem_fp64_fma_peak(ctypes.byref(v)))
    return v.value


# ---------------------------------------------------------------------------------------------
# surrogate
# ---------------------------------------------------------------------------------------------
SUR_FIELDS = ("W", "b", "x_mean", "x_std", "y_mean", "y_std", "box_lo", "box_hi")


class Surrogate:
    """A BF16 MLP surrogate bound to a mechanism (chem_surrogate_create / _load).

    params: dict with W (5 FP32 arrays [out, in]), b (5 arrays), x_mean, x_std, y_mean, y_std,
    box_lo, box_hi, dt; or, for the per-species variant (chem_surrogate_create_per_species),
    hidden = [h1, h2, h3] and nets = {species k: {"W": 4 arrays, "b": 4 arrays}} instead of W, b.
    """

    def __init__(self, mech, params=None, path=None):
        L = _lib.load()
        h = ctypes.c_void_p()
        if path is not None:
            check(L.chem_surrogate_load(path.encode(), mech.handle, ctypes.byref(h)))
        else:
            keep = []

            def arr(a):
                a = np.ascontiguousarray(a, dtype=np.float32)
                keep.append(a)
                return a.ctypes.data_as(ctypes.c_void_p)

            if "nets" in params:
                d = _lib.SurrogatePsDesc()
                d.n_species = mech.ns
                for i in range(3):
                    d.hidden[i] = int(params["hidden"][i])
                d.dt = float(params["dt"])
                for k, net in params["nets"].items():
                    for l in range(4):
                        d.W[int(k)][l] = arr(net["W"][l])
                        d.b[int(k)][l] = arr(net["b"][l])
            else:
                d = _lib.SurrogateDesc()
                d.n_species = mech.ns
                d.hidden = int(np.asarray(params["W"][0]).shape[0])
                d.dt = float(params["dt"])
                for l in range(5):
                    d.W[l] = arr(params["W"][l])
                    d.b[l] = arr(params["b"][l])
            d.x_mean = arr(params["x_mean"]); d.x_std = arr(params["x_std"])
            d.y_mean = arr(params["y_mean"]); d.y_std = arr(params["y_std"])
            d.box_lo = arr(params["box_lo"]); d.box_hi = arr(params["box_hi"])
            create = L.chem_surrogate_create_per_species if "nets" in params else L.chem_surrogate_create
            check(create(ctypes.byref(d), mech.handle, ctypes.byref(h)))
        self.handle = h
        self.mech = mech

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().chem_surrogate_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def surrogate_forward(model, T, p, Y, with_z=False, stream=None):
    """chem_surrogate_forward: returns (ynet [ns, n] FP32, z [ns, n] or None, out_of_box [n])."""
    import torch
    n = T.numel()
    ns = model.mech.ns
    ynet = torch.empty((ns, n), dtype=torch.float32, device=T.device)
    z = torch.empty((ns, n), dtype=torch.float32, device=T.device) if with_z else None
    box = torch.empty(n, dtype=torch.uint8, device=T.device)
    check(_lib.load().chem_surrogate_forward(model.handle, _ptr(T), _ptr(p), _ptr(Y), Y.shape[1], n,
                                             _ptr(ynet), _ptr(z), _ptr(box), _stream_ptr(stream)))
    return ynet, z, box


def surrogate_advance(model, T, p, Y, dt, rtol=1e-6, atol=1e-10, route=None, stream=None):
    """chem_surrogate_advance: network step with FP64 fallback, in place."""
    import torch
    _require(T, torch.float64, "T"); _require(p, torch.float64, "p"); _require(Y, torch.float64, "Y")
    _require(route, torch.int8, "route")
    return check(_lib.load().chem_surrogate_advance(
        model.handle, model.mech.handle, _ptr(T), _ptr(p), _ptr(Y), Y.shape[1], float(dt), T.numel(),
        float(rtol), float(atol), _ptr(route), _stream_ptr(stream)))


def gemm_bf16(A, B, bias=None, err=None, stream=None):
    """chem_gemm_bf16: C = A @ B.T (+ bias) with A [M, K], B [N, K] BF16 (K contiguous), FP32 C."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    own_err = err is None
    if own_err:
        err = torch.zeros(1, dtype=torch.int32, device=A.device)
    check(_lib.load().chem_gemm_bf16(_ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C), C.stride(0),
                                     _ptr(bias), M, N, K, _ptr(err), _stream_ptr(stream)))
    if own_err:
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        if int(err.item()) != 0:
            raise ChemError(-3, "gemm pipeline wait timed out")
    return C


def gemm_bf16_act(A, B, bias=None, gelu=True, err=None, stream=None):
    """chem_gemm_bf16_act: C = bf16(GELU(A @ B.T + bias)) (or without GELU), BF16 [M, N]."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.bfloat16, device=A.device)
    own_err = err is None
    if own_err:
        err = torch.zeros(1, dtype=torch.int32, device=A.device)
    check(_lib.load().chem_gemm_bf16_act(_ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C), C.stride(0),
                                         _ptr(bias), 1 if gelu else 0, M, N, K, _ptr(err), _stream_ptr(stream)))
    if own_err:
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        if int(err.item()) != 0:
            raise ChemError(-3, "gemm pipeline wait timed out")
    return C


def heat_release(mech, T0, p, Y0, Y1, dt, stream=None):
    """chem_heat_release: q [n] (erg/cm^3/s) of a step from (T0, p, Y0) to Y1."""
    import torch
    n = T0.numel()
    q = torch.empty(n, dtype=torch.float64, device=T0.device)
    check(_lib.load().chem_heat_release(mech.handle, _ptr(T0), _ptr(p), _ptr(Y0), _ptr(Y1), Y0.shape[1], n,
                                        float(dt), _ptr(q), _stream_ptr(stream)))
    return q
