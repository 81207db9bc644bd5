"""Oracle: plain FP64 CPU reference of the chemistry hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA path.

* ``chem_oracle.cpp``: NASA-7 thermo, rates, reactor RHS, analytic Jacobian, complex-step
  Jacobian, Rodas4 integrator, RK4 brute force, operation counters (C++, built here).
* ``equilibrium.py``: independent HP Gibbs minimisation (element potentials).
* ``mlp.py``: FP64 MLP forward/backward with BF16 rounding emulation.
* ``surrogate.py``: Box-Cox transforms, element projection, T-from-h Newton, heat release.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libchem_oracle.so")
_lib = None

OK, MAX_STEPS, H_UNDERFLOW, NONFINITE, SINGULAR_LU = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (plain -O2, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "chem_oracle.cpp")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "chem_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, src])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = declare(ctypes.CDLL(_LIB_PATH))
    return _lib


def declare(L):
    """Set the argument and result types of the oracle's C functions on a loaded library."""
    P = ctypes.c_void_p
    d = ctypes.c_double
    i = ctypes.c_int
    i64 = ctypes.c_int64
    L.or_mech_new.restype = P
    L.or_mech_new.argtypes = [i, i, i] + [P] * 13
    L.or_mech_free.argtypes = [P]
    L.or_species_thermo.argtypes = [P, d, P, P, P, P]
    L.or_rates.argtypes = [P, d, d, P, P, P, P, P]
    L.or_rhs.argtypes = [P, d, P, P]
    L.or_rhs_complex.argtypes = [P, d, P, P, P, P]
    L.or_jacobian.argtypes = [P, d, P, P]
    L.or_jacobian_complex_step.argtypes = [P, d, P, P]
    L.or_rodas4.argtypes = [P, d, P, d, d, d, i, P, P]
    L.or_rodas4.restype = i
    L.or_advance.argtypes = [P, i64, P, P, P, i64, d, d, d, P, P, i]
    L.or_advance_dt.argtypes = [P, i64, P, P, P, i64, P, d, d, P, i]
    L.or_rk4.argtypes = [P, d, P, d, i64]
    L.or_rodas4_tableau.argtypes = [P, P, P, P, P]
    L.or_rodas4_linear.argtypes = [i, P, P, d, i, P]
    L.or_count_ops.argtypes = [P, d, P, d, d, d, P, P, P]
    L.or_count_ops.restype = i
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleMech:
    """Oracle-side copy of a synthetic mechanism (synth.mechanism.Mechanism)."""

    RU = 8.314462618e7
    PATM = 1.01325e6

    def __init__(self, mech):
        self.mech = mech
        self.ns, self.nr, self.ne = mech.ns, mech.nr, mech.ne
        self.N = self.ns + 1
        self._keep = [np.ascontiguousarray(a, dtype=t) for a, t in (
            (mech.elem_mass, np.float64), (mech.comp, np.int32), (mech.nasa_lo, np.float64),
            (mech.nasa_hi, np.float64), (mech.rtype, np.int32), (mech.reac, np.int32),
            (mech.prod, np.int32), (mech.A, np.float64), (mech.b, np.float64),
            (mech.Ea, np.float64), (mech.troe, np.float64), (mech.has_t2, np.int32),
            (mech.eff, np.float64))]
        self.h = lib().or_mech_new(self.ns, self.ne, self.nr, *[_p(a) for a in self._keep])
        self.W = np.asarray(mech.comp, np.float64) @ np.asarray(mech.elem_mass, np.float64)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_mech_free(self.h)
            self.h = None

    # -- thermo and kinetics ------------------------------------------------------------
    def thermo(self, T):
        cp, h, s, d = (np.zeros(self.ns) for _ in range(4))
        lib().or_species_thermo(self.h, float(T), _p(cp), _p(h), _p(s), _p(d))
        return cp, h, s, d

    def rates(self, T, p, Y):
        Y = np.ascontiguousarray(Y, np.float64)
        w = np.zeros(self.ns); q, kf, kr = (np.zeros(self.nr) for _ in range(3))
        lib().or_rates(self.h, float(T), float(p), _p(Y), _p(w), _p(q), _p(kf), _p(kr))
        return w, q, kf, kr

    def rhs(self, p, y):
        y = np.ascontiguousarray(y, np.float64)
        f = np.zeros(self.N)
        lib().or_rhs(self.h, float(p), _p(y), _p(f))
        return f

    def rhs_complex(self, p, y):
        y = np.asarray(y, np.complex128)
        yr = np.ascontiguousarray(y.real); yi = np.ascontiguousarray(y.imag)
        fr = np.zeros(self.N); fi = np.zeros(self.N)
        lib().or_rhs_complex(self.h, float(p), _p(yr), _p(yi), _p(fr), _p(fi))
        return fr + 1j * fi

    def jacobian(self, p, y):
        y = np.ascontiguousarray(y, np.float64)
        J = np.zeros((self.N, self.N))
        lib().or_jacobian(self.h, float(p), _p(y), _p(J))
        return J

    def jacobian_complex_step(self, p, y):
        y = np.ascontiguousarray(y, np.float64)
        J = np.zeros((self.N, self.N))
        lib().or_jacobian_complex_step(self.h, float(p), _p(y), _p(J))
        return J

    # -- integration ----------------------------------------------------------------------
    def rodas4(self, p, y, dt, rtol=1e-6, atol=1e-10, max_steps=100000):
        y = np.array(y, np.float64)
        nsub = ctypes.c_int(0); nrej = ctypes.c_int(0)
        st = lib().or_rodas4(self.h, float(p), _p(y), float(dt), float(rtol), float(atol),
                             int(max_steps), ctypes.byref(nsub), ctypes.byref(nrej))
        return y, st, nsub.value, nrej.value

    def advance(self, T, p, Y, dt, rtol=1e-6, atol=1e-10, nthreads=0):
        """Batch advance; T [n], p [n], Y [ns, n] (copies are returned)."""
        T = np.array(T, np.float64)
        p = np.ascontiguousarray(p, np.float64)
        Y = np.array(Y, np.float64, order="C")
        n = T.shape[0]
        st = np.zeros(n, np.int8); nsub = np.zeros(n, np.int32)
        lib().or_advance(self.h, n, _p(T), _p(p), _p(Y), n, float(dt), float(rtol), float(atol),
                         _p(st), _p(nsub), int(nthreads))
        return T, Y, st, nsub

    def advance_dt(self, T, p, Y, dt, rtol=1e-6, atol=1e-10, nthreads=0):
        """Batch advance with a per-cell step length dt [n]."""
        T = np.array(T, np.float64)
        p = np.ascontiguousarray(p, np.float64)
        Y = np.array(Y, np.float64, order="C")
        dt = np.ascontiguousarray(dt, np.float64)
        n = T.shape[0]
        st = np.zeros(n, np.int8)
        lib().or_advance_dt(self.h, n, _p(T), _p(p), _p(Y), n, _p(dt), float(rtol), float(atol),
                            _p(st), int(nthreads))
        return T, Y, st

    def rk4(self, p, y, dt, nsteps):
        y = np.array(y, np.float64)
        lib().or_rk4(self.h, float(p), _p(y), float(dt), int(nsteps))
        return y

    def count_ops(self, p, y, dt, rtol=1e-6, atol=1e-10):
        y = np.ascontiguousarray(y, np.float64)
        c = np.zeros(8)
        nsub = ctypes.c_int(0); nrej = ctypes.c_int(0)
        st = lib().or_count_ops(self.h, float(p), _p(y), float(dt), float(rtol), float(atol), _p(c),
                                ctypes.byref(nsub), ctypes.byref(nrej))
        keys = ["add", "mul", "div", "exp", "log", "pow", "sqrt", "cmp"]
        return dict(zip(keys, c.tolist())), st, nsub.value, nrej.value

    # -- derived quantities -----------------------------------------------------------------
    def density(self, T, p, Y):
        return p / (self.RU * T * np.sum(np.asarray(Y) / self.W))

    def enthalpy_mass(self, T, Y):
        """Mixture specific enthalpy (erg/g): sum_k Y_k h_k / W_k, h_k molar incl. formation."""
        _, h_RT, _, _ = self.thermo(T)
        return float(np.sum(np.asarray(Y) * self.RU * T * h_RT / self.W))

    def cp_mass(self, T, Y):
        cp_R, _, _, _ = self.thermo(T)
        return float(np.sum(np.asarray(Y) * self.RU * cp_R / self.W))


def rodas4_tableau():
    g = np.zeros(1); A = np.zeros((6, 6)); C = np.zeros((6, 6)); M = np.zeros(6); E = np.zeros(6)
    lib().or_rodas4_tableau(_p(g), _p(A), _p(C), _p(M), _p(E))
    return float(g[0]), A, C, M, E


def rodas4_linear(L, y0, h, nsteps):
    L = np.ascontiguousarray(L, np.float64)
    y = np.array(y0, np.float64)
    err = np.zeros_like(y)
    lib().or_rodas4_linear(L.shape[0], _p(L), _p(y), float(h), int(nsteps), _p(err))
    return y, err
