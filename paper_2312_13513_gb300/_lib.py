"""ctypes binding of libchem.so: argument marshalling only.

Every computation runs in the CUDA kernels behind the C ABI (include/chem.h).  There is no CPU
fallback: importing this module fails loudly if the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
D = ctypes.c_double

CHEM_OK = 0
CHEM_WCELLS = 1
CHEM_EINVAL = -1
CHEM_ENOMEM = -2
CHEM_ECUDA = -3
CHEM_EBUSY = -4
CHEM_ETIMEOUT = -5
CHEM_ENOTFOUND = -6

CELL_OK, CELL_MAX_STEPS, CELL_H_UNDERFLOW, CELL_NONFINITE, CELL_SINGULAR_LU = 0, 1, 2, 3, 4


class ChemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libchem error {code}: {msg}")
        self.code = code


class MechDesc(ctypes.Structure):
    _fields_ = [("n_species", I32), ("n_elements", I32), ("n_reactions", I32),
                ("elem_mass", P), ("comp", P), ("nasa_lo", P), ("nasa_hi", P), ("rtype", P),
                ("reac", P), ("prod", P), ("A", P), ("b", P), ("Ea", P), ("troe", P),
                ("has_t2", P), ("eff", P)]


class Options(ctypes.Structure):
    _fields_ = [("max_steps", I32), ("group_threads", I32), ("groups_per_cta", I32),
                ("max_ctas", I32)]


class Segment(ctypes.Structure):
    _fields_ = [("T", P), ("p", P), ("Y", P), ("ld", I64), ("ncells", I64), ("idx", P),
                ("status", P), ("nsub", P), ("nrej", P), ("dt", D), ("rtol", D), ("atol", D)]


class TransportDesc(ctypes.Structure):
    _fields_ = [("n_species", I32), ("mu_poly", P), ("lambda_poly", P), ("diff_poly", P)]


class ServeOptions(ctypes.Structure):
    _fields_ = [("n_streams", I32), ("idle_poll_us", D), ("slice_ms", D), ("max_pause_ms", D)]


class SurrogateDesc(ctypes.Structure):
    _fields_ = [("n_species", I32), ("hidden", I32), ("dt", D), ("W", P * 5), ("b", P * 5),
                ("x_mean", P), ("x_std", P), ("y_mean", P), ("y_std", P), ("box_lo", P),
                ("box_hi", P)]


class FvMeshDesc(ctypes.Structure):
    _fields_ = [("n_cells", I64), ("n_faces", I64), ("n_bfaces", I64), ("owner", P), ("neighbour", P),
                ("weight", P), ("delta", P), ("mag_sf", P), ("b_cell", P), ("b_type", P), ("b_delta", P),
                ("b_mag_sf", P), ("volume", P)]


class FvmTerms(ctypes.Structure):
    _fields_ = [("dt", D), ("rho", P), ("rho_old", P), ("Y_old", P), ("phi", P), ("phi_b", P),
                ("gamma", P), ("gamma_b", P), ("Y_b", P), ("S", P), ("kappa", P)]


class StepDesc(ctypes.Structure):
    _fields_ = [("mech", P), ("model", P), ("transport", P), ("T", P), ("p", P), ("Y", P), ("ld", I64),
                ("ncells", I64), ("dt", D), ("rtol", D), ("atol", D), ("h0", P), ("cp0", P), ("q", P),
                ("route", P), ("status", P), ("nsub", P), ("thermo_status", P), ("mu", P), ("lam", P),
                ("Dmix", P)]


class SurrogatePsDesc(ctypes.Structure):
    _fields_ = [("n_species", I32), ("hidden", I32 * 3), ("dt", D), ("W", (P * 4) * 16),
                ("b", (P * 4) * 16), ("x_mean", P), ("x_std", P), ("y_mean", P), ("y_std", P),
                ("box_lo", P), ("box_hi", P)]


# name -> (restype, argtypes); the library must export every one of them
SIGNATURES = {
    "chem_load_mechanism": (ctypes.c_int, [ctypes.c_char_p, P]),
    "chem_load_mechanism_desc": (ctypes.c_int, [P, P]),
    "chem_free_mechanism": (ctypes.c_int, [P]),
    "chem_mechanism_info": (ctypes.c_int, [P, P, P, P]),
    "chem_advance": (ctypes.c_int, [P, P, P, P, D, I64, D, D, P]),
    "chem_advance_ex": (ctypes.c_int, [P, P, P, P, I64, D, I64, D, D, P, P, P, P, P, P]),
    "chem_advance_noalloc": (ctypes.c_int, [P, P, P, P, I64, D, I64, D, D, P, P, P, P]),
    "chem_eval_rhs_jac": (ctypes.c_int, [P, P, P, P, I64, I64, P, P, P]),
    "chem_fp64_fma_peak": (ctypes.c_int, [P]),
    "chem_fast_exp": (ctypes.c_int, [P, P, I64, P]),
    "chem_mixture_thermo": (ctypes.c_int, [P, P, P, I64, I64, P, P, P]),
    "chem_temperature_from_enthalpy": (ctypes.c_int, [P, P, P, I64, I64, P, P, P]),
    "chem_transport_create": (ctypes.c_int, [P, P, P]),
    "chem_transport_free": (ctypes.c_int, [P]),
    "chem_transport_eval": (ctypes.c_int, [P, P, P, P, I64, I64, P, P, P, P]),
    "chem_surrogate_create": (ctypes.c_int, [P, P, P]),
    "chem_surrogate_load": (ctypes.c_int, [ctypes.c_char_p, P, P]),
    "chem_surrogate_create_per_species": (ctypes.c_int, [P, P, P]),
    "chem_surrogate_free": (ctypes.c_int, [P]),
    "chem_surrogate_forward": (ctypes.c_int, [P, P, P, P, I64, I64, P, P, P, P]),
    "chem_surrogate_advance": (ctypes.c_int, [P, P, P, P, P, I64, D, I64, D, D, P, P]),
    "chem_mlp_trainer_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P,
                                               ctypes.c_uint64, P]),
    "chem_mlp_trainer_create_layers": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                                      ctypes.c_int, P, P, ctypes.c_uint64, P]),
    "chem_mlp_trainer_free": (ctypes.c_int, [P]),
    "chem_mlp_forward": (ctypes.c_int, [P, P, P, P]),
    "chem_mlp_backward": (ctypes.c_int, [P, P, P, P]),
    "chem_mlp_adam_step": (ctypes.c_int, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_float, P]),
    "chem_mlp_adam_step_dev": (ctypes.c_int, [P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, P]),
    "chem_mlp_trainer_get": (ctypes.c_int, [P, ctypes.c_int, P, P]),
    "chem_mlp_grad_count": (ctypes.c_int, [P, P]),
    "chem_mlp_grad_pack": (ctypes.c_int, [P, P, P]),
    "chem_mlp_grad_unpack": (ctypes.c_int, [P, P, ctypes.c_float, P]),
    "chem_mlp_trainer_save": (ctypes.c_int, [P, ctypes.c_char_p]),
    "chem_mlp_trainer_load": (ctypes.c_int, [P, ctypes.c_char_p]),
    "chem_mlp_trainer_step": (ctypes.c_int, [P, P]),
    "chem_train_features": (ctypes.c_int, [P, P, P, P, I64, I64, ctypes.c_int, P, P, P]),
    "chem_column_stats": (ctypes.c_int, [P, I64, ctypes.c_int, P, P]),
    "chem_train_normalize": (ctypes.c_int, [P, I64, ctypes.c_int, P, P, P, ctypes.c_int, P,
                                            ctypes.c_int, P, P, P, P]),
    "chem_heat_release": (ctypes.c_int, [P, P, P, P, P, I64, I64, D, P, P]),
    "chem_advance_batch": (ctypes.c_int, [P, P, ctypes.c_int, P]),
    "chem_surrogate_advance_batch": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
    "chem_serve_create": (ctypes.c_int, [ctypes.c_size_t, P, P]),
    "chem_serve_register_state": (ctypes.c_int, [P, P, P, P, P, P, I64, I64, P]),
    "chem_serve_submit": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, D, D, D, P]),
    "chem_serve_poll": (ctypes.c_int, [P, ctypes.c_uint64, P, P]),
    "chem_serve_wait": (ctypes.c_int, [P, ctypes.c_uint64, D]),
    "chem_serve_stats": (ctypes.c_int, [P, P]),
    "chem_serve_destroy": (ctypes.c_int, [P]),
    "chem_gemm_bf16": (ctypes.c_int, [P, I64, P, I64, P, I64, P, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, P, P]),
    "chem_gemm_bf16_act": (ctypes.c_int, [P, I64, P, I64, P, I64, P, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, P, P]),
    "chem_fvmesh_create": (ctypes.c_int, [P, P]),
    "chem_fvmesh_free": (ctypes.c_int, [P]),
    "chem_fvmesh_csr": (ctypes.c_int, [P, P, P, P]),
    "chem_fvm_assemble": (ctypes.c_int, [P, P, P, P, P, P, P]),
    "chem_fvm_to_csr": (ctypes.c_int, [P, P, P, P, P, P]),
    "chem_pasr_kappa": (ctypes.c_int, [I64, P, P, P, P, P, D, D, P, P]),
    "chem_step_create": (ctypes.c_int, [P, P]),
    "chem_step_run": (ctypes.c_int, [P, ctypes.c_int, P]),
    "chem_step_stage_ms": (ctypes.c_int, [P, P]),
    "chem_step_free": (ctypes.c_int, [P]),
    "chem_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load (building first if needed) libchem.so.  Raises if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libchem.so missing at {path}")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(rc):
    if rc < 0:
        msg = load().chem_last_error()
        raise ChemError(rc, msg.decode() if msg else "")
    return rc
