"""ctypes declarations of the C ABI in include/pf_gb300.h (argument marshalling only).

Loading fails loudly when libpf_gb300.so has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_D = ctypes.c_double
_I = ctypes.c_int
_VP = ctypes.c_void_p

PF_OK, PF_E_INVAL, PF_E_OOM, PF_E_NOCONV, PF_E_BREAKDOWN, PF_E_GAMMA, PF_E_CUDA, PF_E_TIMEOUT, PF_PENDING = range(9)
STATUS_NAMES = ["PF_OK", "PF_E_INVAL", "PF_E_OOM", "PF_E_NOCONV", "PF_E_BREAKDOWN", "PF_E_GAMMA", "PF_E_CUDA",
                "PF_E_TIMEOUT", "PF_PENDING"]
PF_FP64, PF_MIXED = 0, 1
PF_BICGSTAB, PF_CG_SYMMETRIC, PF_CG_ALL = 0, 1, 2
PF_OP_POISSON, PF_OP_PF1, PF_OP_PF2 = 0, 1, 2
PF_MEM_HOST, PF_MEM_DEVICE = 0, 1
PF_NORM_REL2, PF_NORM_ABSINF = 0, 1
PF_MAX_SPECIES = 8
PF_FERMI_NOALLOC_MAX_NODES = 1 << 20
PF_CHARGES_SPREAD, PF_CHARGES_DECOMPOSED = 0, 1


class pf_species(ctypes.Structure):
    _fields_ = [("z", _I), ("radius_A", _D), ("bulk_M", _D)]


class pf_coeffs(ctypes.Structure):
    _fields_ = [("eps", _VP), ("solvent", _VP), ("n_charges", _I), ("charges", _VP), ("phi_zlo_V", _D),
                ("phi_zhi_V", _D), ("n_species", _I), ("species", ctypes.POINTER(pf_species)), ("eps_s", _D),
                ("lc_A", _D), ("T_K", _D)]


class pf_solve_opts(ctypes.Structure):
    _fields_ = [("max_iter", _I), ("tol", _D), ("norm", _I), ("precision", _I), ("inner_tol", _D),
                ("max_refine", _I), ("method", _I)]


class pf_report(ctypes.Structure):
    _fields_ = [("status", _I), ("iterations", _I), ("refinements", _I), ("residual", _D), ("time_ms", _D)]


class pf_nl_opts(ctypes.Structure):
    _fields_ = [("omega", _D), ("tol_outer", _D), ("max_outer", _I), ("lin", pf_solve_opts), ("accel_depth", _I),
                ("lin_forcing", _D), ("warm_start", _I), ("predict", _I)]


class pf_result(ctypes.Structure):
    _fields_ = [("phi_V", _VP), ("C_M", _VP), ("S", _VP), ("Gamma", _VP), ("Psi", _VP), ("mem", _I), ("status", _I),
                ("outer_iters", _I), ("lin_iters_total", _I), ("lin_iters_first", _I), ("delta", _D),
                ("time_ms", _D)]


PF_PROF_KINDS = 18
PROF_NAMES = ["init", "b_fp64", "ca_fp64", "b_fp32", "ca_fp32", "b_fp64_pf1", "ca_fp64_pf1", "b_fp32_pf1",
              "ca_fp32_pf1", "residual_fp64", "fermi", "other", "cg_direction", "cg_update", "cg_fp64", "cg_fp32",
              "cg_fp64_pf1", "cg_fp32_pf1"]


class pf_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("count", ctypes.c_longlong * PF_PROF_KINDS),
                ("ms", _D * PF_PROF_KINDS)]


class pf_request(ctypes.Structure):
    _fields_ = [("nx", _I), ("ny", _I), ("nz", _I), ("h_A", _D), ("origin_A", _D * 3), ("coeffs", pf_coeffs),
                ("opts", pf_nl_opts), ("phi0_V", _VP)]


class pf_sites(ctypes.Structure):
    _fields_ = [("n_sites", _I), ("center_A", _VP), ("radius_A", _VP), ("q_ion", _VP), ("occupied", _VP),
                ("ion_radius_A", _VP), ("eps_b", _D), ("eps_p", _D), ("map_radius_A", _D), ("v_sites_A3", _D)]


class pf_batch_stats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_longlong), ("wall_ms", _D), ("device_ms", _D)]


PF_BATCH_TUNE_MAX = 16


class pf_batch_tune(ctypes.Structure):
    _fields_ = [("n", _I), ("tiles_per_block", _I * PF_BATCH_TUNE_MAX), ("z_planes", _I * PF_BATCH_TUNE_MAX),
                ("ms", ctypes.c_float * PF_BATCH_TUNE_MAX), ("chosen", _I), ("chosen_z", _I)]


# names declared in include/pf_gb300.h, with their ctypes signatures
SIGNATURES = {
    "pf_default_solve_opts": (None, [ctypes.POINTER(pf_solve_opts)]),
    "pf_default_nl_opts": (None, [ctypes.POINTER(pf_nl_opts)]),
    "pf_create_grid": (_I, [_I, _I, _I, _D, ctypes.POINTER(_D), _VP, ctypes.POINTER(_VP)]),
    "pf_grid_bytes": (ctypes.c_size_t, [_I, _I, _I, _I]),
    "pf_set_coeffs": (_I, [_VP, ctypes.POINTER(pf_coeffs)]),
    "pf_set_kappa": (_I, [_VP, _VP, _I]),
    "pf_set_potential": (_I, [_VP, _VP, _I]),
    "pf_linear_solve": (_I, [_VP, _I, _VP, _VP, _I, ctypes.POINTER(pf_solve_opts), ctypes.POINTER(pf_report)]),
    "pf_linear_solve_cg": (_I, [_VP, _I, _VP, _VP, _I, ctypes.POINTER(pf_solve_opts), ctypes.POINTER(pf_report)]),
    "pf_set_filter": (_I, [_VP, _VP, _VP, _I]),
    "pf_set_filter_sites": (_I, [_VP, ctypes.POINTER(pf_sites), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "pf_set_charge_mode": (_I, [_VP, _I, ctypes.POINTER(pf_report)]),
    "pf_get_decomposition": (_I, [_VP, _VP, _VP, _I]),
    "pf_nonlinear_solve": (_I, [_VP, ctypes.POINTER(pf_nl_opts), ctypes.POINTER(pf_result)]),
    "pf_destroy_grid": (_I, [_VP]),
    "pf_profile_enable": (_I, [_VP, _I]),
    "pf_profile_get": (_I, [_VP, ctypes.POINTER(pf_profile)]),
    "pf_last_error": (ctypes.c_char_p, []),
    "pf_selftest_wait_timeout": (_I, [ctypes.c_ulonglong, _VP]),
    "pf_fermi_noalloc": (_I, [ctypes.c_long, _VP, _VP, _I, ctypes.POINTER(pf_species), _D, _I, _VP, _VP, _VP, _VP]),
    "pf_batch_create": (_I, [ctypes.POINTER(_VP), _I, _VP, ctypes.POINTER(_VP)]),
    "pf_batch_get_stats": (_I, [_VP, ctypes.POINTER(pf_batch_stats)]),
    "pf_batch_set_tiles_per_block": (_I, [_VP, _I]),
    "pf_batch_set_tiling": (_I, [_VP, _I, _I]),
    "pf_batch_autotune": (_I, [_VP, ctypes.POINTER(pf_batch_tune)]),
    "pf_batch_get_tune": (_I, [_VP, ctypes.POINTER(pf_batch_tune)]),
    "pf_batch_nonlinear_solve": (_I, [_VP, ctypes.POINTER(pf_nl_opts), ctypes.POINTER(pf_result)]),
    "pf_batch_destroy": (_I, [_VP]),
    "pf_server_create": (_I, [ctypes.c_size_t, _I, ctypes.POINTER(_VP)]),
    "pf_submit": (_I, [_VP, ctypes.POINTER(pf_request), ctypes.POINTER(ctypes.c_uint64)]),
    "pf_poll": (_I, [_VP, ctypes.c_uint64, ctypes.POINTER(pf_result), ctypes.POINTER(_I)]),
    "pf_server_destroy": (_I, [_VP]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libpf_gb300.so; raises if it is missing (build() compiles it)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libpf_gb300.so is not built ({path}); run paper_1711_04060_gb300.build.build() "
                           "(or __graft_entry__.build()) first")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    return load().pf_last_error().decode()
