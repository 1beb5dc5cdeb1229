"""ctypes binding of include/lxo.h: the same names, argument marshalling only.

Loading builds the library if needed (``build.py``) and fails loudly if it
cannot be built or loaded; there is no fallback path."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

LXO_OK, LXO_ERR_ARG, LXO_ERR_CUDA, LXO_ERR_STATE, LXO_ERR_DEVICE, LXO_ERR_NOMEM = 0, -1, -2, -3, -4, -5
LXO_FATES_FIXED = 8
LXO_MAX_MATERIALS = 16
LXO_MAX_SURFACES = 48
LXO_SURF_NONE = 0xFFFF
LXO_NO_HIT = 0xFFFFFFFF
LXO_FLAG_STATS = 1
LXO_FLAG_ADJOINT = 2
LXO_STATIC_SCRATCH_BYTES = 8 << 20
LXO_REF_WAVELENGTH_NM = 175.0
LXO_MAX_TBINS = 1 << 24
LXO_STATS_LEN = 40
FATE_NAMES = ["detected", "qe_fail", "bulk_abs", "surf_abs", "escaped", "truncated", "geom_err"]


class lxo_material(C.Structure):
    _fields_ = [("n", C.c_float), ("abs_len_mm", C.c_float), ("rayleigh_len_mm", C.c_float),
                ("dn_dlambda_per_nm", C.c_float), ("rayleigh_exp", C.c_float)]


class lxo_surface(C.Structure):
    _fields_ = [("type", C.c_int32), ("reflectivity", C.c_float), ("spec_frac", C.c_float), ("qe", C.c_float),
                ("transparency", C.c_float), ("wire_reflectivity", C.c_float), ("wire_spec_frac", C.c_float)]


class lxo_pmt(C.Structure):
    _fields_ = [("channel", C.c_int32), ("array", C.c_int32), ("center", C.c_float * 3)]


class lxo_source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("medium", C.c_int32), ("n_sides", C.c_int32), ("reserved", C.c_int32),
                ("radius", C.c_float), ("phase", C.c_float), ("z_min", C.c_float), ("z_max", C.c_float),
                ("center", C.c_float * 3), ("p1", C.c_float * 3), ("t0", C.c_float),
                ("singlet_frac", C.c_float), ("tau_singlet_ns", C.c_float), ("tau_triplet_ns", C.c_float),
                ("wl_mean_nm", C.c_float), ("wl_fwhm_nm", C.c_float),
                ("pos", C.c_void_p), ("dir", C.c_void_p), ("pol", C.c_void_p)]


class lxo_event(C.Structure):
    _fields_ = [("kind", C.c_int32), ("medium", C.c_int32), ("center", C.c_float * 3), ("p1", C.c_float * 3),
                ("radius", C.c_float), ("t0", C.c_float), ("singlet_frac", C.c_float),
                ("tau_singlet_ns", C.c_float), ("tau_triplet_ns", C.c_float), ("wl_mean_nm", C.c_float),
                ("wl_fwhm_nm", C.c_float), ("reserved", C.c_float), ("n_photons", C.c_uint64)]


class lxo_run_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("max_steps", C.c_uint32), ("n_tbins", C.c_uint32), ("tbin_ns", C.c_float),
                ("flags", C.c_uint32)]


class lxo_results(C.Structure):
    _fields_ = [("lce", C.c_void_p), ("det", C.c_void_p), ("hist", C.c_void_p), ("fates", C.c_void_p),
                ("ph_fate", C.c_void_p), ("ph_detail", C.c_void_p), ("ph_steps", C.c_void_p),
                ("ph_time", C.c_void_p), ("adjoint", C.c_void_p), ("stats", C.c_void_p),
                ("ph_state", C.c_void_p)]


class lxo_bvh_info(C.Structure):
    _fields_ = [("n_tris", C.c_uint32), ("n_nodes", C.c_uint32), ("n_leaves", C.c_uint32), ("max_depth", C.c_uint32),
                ("node_bytes", C.c_uint64), ("tri_bytes", C.c_uint64), ("build_seconds", C.c_double),
                ("sah_cost", C.c_double)]


class lxo_bvh_params(C.Structure):
    _fields_ = [("leaf_size", C.c_uint32), ("sah_bins", C.c_uint32), ("n_threads", C.c_uint32),
                ("reserved", C.c_uint32)]


vp = C.c_void_p
_SIGNATURES = {
    "lxo_create": (C.c_int, [C.POINTER(vp), C.c_int]),
    "lxo_destroy": (None, [vp]),
    "lxo_last_error": (C.c_char_p, [vp]),
    "lxo_load_mesh": (C.c_int, [vp, vp, C.c_uint32, vp, C.c_uint32, vp, vp, vp, vp]),
    "lxo_set_materials": (C.c_int, [vp, C.POINTER(lxo_material), C.c_uint32]),
    "lxo_set_surfaces": (C.c_int, [vp, C.POINTER(lxo_surface), C.c_uint32]),
    "lxo_set_pmts": (C.c_int, [vp, C.POINTER(lxo_pmt), C.c_uint32]),
    "lxo_build_bvh": (C.c_int, [vp, C.POINTER(lxo_bvh_params), C.POINTER(lxo_bvh_info)]),
    "lxo_trace_rays": (C.c_int, [vp, vp, vp, vp, vp, C.c_uint32, vp, vp, vp]),
    "lxo_sample_source": (C.c_int, [vp, C.POINTER(lxo_source), C.c_uint64, C.c_uint64, C.c_uint64, vp, vp, vp, vp,
                                     vp, vp]),
    "lxo_propagate": (C.c_int, [vp, C.POINTER(lxo_source), C.c_uint64, C.c_uint64, C.POINTER(lxo_run_params),
                                C.POINTER(lxo_results), vp]),
    "lxo_propagate_host": (C.c_int, [vp, C.POINTER(lxo_source), C.c_uint64, C.c_uint64,
                                     C.POINTER(lxo_run_params), C.POINTER(lxo_results), vp]),
    "lxo_sync": (C.c_int, [vp, vp]),
    "lxo_set_adjoint": (C.c_int, [vp, vp, C.c_uint32, vp, C.c_uint32]),
    "lxo_upload_events": (C.c_int, [vp, vp, C.c_uint32, C.c_uint32]),
    "lxo_propagate_events": (C.c_int, [vp, C.POINTER(lxo_run_params), C.POINTER(lxo_results), vp]),
    "lxo_set_launch": (C.c_int, [vp, C.c_uint32, C.c_uint32, C.c_uint32]),
    "lxo_adjoint_jacobian": (C.c_int, [vp, vp, C.c_uint32, vp, vp, vp, vp]),
    "lxo_propagate_host_static": (C.c_int, [vp, C.POINTER(lxo_source), C.c_uint64, C.c_uint64,
                                            C.POINTER(lxo_run_params), C.POINTER(lxo_results), vp]),
}

_lib = None


def checked() -> bool:
    """LXO_CHECKED=1 in the environment selects the checked build (every
    kernel index compared with its array size; for debugging)."""
    return os.environ.get("LXO_CHECKED", "0") == "1"


def lib_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def lib():
    """The loaded library (built on first use)."""
    global _lib
    if _lib is None:
        path = _build.build(checked=True) if checked() else _build.build()
        L = C.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class LxoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lxo error {code}: {msg}")
        self.code = code


def check(code, ctx=None):
    if code != LXO_OK:
        msg = lib().lxo_last_error(ctx).decode() if ctx else ""
        raise LxoError(code, msg)
