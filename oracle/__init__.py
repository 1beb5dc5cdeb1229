"""ctypes wrapper of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It builds ``oracle.c`` on first use and
exposes it with numpy arrays.  It imports nothing from the CUDA library; the
detector description it consumes comes from the input module
``paper_2203_14354_gb300.geometry`` (mesh and tables, no tracking arithmetic).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")

DETECTED, QE_FAIL, BULK_ABS, SURF_ABS, ESCAPED, TRUNCATED, GEOM_ERR = range(7)
N_FIXED = 8


class _Source(C.Structure):
    _fields_ = [("src", C.POINTER(C.c_double)), ("explicit_pos", C.c_void_p),
                ("explicit_dir", C.c_void_p), ("explicit_pol", C.c_void_p)]


class _Results(C.Structure):
    _fields_ = [("lce", C.c_void_p), ("det", C.c_void_p), ("hist", C.c_void_p), ("fates", C.c_void_p),
                ("ph_fate", C.c_void_p), ("ph_detail", C.c_void_p), ("ph_steps", C.c_void_p),
                ("ph_time", C.c_void_p), ("adjoint", C.c_void_p), ("ph_state", C.c_void_p)]


def lib():
    """The oracle library: built from oracle.c, or the prebuilt library named
    by the ORACLE_LIB environment variable (the mutation tests load copies
    of oracle.c with one planted mistake this way)."""
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        L.orc_scene_new.restype = C.c_void_p
        L.orc_scene_new.argtypes = [f32p, C.c_uint32, u32p, C.c_uint32, u8p, u8p, u16p, i32p]
        L.orc_scene_free.argtypes = [C.c_void_p]
        L.orc_set_materials.argtypes = [C.c_void_p, f64p, C.c_int]
        L.orc_set_surfaces.argtypes = [C.c_void_p, i32p, f64p, C.c_int]
        L.orc_set_channels.argtypes = [C.c_void_p, C.c_int]
        L.orc_trace.argtypes = [C.c_void_p, C.c_uint64, f32p, f32p, C.c_void_p, C.c_void_p, u32p, f32p, C.c_int]
        L.orc_sample_source.argtypes = [C.c_void_p, C.POINTER(_Source), C.c_uint64, C.c_uint64, C.c_uint64,
                                        f64p, f64p, f64p, i32p, f64p, f64p]
        L.orc_propagate.restype = C.c_int
        L.orc_propagate.argtypes = [C.c_void_p, C.POINTER(_Source), C.c_uint64, C.c_uint64, C.c_uint64,
                                    C.c_uint32, C.c_double, C.c_uint32, C.POINTER(_Results), C.c_int]
        L.orc_set_adjoint.restype = C.c_int
        L.orc_set_adjoint.argtypes = [C.c_void_p, i32p, C.c_int, i32p, C.c_int]
        L.orc_jacobian.argtypes = [C.c_void_p, f64p, f64p]
        L.orc_philox.argtypes = [u32p, u32p, u32p]
        L.orc_uniform.restype = C.c_double
        L.orc_uniform.argtypes = [C.c_uint32]
        L.orc_fresnel.argtypes = [C.c_double, C.c_double, C.c_double, f64p]
        L.orc_dielectric.restype = C.c_int
        L.orc_dielectric.argtypes = [f64p, f64p, f64p, C.c_double, C.c_double, C.c_double, f64p, f64p,
                                     C.POINTER(C.c_double)]
        L.orc_mirror.argtypes = [f64p, f64p, f64p, f64p, f64p]
        L.orc_rayleigh.argtypes = [f64p, f64p, C.c_uint64, C.c_uint32, C.c_uint64, f64p, f64p]
        L.orc_lambert.argtypes = [f64p, C.c_uint64, C.c_uint32, C.c_uint64, f64p, f64p]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def source_array(src) -> np.ndarray:
    return np.array([src.kind, src.medium, src.n_sides, src.radius, src.phase, src.z_min, src.z_max,
                     *src.center, *src.p1, src.t0, src.singlet_frac, src.tau_singlet_ns, src.tau_triplet_ns,
                     src.wl_mean_nm, src.wl_fwhm_nm],
                    np.float64)


class Oracle:
    """Scene built from a ``geometry.Detector``."""

    def __init__(self, det):
        L = lib()
        self.det = det
        self.n_mat = len(det.materials)
        self.n_surf = len(det.surfaces)
        self.n_chan = max(1, det.n_pmts)
        self._s = L.orc_scene_new(np.ascontiguousarray(det.verts, np.float32), det.verts.shape[0],
                                  np.ascontiguousarray(det.tris, np.uint32), det.n_tris,
                                  np.ascontiguousarray(det.mat_inner), np.ascontiguousarray(det.mat_outer),
                                  np.ascontiguousarray(det.surface), np.ascontiguousarray(det.channel))
        if not self._s:
            raise ValueError("oracle rejected the mesh")
        m = np.array([[x.n, x.abs_len_mm, x.rayleigh_len_mm, x.dn_dlambda_per_nm, x.rayleigh_exp]
                      for x in det.materials], np.float64).ravel()
        assert L.orc_set_materials(self._s, m, self.n_mat) == 0
        if self.n_surf:
            t = np.array([x.type for x in det.surfaces], np.int32)
            p = np.array([[x.reflectivity, x.spec_frac, x.qe, x.transparency, x.wire_reflectivity,
                           x.wire_spec_frac] for x in det.surfaces], np.float64).ravel()
            assert L.orc_set_surfaces(self._s, t, p, self.n_surf) == 0
        L.orc_set_channels(self._s, self.n_chan)
        self.adj_mats, self.adj_surfs = [], []

    def set_adjoint(self, mats=(), surfs=()):
        """Track (L_abs, L_ray) of materials `mats` and R or T of surfaces `surfs`."""
        m = np.ascontiguousarray(list(mats) or [0], np.int32)
        sf = np.ascontiguousarray(list(surfs) or [0], np.int32)
        if lib().orc_set_adjoint(self._s, m, len(mats), sf, len(surfs)) != 0:
            raise ValueError("bad adjoint spec")
        self.adj_mats, self.adj_surfs = list(mats), list(surfs)

    @property
    def n_tallies(self):
        return 2 * len(self.adj_mats) + 2 * len(self.adj_surfs)

    @property
    def n_params(self):
        return 2 * len(self.adj_mats) + len(self.adj_surfs)

    def jacobian(self, sums):
        sums = np.ascontiguousarray(sums, np.float64).reshape(self.n_chan, self.n_tallies)
        J = np.zeros((self.n_chan, self.n_params))
        lib().orc_jacobian(self._s, sums, J)
        return J

    def __del__(self):
        if getattr(self, "_s", None) and _lib is not None:
            _lib.orc_scene_free(self._s)
            self._s = None

    def trace(self, org, dir, skip=None, tmax=None, brute=False):
        org = np.ascontiguousarray(org, np.float32).reshape(-1, 3)
        dir = np.ascontiguousarray(dir, np.float32).reshape(-1, 3)
        n = org.shape[0]
        hit = np.empty(n, np.uint32)
        t = np.empty(n, np.float32)
        sk = None if skip is None else np.ascontiguousarray(skip, np.uint32)
        tm = None if tmax is None else np.ascontiguousarray(tmax, np.float32)
        lib().orc_trace(self._s, n, org, dir, _ptr(sk), _ptr(tm), hit, t, int(brute))
        return hit, t

    def _source(self, src, explicit=None):
        arr = source_array(src)
        s = _Source()
        s.src = arr.ctypes.data_as(C.POINTER(C.c_double))
        keep = [arr]
        if explicit is not None:
            pos, dir, pol = (np.ascontiguousarray(x, np.float32).reshape(-1, 3) for x in explicit)
            keep += [pos, dir, pol]
            s.explicit_pos, s.explicit_dir, s.explicit_pol = _ptr(pos), _ptr(dir), _ptr(pol)
        return s, keep

    def sample_source(self, n, base=0, seed=0, src=None, explicit=None, time=False, wavelength=False):
        """First photon states: pos, dir, pol [n, 3], medium [n]; then the
        emission times [n] if time, and the wavelengths [n] (nm) if wavelength."""
        s, keep = self._source(src or self.det.source, explicit)
        pos = np.empty((n, 3)); dir = np.empty((n, 3)); pol = np.empty((n, 3))
        med = np.empty(n, np.int32)
        t = np.empty(n)
        wl = np.empty(n)
        lib().orc_sample_source(self._s, C.byref(s), n, base, seed, pos, dir, pol, med, t, wl)
        return (pos, dir, pol, med) + ((t,) if time else ()) + ((wl,) if wavelength else ())

    def propagate(self, n, base=0, seed=0, src=None, explicit=None, max_steps=10000, tbin_ns=1.0,
                  n_tbins=1000, per_photon=False, threads=None, adjoint=False):
        s, keep = self._source(src or self.det.source, explicit)
        P = self.n_chan
        out = dict(lce=np.zeros(P, np.uint64), det=np.zeros(P, np.uint64),
                   hist=np.zeros((P, n_tbins + 1), np.uint64),
                   fates=np.zeros(N_FIXED + self.n_mat + self.n_surf, np.uint64))
        if per_photon:
            out.update(fate=np.zeros(n, np.uint32), detail=np.zeros(n, np.int32),
                       steps=np.zeros(n, np.uint32), time=np.zeros(n, np.float32),
                       state=np.zeros((n, 9), np.float32))
        if adjoint:
            out["adjoint"] = np.zeros((P, self.n_tallies), np.float64)
        r = _Results()
        r.lce, r.det, r.hist, r.fates = _ptr(out["lce"]), _ptr(out["det"]), _ptr(out["hist"]), _ptr(out["fates"])
        if per_photon:
            r.ph_fate, r.ph_detail = _ptr(out["fate"]), _ptr(out["detail"])
            r.ph_steps, r.ph_time = _ptr(out["steps"]), _ptr(out["time"])
            r.ph_state = _ptr(out["state"])
        if adjoint:
            r.adjoint = _ptr(out["adjoint"])
        if threads is None:
            threads = os.cpu_count() or 1
        rc = lib().orc_propagate(self._s, C.byref(s), n, base, seed, max_steps, tbin_ns, n_tbins, C.byref(r),
                                 int(threads))
        if rc != 0:
            raise ValueError(f"orc_propagate failed ({rc})")
        out["threads"] = int(threads)
        return out


def philox(ctr, key):
    o = np.zeros(4, np.uint32)
    lib().orc_philox(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), o)
    return o


def uniform(x):
    return lib().orc_uniform(int(x))


def fresnel(n1, n2, cos_i):
    o = np.zeros(6)
    lib().orc_fresnel(n1, n2, cos_i, o)
    return dict(rs=o[0], rp=o[1], ts=o[2], tp=o[3], cos_t=o[4], tir=bool(o[5]))


def dielectric(k, eps, N, n1, n2, u):
    ko, eo = np.zeros(3), np.zeros(3)
    pr = C.c_double()
    refl = lib().orc_dielectric(np.asarray(k, float), np.asarray(eps, float), np.asarray(N, float), n1, n2, u,
                                ko, eo, C.byref(pr))
    return bool(refl), ko, eo, pr.value


def mirror(k, eps, N):
    ko, eo = np.zeros(3), np.zeros(3)
    lib().orc_mirror(np.asarray(k, float), np.asarray(eps, float), np.asarray(N, float), ko, eo)
    return ko, eo


def rayleigh(k, eps, pid, step=0, seed=0):
    ko, eo = np.zeros(3), np.zeros(3)
    lib().orc_rayleigh(np.asarray(k, float), np.asarray(eps, float), pid, step, seed, ko, eo)
    return ko, eo


def lambert(N, pid, step=0, seed=0):
    ko, eo = np.zeros(3), np.zeros(3)
    lib().orc_lambert(np.asarray(N, float), pid, step, seed, ko, eo)
    return ko, eo
