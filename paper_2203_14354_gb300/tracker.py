"""Python front end of the photon tracker (the paper's user-level flow, Sec. 1
and 2.1: import the detector as a mesh, assign materials and surfaces,
generate photons, propagate on the GPU, read back per-PMT hits, arrival
times and loss bookkeeping).

Everything here is argument marshalling around the C ABI in
``include/lxo.h``; every step of the photon path runs in the CUDA library.
PyTorch provides device memory and streams.  There is no CPU fallback: the
constructor raises if CUDA or the library is unavailable."""
from __future__ import annotations

import ctypes as C
from dataclasses import replace

import numpy as np
import torch

from . import _capi as A
from .geometry import REFLECTOR, Detector, Source, SRC_EXPLICIT


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def make_source(src: Source, explicit=None) -> A.lxo_source:
    s = A.lxo_source()
    s.kind, s.medium, s.n_sides = int(src.kind), int(src.medium), int(src.n_sides)
    s.radius, s.phase, s.z_min, s.z_max = float(src.radius), float(src.phase), float(src.z_min), float(src.z_max)
    s.center[:] = [float(x) for x in src.center]
    s.p1[:] = [float(x) for x in src.p1]
    s.t0 = float(src.t0)
    s.singlet_frac, s.tau_singlet_ns, s.tau_triplet_ns = (float(src.singlet_frac), float(src.tau_singlet_ns),
                                                          float(src.tau_triplet_ns))
    s.wl_mean_nm, s.wl_fwhm_nm = float(src.wl_mean_nm), float(src.wl_fwhm_nm)
    if explicit is not None:
        pos, dir, pol = explicit
        s.pos, s.dir, s.pol = pos.data_ptr(), dir.data_ptr(), pol.data_ptr()
    return s


def own_tables(det: Detector) -> Detector:
    """A copy of det that shares its mesh arrays but holds its own material
    and surface records, so that changing the tracker's parameters
    (set_theta) never writes into the caller's detector."""
    return replace(det, materials=[replace(m) for m in det.materials],
                   surfaces=[replace(s) for s in det.surfaces])


class Tracker:
    """A detector loaded on one GPU with its BVH built.  The tracker keeps
    its own copy of the detector's material and surface tables (self.det)."""

    def __init__(self, det: Detector, device: int = 0, leaf_size: int = 0, sah_bins: int = 0, n_threads: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("the photon tracker needs a CUDA GPU; no CPU fallback exists")
        L = A.lib()
        self.det = own_tables(det)
        self.device = torch.device("cuda", device)
        ctx = C.c_void_p()
        rc = L.lxo_create(C.byref(ctx), device)
        if rc != A.LXO_OK:
            raise A.LxoError(rc, "lxo_create failed")
        self._ctx = ctx
        self._L = L
        v = np.ascontiguousarray(det.verts, np.float32)
        t = np.ascontiguousarray(det.tris, np.uint32)
        mi = np.ascontiguousarray(det.mat_inner, np.uint8)
        mo = np.ascontiguousarray(det.mat_outer, np.uint8)
        sf = np.ascontiguousarray(det.surface, np.uint16)
        ch = np.ascontiguousarray(det.channel, np.int32)
        self._check(L.lxo_load_mesh(ctx, v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], mi.ctypes.data,
                                    mo.ctypes.data, sf.ctypes.data, ch.ctypes.data))
        self.set_materials(det.materials)
        self.set_surfaces(det.surfaces)
        P = max(1, det.n_pmts)
        pm = (A.lxo_pmt * P)()
        for i in range(P):
            pm[i].channel = i
            if i < det.n_pmts:
                pm[i].array = int(det.pmt_array[i])
                pm[i].center[:] = [float(x) for x in det.pmt_pos[i]]
        self._check(L.lxo_set_pmts(ctx, pm, P))
        self.n_channels = P
        bp = A.lxo_bvh_params(leaf_size, sah_bins, n_threads, 0)
        info = A.lxo_bvh_info()
        self._check(L.lxo_build_bvh(ctx, C.byref(bp), C.byref(info)))
        self.bvh_info = {f: getattr(info, f) for f, _ in A.lxo_bvh_info._fields_}

    def _check(self, rc):
        if rc != A.LXO_OK:
            raise A.LxoError(rc, self._L.lxo_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.lxo_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- tables -------------------------------------------------------------
    def set_materials(self, mats):
        arr = (A.lxo_material * len(mats))()
        for i, m in enumerate(mats):
            arr[i].n = m.n
            # passed as given: inf means no process, NaN is rejected by the library
            arr[i].abs_len_mm = m.abs_len_mm
            arr[i].rayleigh_len_mm = m.rayleigh_len_mm
            arr[i].dn_dlambda_per_nm = m.dn_dlambda_per_nm
            arr[i].rayleigh_exp = m.rayleigh_exp
        self._check(self._L.lxo_set_materials(self._ctx, arr, len(mats)))
        self.n_materials = len(mats)

    def set_surfaces(self, surfs):
        arr = (A.lxo_surface * max(1, len(surfs)))()
        for i, s in enumerate(surfs):
            arr[i].type, arr[i].reflectivity, arr[i].spec_frac, arr[i].qe = s.type, s.reflectivity, s.spec_frac, s.qe
            arr[i].transparency, arr[i].wire_reflectivity = s.transparency, s.wire_reflectivity
            arr[i].wire_spec_frac = s.wire_spec_frac
        self._check(self._L.lxo_set_surfaces(self._ctx, arr, len(surfs)))
        self.n_surfaces = len(surfs)

    @property
    def n_fates(self):
        return A.LXO_FATES_FIXED + self.n_materials + self.n_surfaces

    # -- adjoint --------------------------------------------------------------
    def set_adjoint(self, mats=(), surfs=()):
        """Track theta = (L_abs, L_ray) of each material in `mats`, then R
        (reflector) or T (electrode) of each surface in `surfs`."""
        m = (C.c_int32 * max(1, len(mats)))(*mats)
        sf = (C.c_int32 * max(1, len(surfs)))(*surfs)
        self._check(self._L.lxo_set_adjoint(self._ctx, m, len(mats), sf, len(surfs)))
        self.adj_mats, self.adj_surfs = list(mats), list(surfs)

    @property
    def n_tallies(self):
        return 2 * (len(self.adj_mats) + len(self.adj_surfs))

    @property
    def n_params(self):
        return 2 * len(self.adj_mats) + len(self.adj_surfs)

    def theta(self):
        """Current values of the tracked parameters (float64 tensor [Q])."""
        v = []
        for m in self.adj_mats:
            v += [self.det.materials[m].abs_len_mm, self.det.materials[m].rayleigh_len_mm]
        for q in self.adj_surfs:
            sf = self.det.surfaces[q]
            v.append(sf.reflectivity if sf.type == REFLECTOR else sf.transparency)
        return torch.tensor(v, dtype=torch.float64)

    def set_theta(self, theta):
        """Sets the tracked parameters in the tracker's own material / surface
        tables (not the detector it was built from) and uploads them."""
        th = [float(x) for x in (theta.detach().cpu().tolist() if torch.is_tensor(theta) else theta)]
        k = 0
        for m in self.adj_mats:
            self.det.materials[m].abs_len_mm, self.det.materials[m].rayleigh_len_mm = th[k], th[k + 1]
            k += 2
        for q in self.adj_surfs:
            sf = self.det.surfaces[q]
            if sf.type == REFLECTOR:
                sf.reflectivity = th[k]
            else:
                sf.transparency = th[k]
            k += 1
        self.set_materials(self.det.materials)
        self.set_surfaces(self.det.surfaces)

    def jacobian(self, sums, g=None, stream=None):
        """J [P, Q] (and grad = J^T g [Q] if g is given) from adjoint tally sums
        [P, K] at the current parameter values, computed on the device."""
        shape = sums.shape[:-1]
        sums = sums.reshape(-1, self.n_tallies).contiguous()
        rows = sums.shape[0]
        J = torch.empty((rows, self.n_params), dtype=torch.float64, device=self.device)
        grad = None
        if g is not None:
            g = g.reshape(-1).to(device=self.device, dtype=torch.float64).contiguous()
            grad = torch.empty(self.n_params, dtype=torch.float64, device=self.device)
        self._check(self._L.lxo_adjoint_jacobian(self._ctx, _ptr(sums), rows, _ptr(J), _ptr(g), _ptr(grad),
                                                 _stream(stream)))
        J = J.reshape(*shape, self.n_params)
        return J if g is None else (J, grad)

    # -- geometry query -----------------------------------------------------
    def trace_rays(self, org, dir, skip=None, tmax=None, stream=None):
        org = org.contiguous()
        dir = dir.contiguous()
        n = org.shape[0]
        hit = torch.empty(n, dtype=torch.int32, device=self.device)
        t = torch.empty(n, dtype=torch.float32, device=self.device)
        sk = None if skip is None else skip.to(torch.int32).contiguous()
        tm = None if tmax is None else tmax.contiguous()
        self._check(self._L.lxo_trace_rays(self._ctx, _ptr(org), _ptr(dir), _ptr(sk), _ptr(tm), n, _ptr(hit),
                                           _ptr(t), _stream(stream)))
        return hit, t

    def sample_source(self, n, base=0, seed=0, source=None, stream=None, time=False, wavelength=False):
        """First photon states: pos, dir, pol [n, 3]; then the emission times
        [n] if time, and the wavelengths [n] (nm) if wavelength."""
        src = make_source(source or self.det.source)
        pos = torch.empty((n, 3), dtype=torch.float32, device=self.device)
        dir = torch.empty_like(pos)
        pol = torch.empty_like(pos)
        t = torch.empty(n, dtype=torch.float32, device=self.device) if time else None
        wl = torch.empty(n, dtype=torch.float32, device=self.device) if wavelength else None
        self._check(self._L.lxo_sample_source(self._ctx, C.byref(src), n, base, seed, _ptr(pos), _ptr(dir), _ptr(pol),
                                              _ptr(t), _ptr(wl), _stream(stream)))
        return (pos, dir, pol) + ((t,) if time else ()) + ((wl,) if wavelength else ())

    # -- propagation --------------------------------------------------------
    def alloc_results(self, n_tbins=1000, per_photon_n=0):
        P, dev = self.n_channels, self.device
        out = dict(lce=torch.zeros(P, dtype=torch.int32, device=dev),
                   det=torch.zeros(P, dtype=torch.int32, device=dev),
                   hist=torch.zeros((P, n_tbins + 1), dtype=torch.int32, device=dev),
                   fates=torch.zeros(self.n_fates, dtype=torch.int64, device=dev))
        if per_photon_n:
            out.update(fate=torch.zeros(per_photon_n, dtype=torch.int32, device=dev),
                       detail=torch.zeros(per_photon_n, dtype=torch.int32, device=dev),
                       steps=torch.zeros(per_photon_n, dtype=torch.int32, device=dev),
                       time=torch.zeros(per_photon_n, dtype=torch.float32, device=dev),
                       state=torch.zeros((per_photon_n, 9), dtype=torch.float32, device=dev))
        return out

    def _results(self, out):
        r = A.lxo_results()
        r.lce, r.det, r.hist, r.fates = (out[k].data_ptr() for k in ("lce", "det", "hist", "fates"))
        if "fate" in out:
            r.ph_fate, r.ph_detail = out["fate"].data_ptr(), out["detail"].data_ptr()
            r.ph_steps, r.ph_time = out["steps"].data_ptr(), out["time"].data_ptr()
        if "state" in out:
            r.ph_state = out["state"].data_ptr()
        if "stats" in out:
            r.stats = out["stats"].data_ptr()
        if "adjoint" in out:
            r.adjoint = out["adjoint"].data_ptr()
        return r

    def propagate(self, n, base=0, seed=0, source=None, explicit=None, max_steps=10000, n_tbins=1000, tbin_ns=1.0,
                  per_photon=False, out=None, stream=None, sync=True, stats=False, adjoint=False):
        """Propagates photons base..base+n-1; returns (accumulates into) a dict
        of device tensors: lce, det [P], hist [P, n_tbins+1], fates [8+M+S]
        and, with per_photon, fate / detail / steps / time [n] and state [n, 9]
        (final position, direction, polarisation); with stats,
        stats [LXO_STATS_LEN] as documented for lxo_results.stats in include/lxo.h; with
        adjoint, adjoint [P, K] (tally sums of detected photons)."""
        if out is None:
            out = self.alloc_results(n_tbins, n if per_photon else 0)
        if stats and "stats" not in out:
            out["stats"] = torch.zeros(A.LXO_STATS_LEN, dtype=torch.int64, device=self.device)
        if adjoint and "adjoint" not in out:
            out["adjoint"] = torch.zeros((self.n_channels, self.n_tallies), dtype=torch.float64, device=self.device)
        src = make_source(source or self.det.source, explicit)
        if explicit is not None and src.kind != SRC_EXPLICIT:
            raise ValueError("explicit arrays need an SRC_EXPLICIT source")
        flags = (A.LXO_FLAG_STATS if stats else 0) | (A.LXO_FLAG_ADJOINT if adjoint else 0)
        rp = A.lxo_run_params(seed, max_steps, n_tbins, tbin_ns, flags)
        res = self._results(out)
        st = _stream(stream)
        self._check(self._L.lxo_propagate(self._ctx, C.byref(src), n, base, C.byref(rp), C.byref(res), st))
        if sync:
            self._check(self._L.lxo_sync(self._ctx, st))
        return out

    def propagate_host(self, n, base=0, seed=0, source=None, max_steps=10000, n_tbins=1000, tbin_ns=1.0,
                       out=None, stream=None):
        """End-to-end call with host (numpy) result buffers."""
        P = self.n_channels
        if out is None:
            out = dict(lce=np.zeros(P, np.uint32), det=np.zeros(P, np.uint32),
                       hist=np.zeros((P, n_tbins + 1), np.uint32), fates=np.zeros(self.n_fates, np.uint64))
        src = make_source(source or self.det.source)
        rp = A.lxo_run_params(seed, max_steps, n_tbins, tbin_ns, 0)
        r = A.lxo_results()
        r.lce, r.det, r.hist, r.fates = (out[k].ctypes.data for k in ("lce", "det", "hist", "fates"))
        self._check(self._L.lxo_propagate_host(self._ctx, C.byref(src), n, base, C.byref(rp), C.byref(r),
                                               _stream(stream)))
        return out

    def sync(self, stream=None):
        self._check(self._L.lxo_sync(self._ctx, _stream(stream)))

    # -- batched events -------------------------------------------------------
    def upload_events(self, events, first_event=0):
        """events: list of (Source (POINT / SEGMENT / BALL), n_photons); the
        first has event id first_event (photon ids (id << 32) | i), the
        tallies' rows follow the list."""
        arr = (A.lxo_event * len(events))()
        for i, (src, n) in enumerate(events):
            e = arr[i]
            e.kind, e.medium = int(src.kind), int(src.medium)
            e.center[:] = [float(x) for x in src.center]
            e.p1[:] = [float(x) for x in src.p1]
            e.radius, e.t0, e.n_photons = float(src.radius), float(src.t0), int(n)
            e.singlet_frac, e.tau_singlet_ns, e.tau_triplet_ns = (float(src.singlet_frac), float(src.tau_singlet_ns),
                                                                  float(src.tau_triplet_ns))
            e.wl_mean_nm, e.wl_fwhm_nm = float(src.wl_mean_nm), float(src.wl_fwhm_nm)
        self._check(self._L.lxo_upload_events(self._ctx, arr, len(events), first_event))
        self.n_events = len(events)
        self.event_photons = int(sum(int(n) for _, n in events))

    def alloc_event_results(self, n_tbins=256, hist=True, adjoint=False):
        E, P, dev = self.n_events, self.n_channels, self.device
        out = dict(lce=torch.zeros((E, P), dtype=torch.int32, device=dev),
                   det=torch.zeros((E, P), dtype=torch.int32, device=dev),
                   fates=torch.zeros(self.n_fates, dtype=torch.int64, device=dev))
        if hist:
            out["hist"] = torch.zeros((E, P, n_tbins + 1), dtype=torch.int32, device=dev)
        if adjoint:
            out["adjoint"] = torch.zeros((E, P, self.n_tallies), dtype=torch.float64, device=dev)
        return out

    def propagate_events(self, seed=0, n_tbins=256, tbin_ns=1.0, max_steps=10000, out=None, hist=True,
                         stream=None, sync=True, adjoint=False):
        """All uploaded events in one launch; per-event tallies [E, P] (and
        [E, P, n_tbins+1] time histograms if hist, adjoint sums [E, P, K] if
        adjoint)."""
        if out is None:
            out = self.alloc_event_results(n_tbins, hist, adjoint)
        rp = A.lxo_run_params(seed, max_steps, n_tbins, tbin_ns, A.LXO_FLAG_ADJOINT if adjoint else 0)
        r = A.lxo_results()
        r.lce, r.det, r.fates = out["lce"].data_ptr(), out["det"].data_ptr(), out["fates"].data_ptr()
        r.hist = out["hist"].data_ptr() if "hist" in out else None
        r.adjoint = out["adjoint"].data_ptr() if adjoint else None
        st = _stream(stream)
        self._check(self._L.lxo_propagate_events(self._ctx, C.byref(rp), C.byref(r), st))
        if sync:
            self._check(self._L.lxo_sync(self._ctx, st))
        return out

    def set_launch(self, blocks_per_sm=0, chunk=0, threads=0):
        """Launch shape: CTAs per SM (0 = occupancy limit), photon ids per
        warp grab (0 = 64), threads per CTA (128 or 256; 0 = 256)."""
        self._check(self._L.lxo_set_launch(self._ctx, blocks_per_sm, chunk, threads))


def autotune_launch(tracker, run, blocks=(2, 3, 4, 5), chunks=(32, 64, 128, 256), threads=(256,), reps=2):
    """Times `run()` (one launch of the workload to tune, on the current
    stream) for every launch shape (threads per CTA x CTAs per SM x chunk;
    CTAs per SM are counted in 256-thread units, so 128-thread CTAs run
    twice as many) and keeps the fastest; returns (threads, blocks_per_sm,
    chunk, ms) and the table of timings keyed by (threads, blocks_per_sm,
    chunk)."""
    table = {}
    for t in threads:
        for b in blocks:
            for c in chunks:
                bps = b * (256 // t)
                tracker.set_launch(bps, c, t)
                run()
                torch.cuda.synchronize()
                ts = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    run()
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                table[(t, bps, c)] = min(ts)
    best = min(table, key=table.get)
    tracker.set_launch(best[1], best[2], best[0])
    return (*best, table[best]), table


class LightCollection(torch.autograd.Function):
    """Expected detected hits per PMT as a differentiable function of the
    tracked optical parameters theta (Tracker.set_adjoint): the forward pass
    propagates `n` photons at theta with the adjoint tallies on; the backward
    pass is the score-function gradient J^T g computed by the library's
    adjoint kernels.  Returns float64 hits [P] (counts for n photons)."""

    @staticmethod
    def forward(ctx, theta, tracker, n, seed=0, source=None, base=0):
        tracker.set_theta(theta)
        out = tracker.propagate(n, base=base, seed=seed, source=source, adjoint=True)
        ctx.tracker = tracker
        ctx.theta = theta.detach().clone()
        ctx.save_for_backward(out["adjoint"])
        return out["det"].to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        (sums,) = ctx.saved_tensors
        tr = ctx.tracker
        tr.set_theta(ctx.theta)
        _, grad = tr.jacobian(sums, g)
        return grad.to(ctx.theta.device), None, None, None, None, None


class EventLightCollection(torch.autograd.Function):
    """Expected detected hits per (event, PMT) [E, P] of the uploaded events
    as a differentiable function of the tracked parameters theta; one
    batched launch forward, the adjoint kernels backward."""

    @staticmethod
    def forward(ctx, theta, tracker, seed=0):
        tracker.set_theta(theta)
        out = tracker.propagate_events(seed=seed, hist=False, adjoint=True)
        ctx.tracker = tracker
        ctx.theta = theta.detach().clone()
        ctx.save_for_backward(out["adjoint"])
        return out["det"].to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        (sums,) = ctx.saved_tensors
        tr = ctx.tracker
        tr.set_theta(ctx.theta)
        _, grad = tr.jacobian(sums, g)
        return grad.to(ctx.theta.device), None, None
