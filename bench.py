"""Benchmark: photons propagated to fate per second on the DARWIN-scale mesh.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one lxo_propagate of a batch of photons (default 1e8) uniform in
the active LXe volume of the DARWIN-scale detector (24-sided PTFE wall inscribed
in r = 1300 mm, 889 + 889 3-inch PMTs, gate / anode / cathode as hexagonal
216 um wire meshes at 5 mm pitch: 1.78e7 triangles), all interactions on,
through the whole path (source sampling, BVH traversal, bulk sampling,
Fresnel / TIR, reflectors, wire meshes, photocathodes, tallies).  The BVH
(1.3 GB) is larger than L2, so no flush is needed between steps.

Under torchrun each rank takes its own photon-id range (weak scaling; no
collective on the data path); the timing is the max over ranks.

--impl reference times the CPU oracle (the plain scalar C tracker) on the host
cores on a bounded sample of the same workload.

Output: one JSON line {"details": ...} with every per-ring, per-PMT and
per-shape table, then the bench line itself, kept short enough to be read
whole (the forward+adjoint ratio and the finite-difference summary last).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "photons/sec to fate, DARWIN mesh, 1 GB300"
UNIT = "photons/s"
OPS_PER_NODE, OPS_PER_TRI, OPS_PHYSICS = 40, 50, 250
N_SM, LANES_PER_SM = 152, 128
# DRAM bytes (read + write) per photon of the propagation kernel: ncu
# dram__bytes_read.sum + dram__bytes_write.sum of one timed launch on 2e6
# photons of this workload (8.423 GB + 4.602 GB), divided by 2e6; scales with
# the photon count.  Most of the writes, and a third of the reads, are the
# 32-register build's spills and traversal stack leaving L1 and L2.
DRAM_BYTES_PER_PHOTON = 6512
# warp instructions issued per photon step by the same capture
# (smsp__inst_executed.sum 1.0792e10 over 5.147e7 steps); the issue-slot peak
# is 152 SMs x 4 schedulers x 1 warp instruction per cycle x the SM clock
WARP_INST_PER_STEP = 209.7
SCHEDULERS_PER_SM = 4
# The kernel build those two numbers were captured from: its ptxas
# signature and the SHA-256 of its sources.  When the built kernel differs,
# the line says roofline.stale = true and drops traffic (the counters must
# be taken again).
TIMED_KERNEL = "_ZN3lxo11k_propagateILb0ELb0ELb0ELi256ELi8EEEvNS_10PropParamsE"   # k_propagate<0,0,0,256,8>
KERNEL_SOURCES = ("paper_2203_14354_gb300/csrc/lxo_kernels.cu", "paper_2203_14354_gb300/csrc/lxo_internal.h")
CAPTURED_KERNEL = {"registers": 32, "spill_stores": 538, "spill_loads": 616,
                   "sources_sha256": "1fa675c8893873eba0ba098175fb9ad1a31d29e08863aa4f1dad41da785a8a8a"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--photons", type=float, default=1e8, help="photons per rank per step")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the forward+adjoint cost measurement")
    ap.add_argument("--no-adjoint-fd", action="store_true",
                    help="skip the 1e9-photon finite-difference check of the adjoint")
    ap.add_argument("--no-events", action="store_true", help="skip the batched-events measurement")
    ap.add_argument("--no-calibration", action="store_true", help="skip the reduced calibration fit")
    ap.add_argument("--no-spectral", action="store_true",
                    help="skip the emission-spectrum (photons carry a wavelength) measurement")
    return ap.parse_args()


def workload_config(n, world, n_tris):
    return {"workload": "DARWIN-scale dual-phase TPC forward: 24-gon PTFE wall r=1300 mm, 889+889 3-inch PMTs, "
                        f"gate/anode/cathode hex wire meshes 216 um @ 5 mm, {n_tris / 1e7:.2f}e7 triangles; photons "
                        "uniform in the active LXe, isotropic, random linear polarisation, t=0, 175 nm",
            "photons_per_step": int(n) * world, "photons_per_rank": int(n), "triangles": int(n_tris),
            "lxe_abs_m": 50, "lxe_rayleigh_cm": 40, "ptfe_R": [0.95, 0.70], "qe": 0.3,
            "time_bins_ns": "1000 x 1 ns + overflow", "l2": "inputs larger than L2 (BVH 1.3 GB), no flush",
            "parallelism": f"photon-id ranges per rank x{world}" if world > 1 else "single GPU"}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 4 + i and r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def kernel_signature():
    """ptxas registers and spill bytes of the timed kernel in the library's
    build log, and the SHA-256 of the kernel's sources."""
    from paper_2203_14354_gb300 import build
    sig = {"registers": None, "spill_stores": None, "spill_loads": None}
    try:
        lines = open(os.path.join(build.OUT_DIR, "ptxas.log")).read().splitlines()
    except OSError:
        lines = []
    for i, ln in enumerate(lines):
        if f"Compiling entry function '{TIMED_KERNEL}'" in ln:
            for nxt in lines[i + 1:i + 4]:
                if "spill stores" in nxt:
                    w = nxt.replace(",", " ").split()
                    sig["spill_stores"] = int(w[w.index("spill") - 2])
                    sig["spill_loads"] = int(w[w.index("loads") - 3])
                if "Used" in nxt and "registers" in nxt:
                    w = nxt.split()
                    sig["registers"] = int(w[w.index("registers,") - 1])
            break
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    sig["sources_sha256"] = h.hexdigest()
    return sig


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def cpu_baseline(det, target_s):
    """The oracle as it stands, on all host cores, on a bounded sample."""
    import oracle
    orc = oracle.Oracle(det)
    cores = os.cpu_count() or 1
    n0 = 20000
    t0 = time.perf_counter()
    orc.propagate(n0, base=0, seed=12345, threads=cores)
    dt0 = time.perf_counter() - t0
    n = int(min(5e7, max(n0, n0 * target_s / max(dt0, 1e-3))))
    t0 = time.perf_counter()
    res = orc.propagate(n, base=n0, seed=12345, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": res["threads"], "kind": "oracle",
            "sample": f"{n} photons of the same workload (seed 12345), {dt:.1f} s wall on {res['threads']} threads; "
                      f"scene build excluded"}, res, n


def adjoint_cost(args, n=10_000_000, reps=3):
    """Forward + adjoint against the plain forward on the 50 cm TPC with 61 +
    61 PMTs and thin-disk electrodes, 1e7 photons, 7 parameters: the time of
    the propagation with per-photon tallies (and the Jacobian kernel) over the
    time of the plain propagation, same photons, each at its faster register
    budget (5 or 8 CTAs of 256 threads per SM)."""
    import torch
    from paper_2203_14354_gb300 import geometry, Tracker
    det = geometry.scaled_tpc()
    trk = Tracker(det)
    trk.set_adjoint([geometry.LXE], [0, 1, 4, 5, 6])
    out = trk.alloc_results(1000)
    out["adjoint"] = torch.zeros((trk.n_channels, trk.n_tallies), dtype=torch.float64, device=trk.device)

    def run(adj):
        for v in out.values():
            v.zero_()
        trk.propagate(n, seed=5, out=out, adjoint=adj, sync=False)
        if adj:
            trk.jacobian(out["adjoint"])

    times, shapes, table = {}, {}, {}
    for adj in (False, True):
        for bps in (5, 8):
            trk.set_launch(bps, 0, 256)
            run(adj)
            trk.sync()
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                run(adj)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            table[f"{'adjoint' if adj else 'forward'} {bps} CTAs/SM"] = statistics.median(ts)
            if adj not in times or statistics.median(ts) < times[adj]:
                times[adj], shapes[adj] = statistics.median(ts), bps
    trk.set_launch(0, 0, 0)
    trk.sync()
    res = {"workload": "50 cm dual-phase TPC, 61+61 PMTs, thin-disk gate/anode/cathode, 1e7 photons, 7 parameters",
           "fwd_ms": times[False], "fwd_adjoint_ms": times[True], "ratio": times[True] / times[False],
           "fwd_photons_per_s": n / (times[False] / 1e3),
           "ctas_per_sm": {"forward": shapes[False], "adjoint": shapes[True]}, "ms_by_shape": table}
    if not args.no_adjoint_fd:
        res["fd_check"] = adjoint_fd_check(trk)
    return res


def pmt_rings(det):
    """PMTs grouped by array (top first) and hexagonal ring of the window
    lattice (pitch = nearest-neighbour distance within one array).  Returns
    labels, boolean masks [P] and the pitch."""
    from paper_2203_14354_gb300 import geometry
    pos = np.asarray(det.pmt_pos, np.float64)[:, :2]
    arr = np.asarray(det.pmt_array)
    one = pos[arr == arr[0]]
    d = np.sqrt(((one[:, None] - one[None]) ** 2).sum(-1)) + np.eye(len(one)) * 1e30
    pitch = float(np.median(d.min(1)))
    ring = geometry.hex_ring(pos, pitch)
    labels, masks = [], []
    for a in (1, 0):
        for k in np.unique(ring[arr == a]):
            m = (arr == a) & (ring == k)
            labels.append(f"{'top' if a == 1 else 'bottom'} ring {k} ({int(m.sum())} PMTs)")
            masks.append(m)
    return labels, masks, pitch


def adjoint_fd_check(trk, batches=10, n_batch=100_000_000, h=1e-3, seed=31, h_wide=3e-2, noisy=0.02):
    """Accuracy of the adjoint gradient of detected hits (total, top array,
    bottom array) against central finite differences with common random
    numbers at relative step h (same seed and photon ids at theta +- h), 1e9
    photons in 10 batches; mean and batch-means standard error of both
    estimates per parameter and aggregate.  Parameters whose differences are
    noisier than `noisy` (relative standard error) at h are differenced again
    at h_wide and h_wide / 2 and extrapolated (Richardson): the noise of a
    common-random-number difference falls as h^-1/2, its truncation error
    grows as h^2 and the extrapolation removes that term."""
    top = torch_bool(trk.det.pmt_array == 1, trk.device)
    theta0 = trk.theta()
    aggs = ("total", "top", "bottom")

    def sums(v):  # [P] or [P, Q] -> per aggregate
        return [v.sum(0), v[top].sum(0), v[~top].sum(0)]

    adj = np.zeros((len(aggs), batches, trk.n_params))
    fd = np.zeros((len(aggs), batches, trk.n_params))
    P = trk.n_channels
    adj_pmt = np.zeros((batches, P, trk.n_params))
    fd_pmt = np.zeros((batches, P, trk.n_params))
    t0 = time.perf_counter()
    trk.set_theta(theta0)
    for b in range(batches):
        out = trk.propagate(n_batch, base=b * n_batch, seed=seed, adjoint=True, n_tbins=1)
        J = trk.jacobian(out["adjoint"])
        adj_pmt[b] = J.cpu().numpy()
        for a, v in enumerate(sums(J)):
            adj[a, b] = v.cpu().numpy()
    def differences(q, hq, dst, per_pmt=None):
        step = hq * float(theta0[q])
        for b in range(batches):
            res, dets = [], []
            for sgn in (1.0, -1.0):
                th = theta0.clone()
                th[q] += sgn * step
                trk.set_theta(th)
                det = trk.propagate(n_batch, base=b * n_batch, seed=seed, n_tbins=1)["det"].double()
                res.append([float(x) for x in sums(det)])
                dets.append(det.cpu().numpy())
            for a in range(len(aggs)):
                dst[a, b, q] = (res[0][a] - res[1][a]) / (2.0 * step)
            if per_pmt is not None:
                per_pmt[b, :, q] = (dets[0] - dets[1]) / (2.0 * step)

    for q in range(trk.n_params):
        differences(q, h, fd, fd_pmt)
    fd_w = np.full_like(fd, np.nan)
    fd_half = np.full_like(fd, np.nan)
    wide = [q for q in range(trk.n_params)
            if np.max(fd[:, :, q].std(1, ddof=1) / math.sqrt(batches) / np.abs(fd[:, :, q].mean(1))) > noisy]
    for q in wide:
        # Richardson extrapolation of the central difference, D(h) = f' +
        # c h^2 + O(h^4): (4 D(h/2) - D(h)) / 3 cancels the h^2 term, which
        # at a few per cent of theta exceeds the noise of the common-random-
        # number differences
        differences(q, h_wide, fd_w)
        differences(q, h_wide / 2, fd_half)
        fd_w[:, :, q] = (4.0 * fd_half[:, :, q] - fd_w[:, :, q]) / 3.0
    trk.set_theta(theta0)
    names = ["L_abs_LXe", "L_ray_LXe", "R_PTFE_LXe", "R_PTFE_GXe", "T_gate", "T_anode", "T_cathode"]
    out = {"photons": batches * n_batch, "h_rel": h, "params": names[:trk.n_params],
           "seconds": time.perf_counter() - t0}
    def compare(a, d):
        a_m, f_m = adj[a].mean(0), d[a].mean(0)
        a_s = adj[a].std(0, ddof=1) / math.sqrt(batches)
        f_s = d[a].std(0, ddof=1) / math.sqrt(batches)
        return {"adjoint": a_m.tolist(), "adjoint_se": a_s.tolist(), "fd": f_m.tolist(), "fd_se": f_s.tolist(),
                "rel_diff": (np.abs(a_m - f_m) / np.abs(f_m)).tolist(),
                "z": (np.abs(a_m - f_m) / np.sqrt(a_s ** 2 + f_s ** 2)).tolist()}

    for a, name in enumerate(aggs):
        out[name] = compare(a, fd)
    # per PMT: paired batch differences adjoint - FD (same photons in a
    # batch), t_c = mean / standard error with nu = batches - 1; under
    # agreement sum_c t_c^2 has mean n nu / (nu - 2) and variance
    # n 2 nu^2 (nu - 1) / ((nu - 2)^2 (nu - 4))
    e = adj_pmt - fd_pmt
    se = e.std(0, ddof=1) / math.sqrt(batches)
    nu = batches - 1
    sum_t2, n_pmt, z_sum = [], [], []
    for q in range(trk.n_params):
        ok = se[:, q] > 0
        t2 = (e.mean(0)[ok, q] / se[ok, q]) ** 2
        n = int(ok.sum())
        mean = n * nu / (nu - 2)
        sd = math.sqrt(n * 2 * nu ** 2 * (nu - 1) / ((nu - 2) ** 2 * (nu - 4)))
        sum_t2.append(float(t2.sum()))
        n_pmt.append(n)
        z_sum.append(float((t2.sum() - mean) / sd) if n else None)
    out["per_pmt"] = {"sum_t2": sum_t2, "pmts": n_pmt, "expected": [k * nu / (nu - 2) for k in n_pmt],
                      "z": z_sum}
    # rings: PMTs of one array at the same hexagonal ring (radius / pitch,
    # rounded), the aggregate between one array and one PMT
    labels, masks, pitch = pmt_rings(trk.det)
    rings_out = {"adjoint": [], "fd": [], "rel_diff": [], "z": []}
    for m in masks:
        av, fv = adj_pmt[:, m].sum(1), fd_pmt[:, m].sum(1)  # [batches, Q]
        am, fm = av.mean(0), fv.mean(0)
        sa, sf = av.std(0, ddof=1) / math.sqrt(batches), fv.std(0, ddof=1) / math.sqrt(batches)
        rings_out["adjoint"].append(am.tolist())
        rings_out["fd"].append(fm.tolist())
        rings_out["rel_diff"].append((np.abs(am - fm) / np.abs(fm)).tolist())
        rings_out["z"].append((np.abs(am - fm) / np.sqrt(sa ** 2 + sf ** 2)).tolist())
    zr = np.array(rings_out["z"])
    out["rings"] = {"labels": labels, "pitch_mm": pitch, **rings_out, "z_max": zr.max(0).tolist(),
                    "n_over_2": (zr > 2).sum(0).tolist()}
    if wide:
        out["wide_step"] = {"h_rel": h_wide, "richardson_h_rel": [h_wide, h_wide / 2],
                            "params": [names[q] for q in wide]}
        for a, name in enumerate(aggs):
            c = compare(a, fd_w)
            out["wide_step"][name] = {k: [v[q] for q in wide] for k, v in c.items()}
    out["seconds"] = time.perf_counter() - t0
    return out


def adjoint_summary(adj):
    """The forward+adjoint cost and the finite-difference check in a few
    numbers: per parameter, the relative difference of the adjoint and the
    finite-difference totals and its z; the largest relative difference over
    the aggregates (total, top, bottom) that the differences resolve (their
    standard error under 2 %), at the step used for each parameter."""
    out = {"ratio": round(adj["ratio"], 4), "fwd_ms": round(adj["fwd_ms"], 3),
           "fwd_adjoint_ms": round(adj["fwd_adjoint_ms"], 3)}
    fd = adj.get("fd_check")
    if not fd:
        return out
    worst, worst_z = 0.0, 0.0
    wide = fd.get("wide_step", {})
    for q, name in enumerate(fd["params"]):
        src, k = fd, q
        if name in wide.get("params", []):
            src, k = wide, wide["params"].index(name)
        for agg in ("total", "top", "bottom"):
            a = src[agg]
            if a["fd_se"][k] < 0.02 * abs(a["fd"][k]):
                worst = max(worst, a["rel_diff"][k])
                worst_z = max(worst_z, a["z"][k])
    out["fd"] = {"photons": fd["photons"], "h_rel": fd["h_rel"], "h_wide": wide.get("h_rel"),
                 "wide_params": wide.get("params", []),
                 "rel_diff_total": [round(x, 4) for x in fd["total"]["rel_diff"]],
                 "z_total": [round(x, 2) for x in fd["total"]["z"]],
                 "max_rel_diff_resolved": round(worst, 4), "max_z_resolved": round(worst_z, 2),
                 "per_pmt_z": [None if z is None else round(z, 2) for z in fd["per_pmt"]["z"]],
                 "rings_z_max": round(max(fd["rings"]["z_max"]), 2)}
    return out


def calibration_check():
    """The gradient calibration on the 50 cm TPC (64 point sources x 2e5
    photons on the nodes of a 5 cm 3-D grid in the LXe, hidden L_abs 30 m,
    L_Ray 35 cm, R_PTFE 0.97 / 0.80, start at the defaults): recovered values, their standard deviations from the Fisher
    information, pulls, and the time per model launch."""
    import torch
    from paper_2203_14354_gb300 import calibrate, geometry, Tracker
    det = geometry.scaled_tpc()
    trk = Tracker(det)
    trk.set_adjoint([geometry.LXE], [0, 1])
    theta0 = trk.theta().tolist()
    truth = [30_000.0, 350.0, 0.97, 0.80]
    ev = geometry.grid_sources(det, 200_000, 64, spacing=50.0, margin=50.0, seed=7)
    trk.upload_events(ev)
    target = calibrate.hit_maps(trk, truth, seed=7)
    cal = calibrate.Calibration(trk, ev, target, model_scale=2)
    res = cal.fit(theta0)
    rec = torch.tensor(res["theta"], dtype=torch.float64)
    cov = cal.covariance(rec, seed=98)
    sigma = cov.diagonal().sqrt()
    # the parameters are correlated (L_abs and R_PTFE both scale the total
    # light): chi^2 of the deviation with the full covariance, 4 degrees of
    # freedom, beside the per-parameter pulls
    st = calibrate.deviation_stats(rec, truth, cov)
    return {"workload": "50 cm TPC, 64 point sources x 2e5 photons on a 5 cm 3-D grid (model 2x), 4 parameters",
            "params": ["L_abs_LXe_mm", "L_ray_LXe_mm", "R_PTFE_LXe", "R_PTFE_GXe"], "truth": truth,
            "start": theta0, "recovered": res["theta"], "sigma": sigma.tolist(), "pull": st["pull"],
            "chi2": st["chi2"], "dof": len(truth), "z_eigen": st["z_eigen"], "corr": st["corr"],
            "launches": res["launches"], "scoring_steps": res["scoring_steps"], "seconds": res["seconds"]}


def torch_bool(mask, device):
    import torch
    return torch.from_numpy(np.asarray(mask, bool)).to(device)


def events_throughput(det, reps=3):
    """Batched events on the DARWIN-scale mesh: 4096 S1 point sources
    (log-uniform 1e2..1e5 photons) and 512 S2 segments in the gas gap
    (log-uniform 1e5..1e6), 2.6e8 photons, per-event per-PMT counts and
    256 x 1 ns time histograms; launch shape autotuned on a 10 % subset, then
    one launch captured in a CUDA graph and replayed."""
    import torch
    from paper_2203_14354_gb300 import geometry, Tracker
    from paper_2203_14354_gb300.tracker import autotune_launch
    ev = geometry.darwin_events(seed=0)
    trk = Tracker(det)
    trk.upload_events(ev[::10])
    sub = trk.alloc_event_results(256, hist=False)
    best, table = autotune_launch(trk, lambda: trk.propagate_events(seed=1, out=sub, hist=False, sync=False),
                                  blocks=(5, 6, 8), chunks=(32, 64, 128), threads=(128, 256), reps=2)
    del sub
    trk.upload_events(ev)
    out = trk.alloc_event_results(256, hist=True)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        trk.propagate_events(seed=2, out=out, sync=False)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for v in out.values():
            v.zero_()
        trk.propagate_events(seed=2, out=out, sync=False)
    graph.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    trk.sync()
    f = out["fates"].cpu().numpy()
    ms = statistics.median(ts)
    return {"workload": "4096 S1 + 512 S2 events, DARWIN-scale mesh, one persistent launch under a CUDA graph, "
                        "per-event per-PMT counts + 257-bin histograms", "events": len(ev),
            "photons": trk.event_photons, "ms": ms, "photons_per_s": trk.event_photons / (ms / 1e3),
            "launch": {"threads": best[0], "blocks_per_sm": best[1], "chunk": best[2]},
            "autotune_ms": {f"{t}t x {b} x {c}": round(ms, 3) for (t, b, c), ms in table.items()},
            "lce": float(out["lce"].sum().item()) / trk.event_photons, "escaped": int(f[4]), "geom_err": int(f[6])}


def spectral_throughput(trk, det, base, n=50_000_000, reps=3):
    """DARWIN-scale photons/s of the kernel built for photons that carry a
    wavelength: the LXe emission spectrum with Rayleigh's lambda^-4 law for
    the Rayleigh lengths of the liquid and the gas (no index dispersion, for
    which the paper gives no numbers), beside the same photon ids at 175 nm
    with the plain kernel.  CUDA events, median of `reps` launches."""
    import torch
    from dataclasses import replace
    from paper_2203_14354_gb300 import analysis, geometry
    mats = list(det.materials)
    lam4 = [replace(m, rayleigh_exp=4.0) if i in (geometry.LXE, geometry.GXE) else m for i, m in enumerate(mats)]
    spectral_src = det.source.with_spectrum(geometry.LXE_SPECTRUM)
    stream = torch.cuda.current_stream()
    res = {}
    try:
        for name, table, src in (("plain", mats, det.source), ("spectral", lam4, spectral_src)):
            trk.set_materials(table)
            out = trk.alloc_results(1000)
            trk.propagate(n // 10, base=base, seed=4, out=out, source=src)  # warm-up
            ms = []
            for r in range(reps):
                for v in out.values():
                    v.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                trk.propagate(n, base=base + (r + 1) * n, seed=4, out=out, source=src, sync=False)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            trk.sync()
            res[name] = dict(photons_per_s=n / (statistics.median(ms) / 1e3),
                             lce=float(out["lce"].sum()) / n,
                             t90_ns=analysis.t90(out["hist"].cpu().numpy(), 1.0))
    finally:
        trk.set_materials(mats)
    return {"workload": f"DARWIN-scale mesh, {n:.0e} photons uniform in the active LXe; LXe spectrum "
                        f"{geometry.LXE_SPECTRUM[0]} nm mean, {geometry.LXE_SPECTRUM[1]} nm FWHM; Rayleigh "
                        "length x (lambda/175 nm)^4 in LXe and GXe",
            "photons_per_s": res["spectral"]["photons_per_s"], "lce": res["spectral"]["lce"],
            "t90_ns": res["spectral"]["t90_ns"], "plain_175nm": res["plain"],
            "cost_ratio": res["plain"]["photons_per_s"] / res["spectral"]["photons_per_s"]}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2203_14354_gb300 import geometry
    det = geometry.darwin()
    import oracle
    orc = oracle.Oracle(det)
    cores = os.cpu_count() or 1
    per_step = max(20000, int(args.cpu_seconds * 90000 * cores / 8 / max(args.steps, 1)))
    per_step = min(per_step, 2_000_000)
    for w in range(args.warmup):
        orc.propagate(min(per_step, 20000), base=w * per_step, seed=999, threads=cores)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        orc.propagate(per_step, base=(args.warmup + s) * per_step, seed=999, threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 physics / f32 intersection", "data": "synthetic",
            "impl": "reference",
            "config": dict(workload_config(per_step, 1, det.n_tris), sample=f"{per_step} photons per step on the CPU"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} photons per step x {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    from paper_2203_14354_gb300 import analysis, geometry, Tracker

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = int(args.photons)
    det = geometry.darwin()
    t0 = time.perf_counter()
    trk = Tracker(det, device=local)
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    base0 = rank * n * (args.warmup + args.steps + 4)
    out = trk.alloc_results(1000)

    def barrier():
        if world > 1:
            dist.barrier()

    def step(k):
        for v in out.values():
            v.zero_()
        trk.propagate(n, base=base0 + k * n, seed=1, out=out, sync=False)

    for w in range(args.warmup):
        step(w)
    trk.sync()
    # per-step timing of the propagation kernel alone (events on the launching stream)
    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            for v in out.values():
                v.zero_()
            k_start[k].record(stream)
            trk.propagate(n, base=base0 + (args.warmup + k) * n, seed=1, out=out, sync=False)
            k_end[k].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    trk.sync()
    barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in zip(k_start, k_end)]
    if world > 1:
        # the one collective of the photon-id split: the tallies of the last
        # timed step summed over the ranks, checked against the photons run
        from paper_2203_14354_gb300.shard import reduce_tallies
        reduce_tallies(out)
    fates = out["fates"].cpu().numpy()
    lce = out["lce"].cpu().numpy()
    t90 = analysis.t90(out["hist"].cpu().numpy(), 1.0)
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps
    value = world * n * args.steps / (elapsed_ms / 1e3)
    tallies = {"photons": world * n, "fates_sum": int(fates[:7].sum()), "reduced_over_ranks": world,
               "ok": int(fates[:7].sum()) == world * n}
    # traversal work of the same batch (separate, untimed launch of the counting build)
    st_out = trk.alloc_results(1000)
    trk.propagate(n, base=base0 + args.warmup * n, seed=1, out=st_out, stats=True)
    stats = st_out["stats"].cpu().numpy().astype(np.float64)
    steps_total, nodes, leaves, tris, node_it, leaf_it, outer_it, trav_cyc, loop_cyc = stats[:9]
    simd = {"node_loop": nodes / max(32 * node_it, 1), "leaf_loop": leaves / max(32 * leaf_it, 1),
            "photon_loop": steps_total / max(32 * outer_it, 1), "traversal_cycle_share": trav_cyc / max(loop_cyc, 1)}
    bytes_per_step = (nodes * 64 + tris * 48) / steps_total
    kern_s = statistics.mean(kern_ms) / 1e3
    fetch_gbs = steps_total * bytes_per_step / kern_s / 1e9
    # algorithmic lane operations per photon step: 40 per BVH node visit (two slab
    # tests), 50 per triangle test (watertight), 250 of physics (Philox, logs,
    # interaction); peak = 152 SMs x 128 FP32/INT32 lanes x max SM clock
    ops_per_step = (nodes * OPS_PER_NODE + tris * OPS_PER_TRI) / steps_total + OPS_PHYSICS
    achieved = steps_total * ops_per_step / kern_s / 1e9
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    alu_peak = N_SM * LANES_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e9
    issue_rate = steps_total * WARP_INST_PER_STEP / kern_s
    issue_peak = N_SM * SCHEDULERS_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6

    # end to end through the C ABI with host result buffers (copies in the timed region)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    host = None
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        host = trk.propagate_host(n, base=base0 + (args.warmup + args.steps + k) * n, seed=2)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    P = trk.n_channels
    d2h = 4 * (2 * P + P * 1001) + 8 * trk.n_fates
    import ctypes
    from paper_2203_14354_gb300 import _capi
    h2d = ctypes.sizeof(_capi.lxo_source) + ctypes.sizeof(_capi.lxo_run_params)

    # t90 with the nuclear-recoil scintillation time profile (untimed side run, 1e7 photons)
    t90_nr = None
    if rank == 0:
        nr = trk.propagate(min(n, 10_000_000), base=base0 + 10**12, seed=3,
                           source=det.source.with_profile(geometry.NR_PROFILE))
        t90_nr = analysis.t90(nr["hist"].cpu().numpy(), 1.0)

    adjoint = adjoint_cost(args) if (rank == 0 and not args.no_adjoint) else None
    events = events_throughput(det) if (rank == 0 and not args.no_events) else None
    spectral = (spectral_throughput(trk, det, base0 + 2 * 10**12)
                if (rank == 0 and not args.no_spectral) else None)
    calibration = calibration_check() if (rank == 0 and not args.no_calibration) else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, _, _ = cpu_baseline(det, args.cpu_seconds)

    if rank == 0:
        sig = kernel_signature()
        stale = any(sig[k] != CAPTURED_KERNEL[k] for k in CAPTURED_KERNEL)
        phases = dict(zip(("node_loop", "leaf_loop", "trav_setup", "draws", "interaction", "refill"),
                          stats[29:35] / max(stats[29:35].sum(), 1.0)))
        details = {
            "roofline": {"per_step": {"nodes": nodes / steps_total, "leaves": leaves / steps_total,
                                      "triangles": tris / steps_total, "ops": ops_per_step,
                                      "fetch_bytes": bytes_per_step},
                         "fetch": {"achieved_gbs": fetch_gbs, "hbm_peak_gbs": hbm, "frac_of_hbm": fetch_gbs / hbm},
                         "simd_efficiency": simd, "lane_cycle_share": phases,
                         "issue": {"warp_inst_per_step": WARP_INST_PER_STEP,
                                   "achieved_g_warp_inst_s": issue_rate / 1e9,
                                   "peak_g_warp_inst_s": issue_peak / 1e9, "frac": issue_rate / issue_peak},
                         "kernel_signature": sig, "captured_kernel": CAPTURED_KERNEL},
            "physics": {"fates": fates.tolist()}, "setup_s": setup_s, "bvh": dict(trk.bvh_info),
            "adjoint": adjoint, "events": events, "spectral": spectral, "calibration": calibration,
        }
        print(json.dumps({"details": details}), flush=True)
        r3 = lambda v: None if v is None else round(float(v), 4)   # noqa: E731
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(n, world, det.n_tris),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                         "unit": "G lane-ops/s (FP32/INT32)", "frac": achieved / alu_peak,
                         "traffic": None if stale else DRAM_BYTES_PER_PHOTON * n, "stale": stale,
                         "peak_source": f"{N_SM} SMs x {LANES_PER_SM} lanes x sm_max_mhz ({peak_kind})",
                         "ops_per_step": r3(ops_per_step), "kernel_ms": r3(statistics.mean(kern_ms)),
                         "lanes_active": {k: r3(v) for k, v in simd.items()},
                         "issue_frac": None if stale else r3(issue_rate / issue_peak)},
            "e2e": {"value": world * n * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * 1,
            "clocks": clk.summary(),
            "physics": {"lce": r3(float(lce.sum()) / (world * n)), "steps_per_photon": r3(float(fates[7]) / (world * n)),
                        "escaped": int(fates[4]), "geom_err": int(fates[6]), "t90_ns": r3(t90),
                        "t90_nr_profile_ns": r3(t90_nr), "tallies": tallies},
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if events is not None:
            line["events"] = {"photons_per_s": events["photons_per_s"], "ms": r3(events["ms"]),
                              "launch": events["launch"]}
        if spectral is not None:
            line["spectral"] = {"photons_per_s": spectral["photons_per_s"], "cost_ratio": r3(spectral["cost_ratio"])}
        if calibration is not None:
            line["calibration"] = {"pull": [r3(x) for x in calibration["pull"]],
                                   "chi2_4dof": r3(calibration["chi2"]), "launches": calibration["launches"]}
        if adjoint is not None:
            line["adjoint"] = adjoint_summary(adjoint)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
