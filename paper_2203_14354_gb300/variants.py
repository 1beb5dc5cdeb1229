"""Design variants of the DARWIN-scale detector (Sec. 5 of the paper) as
geometry and surface switches, each propagated on the GPU: light-collection
efficiency (photons reaching a photocathode, Sec. 3) in total and per array,
and t90 with the nuclear-recoil scintillation profile.

The paper's printed results are reported beside each variant as context: its
geometry came from CAD (five electrodes of parallel wires, frames, PTFE
around the PMTs), this one is procedural (three hexagonal meshes, flat
plates), so absolute values differ; the direction and rough size of each
change are the comparison.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import analysis
from . import geometry as g

# The paper's own detector layout as far as it is described (Sec. 2.1): five
# planes of parallel wires on frames, and a conical PTFE reflector on each
# PMT window (6 mm high: the paper gives no size)
PAPER_LAYOUT = dict(electrode_kind="wires", pmt_cones=6.0)

# Sec. 5 results at L_abs = 50 m, best-guess optics (LCE %, top, bottom; t90 ns)
PAPER = {
    "baseline": dict(lce=43.1, top=14.8, bottom=28.2, t90=200.0),
    "gate_coated": dict(lce=46.0, top=16.8, bottom=29.2),
    "all_coated": dict(lce=51.8, top=18.6, bottom=33.2),
    "single_phase": dict(lce_change_abs=4.9, t90=175.0),
    "no_bottom_array": dict(lce=18.0, t90=265.0),
    "baseline_abs500m": dict(lce=54.0, top=18.7, bottom=35.3),
    "all_coated_abs500m": dict(lce=67.0, top=24.3, bottom=42.7, t90=240.0),
}
# Sec. 4.2, sources of photon losses (% of photons, baseline)
PAPER_LOSSES = dict(not_detected=56.9, LXe=22.7, electrodes=18.0, gate=7.7, cathode=3.1, screen_bottom=2.6,
                    anode=1.7, screen_top=1.6, frames=1.3, pmt_caps=9.0, ptfe=7.2)


def measure(trk, det, n, seed=0, losses=False):
    """LCE (total, top, bottom) of n photons uniform in the active LXe, and
    t90 (ns) of the detected photons with the nuclear-recoil profile; with
    losses, the loss table."""
    out = trk.propagate(n, seed=seed, source=det.source.with_profile(g.NR_PROFILE), n_tbins=1000, tbin_ns=1.0)
    lce = out["lce"].cpu().numpy().astype(np.float64)
    top = det.pmt_array == 1
    res = dict(lce=100.0 * lce.sum() / n, top=100.0 * lce[top].sum() / n, bottom=100.0 * lce[~top].sum() / n,
               t90=analysis.t90(out["hist"].cpu().numpy(), 1.0),
               escaped=int(out["fates"][4]), geom_err=int(out["fates"][6]))
    if losses:
        res["losses"] = analysis.loss_table(det, out["fates"].cpu().numpy(), n)
    return res


def coated_table(surfaces, coated, r_coat=0.90, coat_spec_frac=0.85 / 0.90):
    """The surface table with the stainless-steel surfaces of the electrodes
    named in `coated` replaced by an Al/MgF2 coating (Sec. 5.1)."""
    out = []
    for sf in surfaces:
        el = sf.name[:-3] if sf.name.endswith("_SS") else None
        out.append(g.Surface(f"{el}_AlMgF2", g.REFLECTOR, r_coat, coat_spec_frac) if el in coated else sf)
    return out


def run(n=10_000_000, electrodes=("gate", "anode", "cathode"), log=print):
    from .tracker import Tracker

    res = {}
    el = tuple(electrodes)
    t0 = time.perf_counter()
    det = g.darwin(electrodes=el, **g.PAPER_OPTICS)
    trk = Tracker(det)
    log(f"baseline mesh: {det.n_tris} triangles, {time.perf_counter() - t0:.0f} s")
    base_surfs = list(det.surfaces)
    opt = g.PAPER_OPTICS
    # coatings and the absorption length change only the tables of the same mesh
    for name, coated, abs_mm in (("baseline", (), 50_000.0), ("gate_coated", ("gate",), 50_000.0),
                                 ("all_coated", el, 50_000.0), ("baseline_abs500m", (), 500_000.0),
                                 ("all_coated_abs500m", el, 500_000.0)):
        det.surfaces = coated_table(base_surfs, coated)
        det.materials = g.default_materials(abs_mm, opt["lxe_ray_mm"], opt["gxe_abs_mm"], opt["gxe_ray_mm"])
        trk.set_surfaces(det.surfaces)
        trk.set_materials(det.materials)
        res[name] = measure(trk, det, n)
        log(f"{name}: {res[name]}")
    trk.close()
    for name, kw in (("single_phase", dict(single_phase=True)), ("no_bottom_array", dict(bottom_array=False))):
        d = g.darwin(electrodes=el, **opt, **kw)
        t = Tracker(d)
        res[name] = measure(t, d, n)
        t.close()
        log(f"{name}: {res[name]}")
    res["single_phase"]["lce_change_abs"] = res["single_phase"]["lce"] - res["baseline"]["lce"]
    # the paper's own electrodes: five planes of parallel wires on frames
    d = g.darwin(**PAPER_LAYOUT, **opt)
    t = Tracker(d)
    res["paper_electrodes"] = measure(t, d, n, losses=True)
    base_surfs = list(d.surfaces)
    d.surfaces = coated_table(base_surfs, ("gate",))
    t.set_surfaces(d.surfaces)
    res["paper_electrodes_gate_coated"] = measure(t, d, n)
    t.close()
    log(f"paper_electrodes: {res['paper_electrodes']}")
    return res


# Sec. 4.1, LCE systematics: one parameter at a time over its spread (LCE %)
PAPER_SYSTEMATICS = dict(L_abs_m=((20.0, 100.0), (32.0, 49.0)), L_ray_cm=((20.0, 50.0), (40.0, 45.0)),
                         R_PTFE_LXe=((0.93, 1.00), (34.0, 45.0)))


def systematics(trk, det, n=10_000_000, seed=0):
    """The paper's one-at-a-time scans (Sec. 4.1) on the uploaded detector:
    average LCE at each end of the spread of L_abs, L_Ray and the PTFE
    reflectivity in LXe, the LCE against L_abs up to 1000 m, and the
    first-order prediction of each end from the adjoint gradient at the
    best-guess values (dLCE/dtheta = dE[detected]/dtheta / (QE n))."""
    import torch

    mats0 = [dataclasses_replace(m) for m in det.materials]
    surfs0 = [dataclasses_replace(sf) for sf in det.surfaces]
    qe = next(sf.qe for sf in det.surfaces if sf.type == g.PHOTOCATHODE)

    def run(mats, surfs):
        trk.set_materials(mats)
        trk.set_surfaces(surfs)
        out = trk.propagate(n, seed=seed, n_tbins=1)
        return 100.0 * float(out["lce"].sum().item()) / n

    def with_lxe(**kw):
        mats = [dataclasses_replace(m) for m in mats0]
        for k, v in kw.items():
            setattr(mats[g.LXE], k, v)
        return mats

    def with_ptfe(r):
        surfs = [dataclasses_replace(sf) for sf in surfs0]
        surfs[0].reflectivity = r
        return surfs

    base = run(mats0, surfs0)
    # gradient at the best-guess point: L_abs, L_ray of LXe and R of PTFE in LXe
    trk.set_materials(mats0)
    trk.set_surfaces(surfs0)
    trk.set_adjoint([g.LXE], [0])
    out = trk.propagate(n, seed=seed, n_tbins=1, adjoint=True)
    grad = (trk.jacobian(out["adjoint"]).sum(0) / (qe * n) * 100.0).cpu().numpy()  # LCE % per unit
    res = {"best_guess_lce": base, "gradient_lce_per_unit": {"L_abs_mm": float(grad[0]),
                                                             "L_ray_mm": float(grad[1]),
                                                             "R_PTFE_LXe": float(grad[2])}}
    th0 = (mats0[g.LXE].abs_len_mm, mats0[g.LXE].rayleigh_len_mm, surfs0[0].reflectivity)
    scans = {}
    for name, (lo, hi), mk, q, scale in (("L_abs_m", (20.0, 100.0), lambda v: (with_lxe(abs_len_mm=v), surfs0), 0, 1e3),
                                         ("L_ray_cm", (20.0, 50.0), lambda v: (with_lxe(rayleigh_len_mm=v), surfs0), 1, 10.0),
                                         ("R_PTFE_LXe", (0.93, 1.00), lambda v: (mats0, with_ptfe(v)), 2, 1.0)):
        ends = []
        for v in (lo, hi):
            ends.append(dict(value=v, lce=run(*mk(v * scale)),
                             first_order=base + float(grad[q]) * (v * scale - th0[q])))
        scans[name] = ends
    res["scans"] = scans
    res["lce_vs_L_abs_m"] = [(L, run(with_lxe(abs_len_mm=L * 1e3), surfs0)) for L in (20, 50, 100, 200, 300, 500, 1000)]
    trk.set_materials(mats0)
    trk.set_surfaces(surfs0)
    return res


def dataclasses_replace(x):
    import dataclasses
    return dataclasses.replace(x)


def lce_map(trk, det, n_z=50, n_r2=50, photons=1_000_000, r_max=1280.0, z_range=(-2597.0, -1.0), seed=0,
            n_tbins=600, profile=g.NR_PROFILE):
    """LCE and t90 on a Z x R^2 grid of isotropic point sources at x = 0
    (Sec. 4.1: close to 2500 positions, 1e6 photons each), all of them in one
    batched launch.  Returns LCE [n_z, n_r2] in %, top and bottom parts, t90
    [n_z, n_r2] in ns, and the grid."""
    import torch

    zs = np.linspace(z_range[0], z_range[1], n_z)
    r2 = (np.arange(n_r2) + 0.5) / n_r2 * r_max ** 2
    ev = [(g.Source(g.SRC_POINT, g.LXE, center=(0.0, float(np.sqrt(q)), float(z))).with_profile(profile), photons)
          for z in zs for q in r2]
    trk.upload_events(ev)
    out = trk.propagate_events(seed=seed, n_tbins=n_tbins, tbin_ns=1.0)
    lce = out["lce"].to(torch.float64)
    top = torch.from_numpy(det.pmt_array == 1).to(lce.device)
    shape = (n_z, n_r2)
    hist = out["hist"].sum(1).cpu().numpy()  # [E, B+1] summed over channels
    del out
    t90 = np.array([analysis.t90(h, 1.0) for h in hist]).reshape(shape)
    return dict(z=zs, r2=r2, lce=(100.0 * lce.sum(1) / photons).cpu().numpy().reshape(shape),
                top=(100.0 * lce[:, top].sum(1) / photons).cpu().numpy().reshape(shape),
                bottom=(100.0 * lce[:, ~top].sum(1) / photons).cpu().numpy().reshape(shape), t90=t90)


def map_summary(m):
    """The features the paper reads off its maps (Sec. 4.1)."""
    lce, top, bot, t90, z, r2 = m["lce"], m["top"], m["bottom"], m["t90"], m["z"], m["r2"]
    prof_top, prof_bot = top.mean(1), bot.mean(1)
    cross = np.nonzero(np.diff(np.sign(prof_top - prof_bot)))[0]
    z_equal = float(np.interp(0.0, (prof_top - prof_bot)[cross[0]:cross[0] + 2], z[cross[0]:cross[0] + 2])) \
        if cross.size else None
    mid = slice(len(z) // 4, 3 * len(z) // 4)
    inner = np.sqrt(m["r2"]) < np.sqrt(r2[-1]) - 20.0
    radial = lce[mid][:, inner]
    return dict(mean_lce=float(lce.mean()), mean_top=float(top.mean()), mean_bottom=float(bot.mean()),
                z_equal_split=z_equal, z_top=float(z[-1]), z_bottom=float(z[0]),
                radial_spread_mid_z=float((radial.max(1) - radial.min(1)).mean()),
                bottom_edge_minus_bottom_centre=float(lce[0, -1] - lce[0, 0]),
                top_edge_minus_top_centre=float(lce[-1, -1] - lce[-1, 0]),
                mean_t90=float(np.mean(t90[np.isfinite(t90)])),
                t90_near_bottom=float(np.mean(t90[0])), t90_middle=float(np.mean(t90[len(z) // 2])),
                t90_near_top=float(np.mean(t90[-1])))


def main(argv=None):
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("--photons", type=float, default=1e7)
    ap.add_argument("--map", action="store_true",
                    help="LCE and t90 maps on a Z x R^2 grid (paper's electrode layout), not the variants")
    ap.add_argument("--map-photons", type=float, default=1e6)
    ap.add_argument("--systematics", action="store_true",
                    help="the paper's one-at-a-time LCE scans (paper's electrode layout), not the variants")
    a = ap.parse_args(argv)
    t0 = time.perf_counter()
    if a.systematics:
        from .tracker import Tracker
        det = g.darwin(**PAPER_LAYOUT, **g.PAPER_OPTICS)
        trk = Tracker(det)
        res = systematics(trk, det, n=int(a.photons))
        print(json.dumps(dict(photons=int(a.photons), ours=res, paper=PAPER_SYSTEMATICS,
                              seconds=time.perf_counter() - t0)))
        return
    if a.map:
        from .tracker import Tracker
        det = g.darwin(**PAPER_LAYOUT, **g.PAPER_OPTICS)
        trk = Tracker(det)
        t1 = time.perf_counter()
        m = lce_map(trk, det, photons=int(a.map_photons))
        trk.sync()
        t_map = time.perf_counter() - t1
        print(json.dumps(dict(sources=int(m["lce"].size), photons_per_source=int(a.map_photons),
                              seconds_map=t_map, summary=map_summary(m),
                              lce_on_axis=[round(float(x), 3) for x in m["lce"][:, 0]],
                              t90_on_axis=[round(float(x), 1) for x in m["t90"][:, 0]])))
        return
    res = run(int(a.photons), log=lambda s: print(s, flush=True))
    print(json.dumps(dict(photons=int(a.photons), optics="paper best guess (Table 2)", ours=res, paper=PAPER,
                          paper_losses=PAPER_LOSSES, seconds=time.perf_counter() - t0)))


if __name__ == "__main__":
    main()
