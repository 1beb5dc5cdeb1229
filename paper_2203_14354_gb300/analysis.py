"""Host-side summaries of the tracker's tallies (Sec. 3 and 4 of the paper):
light-collection efficiency and t90, the time by which 90 % of the detected
photons have arrived."""
from __future__ import annotations

import numpy as np


def t90(hist, tbin_ns=1.0, frac=0.9):
    """Time (ns) by which `frac` of the detected photons arrived, from arrival
    histograms [..., B + 1] (bin B = overflow) summed over all leading axes;
    linear within the bin where the cumulative count crosses frac x total.
    inf if the crossing lies in the overflow bin, nan if nothing was
    detected."""
    h = np.asarray(hist, dtype=np.float64)
    h = h.reshape(-1, h.shape[-1]).sum(0)
    total = h.sum()
    if total <= 0:
        return float("nan")
    need = frac * total
    c = np.cumsum(h[:-1])
    k = int(np.searchsorted(c, need, side="left"))
    if k >= h.shape[0] - 1:
        return float("inf")
    below = c[k - 1] if k > 0 else 0.0
    return (k + (need - below) / h[k]) * tbin_ns


def lce(det_or_lce, n_photons):
    """Fraction of the photons counted over all channels."""
    return float(np.asarray(det_or_lce, dtype=np.float64).sum()) / float(n_photons)


def loss_table(det, fates, n):
    """Where the photons that never reached a photocathode ended (Sec. 4.2,
    sources of photon losses), in % of the n photons: bulk absorption per
    medium, each electrode (wires, frames listed apart), PMT caps (photons
    that entered a window but missed the photocathode), PTFE and the rest.
    fates: the fate counters [8 + M + S]."""
    f = np.asarray(fates, dtype=np.float64)
    M = len(det.materials)
    out = {"lce": 100.0 * (f[0] + f[1]) / n}
    for m, mat in enumerate(det.materials):
        if f[8 + m]:
            out[mat.name] = 100.0 * f[8 + m] / n
    electrodes, frames, ptfe, caps, other = 0.0, 0.0, 0.0, 0.0, 0.0
    per = {}
    for k, sf in enumerate(det.surfaces):
        v = 100.0 * f[8 + M + k] / n
        if not v:
            continue
        name = sf.name
        if name.endswith("_frame"):
            frames += v
            per[name] = v
        elif name.endswith("_SS") or name.endswith("_AlMgF2") or name.endswith("_T"):
            electrodes += v
            per[name] = v
        elif name.startswith("PTFE"):
            ptfe += v
        elif name.startswith("PMT_cap"):
            caps += v
        else:
            other += v
    out.update(electrodes=electrodes + frames, electrode_parts=per, frames=frames, pmt_caps=caps, ptfe=ptfe,
               other_surfaces=other, escaped=100.0 * f[4] / n, truncated=100.0 * f[5] / n)
    out["not_detected"] = 100.0 - out["lce"]
    return out
