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
