"""Paired comparison of two runs of the same photons.

The GPU and the oracle draw the same random numbers for a photon, so most
photons end alike on both sides; a photon ends differently only where a
uniform falls within rounding of a decision threshold, and from there on
its two continuations are independent draws of the same process.  For any
outcome c (a fate and its detail: a PMT channel, a material, a surface),
the photons that end in c on one side only are then as likely to be the
GPU's as the oracle's: with a = #(GPU c, oracle not c) and b = #(oracle c,
GPU not c), a ~ Binomial(a + b, 1/2) under parity (a sign test).  A bug
that moves even a small share of outcomes shifts a - b by far more than its
standard deviation sqrt(a + b), although it hides inside the two-sample
binomial band of the unpaired tallies."""
import numpy as np


def outcome(fate, detail):
    """one integer per (fate, detail) pair"""
    return np.asarray(fate, np.int64) * (1 << 32) + (np.asarray(detail, np.int64) + 1)


def sign_test(fate_g, detail_g, fate_o, detail_o, z_max=4.0, min_pairs=1):
    """Sign test of the discordant photons, per outcome.  Returns a dict with
    the share of photons that end alike, the largest |a - b| / sqrt(a + b)
    over the outcomes (with at least min_pairs discordant photons) and the
    outcome where it occurs; asserts it is below z_max."""
    g = outcome(fate_g, detail_g)
    o = outcome(fate_o, detail_o)
    diff = g != o
    cats, a = np.unique(g[diff], return_counts=True)
    cats_o, b = np.unique(o[diff], return_counts=True)
    keys = np.union1d(cats, cats_o)
    A = np.zeros(keys.size)
    B = np.zeros(keys.size)
    A[np.searchsorted(keys, cats)] = a
    B[np.searchsorted(keys, cats_o)] = b
    n = A + B
    ok = n >= min_pairs
    z = np.zeros(keys.size)
    z[ok] = np.abs(A[ok] - B[ok]) / np.sqrt(n[ok])
    worst = int(np.argmax(z)) if z.size else -1
    res = {"same": float(1.0 - diff.mean()), "discordant": int(diff.sum()), "outcomes": int(keys.size),
           "z_max": float(z.max()) if z.size else 0.0,
           "worst": (int(keys[worst] >> 32), int((keys[worst] & 0xFFFFFFFF) - 1), int(A[worst]), int(B[worst]))
           if z.size else None}
    assert res["z_max"] < z_max, res
    return res
