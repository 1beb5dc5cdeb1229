"""Pins of the oracle's scintillation time profile (Sec. 2.2, Table 2: two
exponential components) and of the t90 summary: the emission delays follow
the two-exponential mixture CDF, their mean is f tau_s + (1 - f) tau_t, a
singlet fraction of 1 (or 0) gives a single exponential, no profile leaves
every photon at t0, and t90 of an exponential arrival distribution is
tau ln 10."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2203_14354_gb300 import analysis
from paper_2203_14354_gb300 import geometry as g


@pytest.fixture(scope="module")
def orc():
    return O.Oracle(g.icosphere(100.0, subdiv=2))


def delays(orc, src, n=40_000, seed=3):
    return orc.sample_source(n, seed=seed, src=src, time=True)[4] - src.t0


def test_no_profile_starts_at_t0(orc):
    src = g.Source(g.SRC_POINT, 0, t0=7.25)
    assert np.all(delays(orc, src, 2000) == 0.0)


def test_nr_profile_mixture_cdf(orc):
    f, ts, tt = g.NR_PROFILE
    src = g.Source(g.SRC_POINT, 0, t0=1.5).with_profile(g.NR_PROFILE)
    d = delays(orc, src)
    cdf = lambda t: f * (1 - np.exp(-t / ts)) + (1 - f) * (1 - np.exp(-t / tt))
    assert stats.kstest(d, cdf).pvalue > 1e-3
    mean = f * ts + (1 - f) * tt  # 10.47 ns
    assert abs(d.mean() - mean) < 4 * math.sqrt(f * 2 * ts ** 2 + (1 - f) * 2 * tt ** 2 - mean ** 2) / math.sqrt(d.size)
    # ER light is slower: more triplet
    de = delays(orc, g.Source(g.SRC_POINT, 0).with_profile(g.ER_PROFILE))
    assert de.mean() > d.mean() + 5.0


@pytest.mark.parametrize("frac", [0.0, 1.0])
def test_single_component(orc, frac):
    src = g.Source(g.SRC_POINT, 0).with_profile((frac, 3.5, 24.0))
    tau = 3.5 if frac == 1.0 else 24.0
    d = delays(orc, src, 20_000)
    assert stats.kstest(d, stats.expon(scale=tau).cdf).pvalue > 1e-3


def test_profile_does_not_change_positions_or_directions(orc):
    src = g.Source(g.SRC_BALL, 0, center=(1.0, 2.0, 3.0), radius=20.0)
    a = orc.sample_source(3000, seed=4, src=src)
    b = orc.sample_source(3000, seed=4, src=src.with_profile(g.NR_PROFILE))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_t90_closed_forms():
    tau, tb, B = 20.0, 0.5, 4000
    edges = np.arange(B + 1) * tb
    h = np.zeros(B + 1)
    h[:B] = np.exp(-edges[:-1] / tau) - np.exp(-edges[1:] / tau)
    h[B] = math.exp(-edges[-1] / tau)
    # exact: the cumulative is linear within each bin only approximately; 1 % of a bin
    assert analysis.t90(h * 1e6, tb) == pytest.approx(tau * math.log(10.0), abs=0.01 * tb + 1e-9)
    assert analysis.t90(h * 1e6, tb, frac=0.5) == pytest.approx(tau * math.log(2.0), abs=0.01 * tb + 1e-9)
    # uniform arrivals over [0, 100): t90 = 90
    u = np.zeros(201); u[:200] = 1.0
    assert analysis.t90(u, 0.5) == pytest.approx(90.0)
    # leading axes are summed; the overflow counts in the total
    assert analysis.t90(np.stack([u, u]), 0.5) == pytest.approx(90.0)
    o = u.copy(); o[200] = 100.0
    assert analysis.t90(o, 0.5) == float("inf")
    assert math.isnan(analysis.t90(np.zeros(11)))
