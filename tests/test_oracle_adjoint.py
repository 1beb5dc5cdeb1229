"""Pins of the oracle's score-function adjoint against closed-form derivatives
of expected detected hits: exponential survival d/dL exp(-R/L), the
derivative of the escape fraction from a uniform source in an absorbing
sphere, the zero derivative with respect to the Rayleigh length when every
photon is detected, and the linear dependence of the detected fraction on an
electrode's transparency and on a mirror's reflectivity."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2203_14354_gb300 import geometry as g


def beam_down_up(n, z, up=True, seed=1, spread=10.0):
    rng = np.random.default_rng(seed)
    p = np.zeros((n, 3), np.float32)
    p[:, 0] = rng.uniform(-spread, spread, n)
    p[:, 1] = rng.uniform(-spread, spread, n)
    p[:, 2] = z
    d = np.zeros((n, 3), np.float32)
    d[:, 2] = 1.0 if up else -1.0
    a = rng.uniform(0, 2 * np.pi, n)
    pol = np.stack([np.cos(a), np.sin(a), np.zeros(n)], 1).astype(np.float32)
    return p, d, pol


def test_adjoint_exponential_survival():
    lam, R, n = 100.0, 100.0, 200_000
    o = O.Oracle(g.icosphere(R, subdiv=5, abs_len_mm=lam))
    o.set_adjoint([0], [])
    res = o.propagate(n, adjoint=True)
    J = o.jacobian(res["adjoint"])
    want = n * R / lam ** 2 * math.exp(-R / lam)
    # detected photons all travelled ~R: J = N_det R / L^2, binomial noise on N_det
    sig = R / lam ** 2 * math.sqrt(n * math.exp(-R / lam) * (1 - math.exp(-R / lam)))
    assert abs(J[0, 0] - want) < 4 * sig + 1e-3 * want
    assert J[0, 1] == 0.0  # no Rayleigh in this medium: no dependence


def test_adjoint_escape_from_ball():
    R, tau, n = 100.0, 1.0, 200_000
    lam = R / tau
    det = g.icosphere(R, subdiv=5, abs_len_mm=lam)
    det.source = g.Source(g.SRC_BALL, 0, radius=R * 0.999)
    o = O.Oracle(det)
    o.set_adjoint([0], [])
    res = o.propagate(n, seed=3, adjoint=True)
    J = o.jacobian(res["adjoint"])[0, 0]
    P = lambda t: 3.0 / (8 * t ** 3) * (2 * t ** 2 - 1 + (1 + 2 * t) * math.exp(-2 * t))
    h = 1e-5
    dP_dtau = (P(tau + h) - P(tau - h)) / (2 * h)
    want = n * dP_dtau * (-R / lam ** 2)  # d tau / d lambda = -R / lambda^2
    # per-photon score l/L^2 with l in [0, 2R]: bound the noise by its range
    sig = math.sqrt(n) * (2 * R / lam ** 2)
    assert abs(J - want) < 4 * sig * 0.5 + 0.01 * abs(want)


def test_adjoint_rayleigh_length_zero_when_all_detected():
    L, R, n = 80.0, 100.0, 100_000
    o = O.Oracle(g.icosphere(R, subdiv=5, ray_len_mm=L))
    o.set_adjoint([0], [])
    res = o.propagate(n, seed=5, adjoint=True)
    assert res["det"][0] == n
    J = o.jacobian(res["adjoint"])[0, 1]
    scatters = res["adjoint"][0, 1]
    # E[N_scatter] = E[path] / L (Poisson process): the score l/L^2 - N/L has mean 0
    assert abs(J) < 5 * math.sqrt(scatters) / L
    assert scatters > 0.5 * n


def test_adjoint_electrode_transparency():
    T, Rw, n = 0.9, 0.3, 200_000
    o = O.Oracle(g.electrode_box(T, Rw))
    o.set_adjoint([], [2])
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, 0), explicit=beam_down_up(n, -50.0), adjoint=True)
    J = o.jacobian(res["adjoint"])
    # top = N T exactly in expectation -> d top / dT = N; J_top = N_top / T
    assert abs(J[1, 0] - n) < 4 * math.sqrt(n * T * (1 - T)) / T
    # bottom photons were wire-reflected once: d bottom / dT = -bottom / (1 - T)
    assert J[0, 0] == pytest.approx(-float(res["det"][0]) / (1 - T), rel=1e-12)
    assert res["det"][0] > 0


def test_adjoint_mirror_reflectivity():
    R, n = 0.8, 200_000
    o = O.Oracle(g.reflector_box(R, 1.0))
    o.set_adjoint([], [1])
    res = o.propagate(n, src=g.Source(g.SRC_EXPLICIT, 0), explicit=beam_down_up(n, 0.0, up=False), adjoint=True)
    J = o.jacobian(res["adjoint"])[0, 0]
    # every detected photon reflected once off the floor: E[top] = N R, d/dR = N
    assert res["det"][0] / n == pytest.approx(R, abs=4 * math.sqrt(R * (1 - R) / n))
    assert abs(J - n) < 4 * math.sqrt(n * R * (1 - R)) / R
