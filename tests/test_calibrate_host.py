"""Host logic of the calibration fit on a CPU stand-in for the tracker whose
expected hits are a known smooth function of the four parameters: the
unconstrained transforms invert each other, the deviance is zero at the
target and its gradient is the Poisson score, and Adam through the autograd
Function recovers the hidden parameters from noise-free and from noisy hit
maps, the cross-fitted Fisher information stays unbiased when the
per-cell Jacobians are noisy, and the deviation statistics of an estimate
(pulls, chi^2 with the full covariance, eigen-deviations) match a worked
example."""
import math

import pytest
import torch

from paper_2203_14354_gb300 import calibrate as cal
from paper_2203_14354_gb300 import geometry as g


class _FakeTracker:
    """Mean hits mu[e, c] = n_e * w * exp(-d / L_abs) * (1 - s exp(-L_ray / r))
    * (1 + a R_l / (1 - R_l)) * (1 + b R_g), cells differing in d, r, a, b so
    that all four parameters are identifiable."""

    adj_mats, adj_surfs = [0], [0, 1]
    device = torch.device("cpu")

    def __init__(self, n_events=12, n_chan=9, seed=0):
        gen = torch.Generator().manual_seed(seed)
        E, P = n_events, n_chan
        self.n_channels = P
        self.w = 1e-3 * (0.5 + torch.rand(E, P, generator=gen, dtype=torch.float64))
        self.d = 500.0 + 4000.0 * torch.rand(E, P, generator=gen, dtype=torch.float64)
        self.r = 100.0 + 400.0 * torch.rand(E, P, generator=gen, dtype=torch.float64)
        self.s = 0.2 + 0.6 * torch.rand(E, P, generator=gen, dtype=torch.float64)
        self.a = 0.02 * torch.rand(E, P, generator=gen, dtype=torch.float64)
        self.b = torch.rand(E, P, generator=gen, dtype=torch.float64)
        self._theta = torch.tensor([50_000.0, 400.0, 0.95, 0.70], dtype=torch.float64)
        self.n = None
        self.launches = 0

    def theta(self):
        return self._theta.clone()

    def set_theta(self, th):
        self._theta = torch.as_tensor(th, dtype=torch.float64).detach().clone()

    def upload_events(self, events):
        self.n = torch.tensor([n for _, n in events], dtype=torch.float64)

    def mean_hits(self, th):
        # an event list uploaded k times repeats the cells of the first copy
        La, Lr, Rl, Rg = th
        k = self.n.shape[0] // self.w.shape[0]
        w, d, r, s, a, b = (x.repeat(k, 1) for x in (self.w, self.d, self.r, self.s, self.a, self.b))
        return (self.n[:, None] * w * torch.exp(-d / La) * (1 - s * torch.exp(-Lr / r))
                * (1 + a * Rl / (1 - Rl)) * (1 + b * Rg))

    def propagate_events(self, seed=0, hist=False, adjoint=False, **kw):
        self.launches += 1
        out = dict(det=self.mean_hits(self._theta))
        if adjoint:
            out["adjoint"] = torch.zeros(out["det"].shape + (8,), dtype=torch.float64)
        return out

    def jacobian(self, sums, g=None):
        J = torch.autograd.functional.jacobian(self.mean_hits, self._theta)  # [E, P, 4]
        return J if g is None else (J, (J * g[..., None]).sum((0, 1)))

    def sync(self):
        pass


def test_transforms_round_trip():
    kinds = [cal.LENGTH, cal.LENGTH, cal.FRACTION, cal.FRACTION]
    th = torch.tensor([30_000.0, 350.0, 0.97, 0.8], dtype=torch.float64)
    u = cal.to_unconstrained(th, kinds)
    assert u[0] == pytest.approx(math.log(30_000.0))
    assert u[2] == pytest.approx(math.log(0.97 / 0.03))
    torch.testing.assert_close(cal.from_unconstrained(u, kinds), th, rtol=1e-14, atol=0)


def test_deviance_zero_at_target_and_score():
    k = torch.tensor([[0.0, 3.0, 10.0]], dtype=torch.float64)
    assert float(cal.poisson_deviance(k.clamp(min=1e-3), k)) == pytest.approx(2e-3, abs=1e-12)
    mu = torch.tensor([[1.5, 2.0, 12.0]], dtype=torch.float64, requires_grad=True)
    cal.poisson_deviance(mu, k).backward()
    # d/dmu 2 (mu - k log mu) = 2 (1 - k / mu)
    torch.testing.assert_close(mu.grad, 2 * (1 - k / mu.detach()))
    # the deviance equals -2 log-likelihood ratio against the saturated model
    ll = lambda m: (k * torch.log(m.clamp(min=1e-300)) - m - torch.lgamma(k + 1)).sum()
    sat = ll(torch.where(k > 0, k, torch.full_like(k, 1e-300)))
    assert float(cal.poisson_deviance(mu.detach(), k)) == pytest.approx(float(2 * (sat - ll(mu.detach()))), rel=1e-12)


def test_calibration_recovers_hidden_parameters(monkeypatch):
    from paper_2203_14354_gb300 import tracker as T

    class _EventFn(torch.autograd.Function):
        # the library's EventLightCollection with the fake in place of the GPU
        forward = staticmethod(T.EventLightCollection.forward)
        backward = staticmethod(T.EventLightCollection.backward)

    trk = _FakeTracker()
    events = g.calibration_sources(20_000_000, n_x=4, n_z=3, spacing=100.0)
    truth = torch.tensor([30_000.0, 350.0, 0.97, 0.80], dtype=torch.float64)
    trk.upload_events(events)
    target = trk.mean_hits(truth)
    c = cal.Calibration(trk, events, target, model_scale=2)
    c._fn = _EventFn
    dev0, grad0 = c.loss(trk.theta(), seed=0)
    assert dev0 > 0 and torch.all(torch.isfinite(grad0))
    # the gradient through the adjoint path equals autograd through the model
    th = trk.theta().requires_grad_(True)
    # the model runs every source twice (two halves), each half with the target's photon count
    E = len(events)
    assert trk.n.shape[0] == 2 * E and torch.equal(trk.n[:E], trk.n[E:])
    cal.poisson_deviance(c._mean(trk.mean_hits(th)), target).backward()
    torch.testing.assert_close(grad0, th.grad, rtol=1e-9, atol=0)
    # Fisher information: at zero residual the Hessian of the deviance is 2 F
    F = c.fisher(truth, seed=0)
    H = torch.autograd.functional.hessian(lambda th: cal.poisson_deviance(c._mean(trk.mean_hits(th)), target), truth)
    torch.testing.assert_close(2 * F, H, rtol=1e-7, atol=0)
    launches = trk.launches
    res = c.fit([50_000.0, 400.0, 0.95, 0.70], steps=40, cycle=10)
    # one launch per step, plus one Fisher launch per Adam cycle
    n_adam = 40 - res["scoring_steps"]
    assert trk.launches - launches == 40 + (n_adam + 9) // 10 == res["launches"]
    assert 1 <= res["scoring_steps"] <= 10
    rec = torch.tensor(res["theta"], dtype=torch.float64)
    sigma = c.covariance(rec, seed=0).diagonal().sqrt()
    # noise-free model: the fit lands on the hidden values well inside one standard deviation
    assert torch.all(torch.abs(rec - truth) < 0.1 * sigma), (rec, sigma)
    assert res["history"][-1]["deviance"] < 1e-3 * res["history"][0]["deviance"]


@pytest.mark.parametrize("photons", [20_000_000, 2_000_000_000])
def test_calibration_with_counting_noise(photons):
    """Poisson noise on the target and on every model evaluation (a model
    of twice the photons): the estimate lands within 4 standard deviations
    of the covariance F^-1 (1 + 1/2) on each parameter, also when the start
    is hundreds of standard deviations away (2e9 photons per source)."""
    from paper_2203_14354_gb300 import tracker as T

    class _EventFn(torch.autograd.Function):
        forward = staticmethod(T.EventLightCollection.forward)
        backward = staticmethod(T.EventLightCollection.backward)

    trk = _FakeTracker()
    events = g.calibration_sources(photons, n_x=4, n_z=3, spacing=100.0)
    truth = torch.tensor([30_000.0, 350.0, 0.97, 0.80], dtype=torch.float64)
    trk.upload_events(events)
    target = torch.poisson(trk.mean_hits(truth), generator=torch.Generator().manual_seed(5))
    exact = trk.propagate_events

    def noisy(seed=0, **kw):
        out = exact(seed=seed, **kw)
        out["det"] = torch.poisson(out["det"], generator=torch.Generator().manual_seed(1000 + seed))
        return out

    trk.propagate_events = noisy
    c = cal.Calibration(trk, events, target, model_scale=2)
    c._fn = _EventFn
    res = c.fit([50_000.0, 400.0, 0.95, 0.70])
    rec = torch.tensor(res["theta"], dtype=torch.float64)
    sigma = c.covariance(rec, seed=0).diagonal().sqrt()
    assert torch.all(torch.abs(rec - truth) < 4 * sigma), ((rec - truth) / sigma)


def test_cross_fitted_fisher_is_unbiased_under_noisy_jacobians():
    """Each model row's Jacobian carries independent zero-mean noise far
    larger than its signal (as the Rayleigh-length score does for cells of
    few counts): the Fisher estimate from the product of the two halves
    stays on the exact sum J J^T / mu, while the square of one estimate is
    inflated by the noise covariance."""
    trk = _FakeTracker(n_events=80, n_chan=40)
    events = g.calibration_sources(2_000_000, n_x=10, n_z=8, spacing=50.0)
    truth = torch.tensor([30_000.0, 350.0, 0.97, 0.80], dtype=torch.float64)
    trk.upload_events(events)
    target = trk.mean_hits(truth)
    c = cal.Calibration(trk, events, target, model_scale=2)
    trk.set_theta(truth)
    J = torch.autograd.functional.jacobian(trk.mean_hits, truth)  # [2E, P, 4]
    E = len(events)
    mu = c._mean(trk.mean_hits(truth))
    Jm = J[:E]  # both halves have the same expectation
    exact = torch.einsum("epq,epr->qr", Jm, Jm / mu[..., None])
    scale = Jm.abs().mean((0, 1)) * 2.0
    gen = torch.Generator().manual_seed(3)

    def noisy_jacobian(sums, g=None):
        return J + torch.randn(J.shape, generator=gen, dtype=torch.float64) * scale

    trk.jacobian = noisy_jacobian
    F = c.fisher(truth, seed=0)
    d = exact.diagonal()
    Jn = noisy_jacobian(None)[:E]
    naive = torch.einsum("epq,epr->qr", Jn, Jn / mu[..., None])
    assert torch.all(naive.diagonal() > 3 * d)  # the square of one estimate: noise dominates
    assert torch.all((F.diagonal() - d).abs() < 0.25 * d), (F.diagonal(), d)


def test_deviation_stats_of_a_correlated_estimate():
    """chi^2 = d^T C^-1 d worked by hand for C = [[4, 2], [2, 3]] and
    d = (1, -1): C^-1 = [[3, -2], [-2, 4]] / 8, so chi^2 = (3 + 4 + 4) / 8;
    pulls d_i / sqrt(C_ii); the eigen-deviations square-sum to chi^2; a
    deviation along an eigenvector shows in that component alone."""
    st = cal.deviation_stats([11.0, 19.0], [10.0, 20.0], [[4.0, 2.0], [2.0, 3.0]])
    assert math.isclose(st["chi2"], 11.0 / 8.0, rel_tol=1e-12)
    assert st["pull"] == pytest.approx([0.5, -1.0 / math.sqrt(3.0)], rel=1e-12)
    assert sum(z * z for z in st["z_eigen"]) == pytest.approx(11.0 / 8.0, rel=1e-12)
    assert st["corr"][0][1] == pytest.approx(2.0 / math.sqrt(12.0), rel=1e-12)
    cov = torch.tensor([[4.0, 2.0], [2.0, 3.0]], dtype=torch.float64)
    lam, vec = torch.linalg.eigh(cov)
    d = 2.0 * lam[0].sqrt() * vec[:, 0]   # two standard deviations along the tightest direction
    st = cal.deviation_stats(d, torch.zeros(2, dtype=torch.float64), cov)
    assert st["z_eigen"] == pytest.approx([2.0, 0.0], abs=1e-12)
    assert st["chi2"] == pytest.approx(4.0, rel=1e-12)
