"""Gradient-based calibration of optical parameters from per-PMT hit maps.

The paper studies how the light collection depends on the LXe absorption
length, the Rayleigh length and the PTFE reflectivity one parameter at a time
(Sec. 3, the LCE systematics table).  Here the same dependence is used the
other way round: given measured hit maps k[e, c] of a set of calibration
sources e in PMTs c, find the parameters theta whose expected hits mu[e, c]
fit them best.

* Model: mu[e, c](theta) is the mean detected-hit count, estimated by one
  batched launch of ``model_scale`` times the sources' photon counts (as two
  independent halves) divided by ``model_scale``; its gradient comes from the
  score-function adjoint of the tracker (``EventLightCollection``).
* Objective: the Poisson deviance 2 sum (mu - k + k log(k / mu)), which is
  minus twice the Poisson log-likelihood up to a theta-independent constant.
* Optimiser: a Fisher-scoring warm start, then Adam (Kingma & Ba, 2015)
  through the autograd adjoint, both on unconstrained coordinates u (log L
  for lengths, logit R for reflectivities / transparencies) and both using
  the Poisson Fisher information F = sum_cells J J^T / mu from the adjoint's
  Jacobian rows.  Absorption length and PTFE reflectivity both scale the
  total light, so in u the deviance is a long, curved, narrow valley where
  per-coordinate step sizes crawl; whitened, z = F^(1/2) (u - u_c), its
  Hessian is about 2 I and one unit of z is one standard deviation of the
  estimate.  Fresh random numbers every launch; the mean of the last
  ``average_last`` iterates (Polyak averaging) is the estimate.
* Uncertainty: the covariance of the fit is F^-1 (1 + 1/model_scale) (target
  counts plus model noise), evaluated at the estimate.

Everything here is host-side orchestration: each model evaluation is one
launch of the propagation kernel plus the Jacobian kernel of the library.
"""
from __future__ import annotations

import time

import torch

LENGTH, FRACTION = 0, 1


def param_kinds(tracker):
    """LENGTH for the (L_abs, L_ray) pair of each tracked material, FRACTION
    for each tracked surface (reflectivity or transparency)."""
    return [LENGTH] * (2 * len(tracker.adj_mats)) + [FRACTION] * len(tracker.adj_surfs)


def to_unconstrained(theta, kinds):
    theta = torch.as_tensor(theta, dtype=torch.float64)
    return torch.stack([torch.log(t) if k == LENGTH else torch.log(t / (1.0 - t)) for t, k in zip(theta, kinds)])


def from_unconstrained(u, kinds):
    return torch.stack([torch.exp(x) if k == LENGTH else torch.sigmoid(x) for x, k in zip(u, kinds)])


def poisson_deviance(mu, k, floor=1e-3):
    """2 sum(mu - k + k log(k / mu)) over all (event, PMT) cells; mu is
    clamped below at ``floor`` so a cell the model left empty stays finite."""
    mu = mu.clamp(min=floor)
    k = k.to(mu.dtype)
    klog = torch.where(k > 0, k * torch.log(k.clamp(min=1e-300) / mu), torch.zeros_like(k))
    return 2.0 * (mu - k + klog).sum()


def deviation_stats(theta, truth, cov):
    """How far an estimate lies from the truth under its covariance:
    pulls (per parameter, in its own standard deviation), the chi^2 of the
    whole deviation d^T C^-1 d (the parameters are correlated), the
    deviation along the covariance's eigenvectors in their own standard
    deviations (tightest first; their squares sum to chi^2) and the
    correlation matrix."""
    theta = torch.as_tensor(theta, dtype=torch.float64)
    truth = torch.as_tensor(truth, dtype=torch.float64)
    cov = torch.as_tensor(cov, dtype=torch.float64)
    d = theta - truth
    sigma = cov.diagonal().sqrt()
    lam, vec = torch.linalg.eigh(cov)
    return dict(pull=(d / sigma).tolist(), chi2=float(d @ torch.linalg.solve(cov, d)),
                z_eigen=((vec.T @ d) / lam.sqrt()).tolist(),
                corr=(cov / (sigma[:, None] * sigma[None, :])).tolist())


def hit_maps(tracker, theta, seed):
    """Detected hits [E, P] of the tracker's uploaded events at theta (no
    gradient)."""
    tracker.set_theta(theta)
    return tracker.propagate_events(seed=seed, hist=False)["det"].to(torch.float64)


class Calibration:
    """Fit of the tracker's tracked parameters (``Tracker.set_adjoint``) to
    target hit maps [E, P] of ``events`` (list of (Source, n_photons))."""

    def __init__(self, tracker, events, target, model_scale=2):
        from .tracker import EventLightCollection

        self._fn = EventLightCollection
        self.tracker = tracker
        self.kinds = param_kinds(tracker)
        self.scale = int(model_scale)
        self.n_events = len(events)
        # every source is uploaded twice, as two independent halves A (rows
        # 0..E-1) and B (rows E..2E-1) of model_scale times its photons
        half = [max(1, (int(n) * self.scale + 1) // 2) for _, n in events]
        tracker.upload_events([(src, h) for (src, _), h in zip(events, half)] * 2)
        n = torch.tensor([max(1, int(n)) for _, n in events], dtype=torch.float64, device=tracker.device)
        # model counts of one half x per_half = an estimate for the target's photon count
        self.per_half = (n / torch.tensor(half, dtype=torch.float64, device=tracker.device))[:, None]
        self.target = torch.as_tensor(target, dtype=torch.float64, device=tracker.device)
        if self.target.shape != (len(events), tracker.n_channels):
            raise ValueError(f"target shape {tuple(self.target.shape)} != ({len(events)}, {tracker.n_channels})")

    def _mean(self, det):
        """Expected hits [E, P] from the two halves' counts [2E, P]."""
        E = self.n_events
        return (det[:E] + det[E:]) * (0.5 * self.per_half)

    def loss(self, theta, seed):
        """Deviance at theta and its gradient with respect to theta."""
        th = torch.as_tensor(theta, dtype=torch.float64).detach().clone().requires_grad_(True)
        mu = self._mean(self._fn.apply(th, self.tracker, seed))
        dev = poisson_deviance(mu, self.target)
        dev.backward()
        return float(dev.detach()), th.grad.detach().cpu()

    def scoring_step(self, theta, seed):
        """One model launch with adjoint tallies at theta: deviance, its
        gradient [Q] and the Fisher information sum_cells J J^T / mu [Q, Q]
        (theta coordinates) of the target-sized experiment.  J J^T is
        estimated by the product of the two halves' independent Jacobians,
        J_A J_B^T: the product of one estimate with itself would add its
        covariance, which dominates for cells of few counts and noisy scores
        (the Rayleigh-length score of a photon that scattered ten times)."""
        trk = self.tracker
        trk.set_theta(theta)
        out = trk.propagate_events(seed=seed, hist=False, adjoint=True)
        E = self.n_events
        J = trk.jacobian(out["adjoint"])
        JA, JB = J[:E] * self.per_half[..., None], J[E:] * self.per_half[..., None]
        det = out["det"].to(torch.float64)
        mu = self._mean(det)
        dev = float(poisson_deviance(mu, self.target))
        keep = mu > 0
        JA, JB, mk, kk = JA[keep], JB[keep], mu[keep], self.target[keep]
        grad = ((JA + JB) * (1.0 - kk / mk)[:, None]).sum(0)  # 2 (1 - k/mu) times the mean of the halves
        F = JA.T @ (JB / mk[:, None])
        return dev, grad.cpu(), (0.5 * (F + F.T)).cpu()

    def fisher(self, theta, seed):
        """Fisher information [Q, Q] at theta (one model launch)."""
        return self.scoring_step(theta, seed)[2]

    def covariance(self, theta, seed):
        """Covariance of the fitted theta: F^-1 (1 + 1/model_scale)."""
        return torch.linalg.inv(self.fisher(theta, seed)) * (1.0 + 1.0 / self.scale)

    def _dtheta_du(self, theta):
        return torch.stack([t if k == LENGTH else t * (1.0 - t) for t, k in zip(theta, self.kinds)])

    def fit(self, theta0, steps=40, scoring_steps=10, scoring_tol=3.0, cycle=10, lr_scale=0.5, lr_final=0.05,
            average_last=10, seed=1000, max_du=0.3, betas=(0.5, 0.9), log=None):
        """Two phases over ``steps`` model launches (plus one Fisher launch per
        Adam cycle).

        1. Warm start by Fisher scoring (Gauss-Newton for the Poisson
           likelihood): u <- u - F_u^-1 grad_u / 2, each step shrunk so that no
           unconstrained coordinate moves by more than ``max_du``, until the
           step is within ``scoring_tol`` standard deviations or after
           ``scoring_steps`` launches.  A per-coordinate optimiser alone
           crawls here: absorption length and PTFE reflectivities are nearly
           degenerate, and the start can be hundreds of standard deviations
           from the minimum.
        2. Adam through the autograd adjoint, in cycles of ``cycle`` steps.
           Each cycle whitens by the Fisher information at its start,
           z = F^(1/2) (u - u_c), restarts Adam's moments, and lowers the step
           size linearly from lr0 to lr_final.  lr0 (z units, one unit = one
           standard deviation) is ``lr_scale`` times the largest component of
           the step to the minimum that the cycle's first gradient implies
           (the Hessian of the deviance in z is about 2 I), shrunk until that
           step changes no unconstrained coordinate by more than ``max_du``;
           each Adam step is shrunk the same way.

        The estimate is the mean of the last ``average_last`` iterates
        (Polyak averaging); every launch draws fresh random numbers."""
        theta0 = torch.as_tensor(theta0, dtype=torch.float64).cpu()
        u = to_unconstrained(theta0, self.kinds)
        history, tail = [], []
        t0 = time.perf_counter()
        launches = 0
        it = 0
        while it < min(scoring_steps, steps):
            theta = from_unconstrained(u, self.kinds)
            D = self._dtheta_du(theta)
            dev, grad, F = self.scoring_step(theta, seed + it)
            launches += 1
            Fu = D[:, None] * F * D[None, :]
            du = -torch.linalg.solve(Fu, grad * D) / 2.0
            z_len = float(torch.sqrt(du @ Fu @ du))  # length of the step in standard deviations
            u = u + du * min(1.0, max_du / float(du.abs().max()))
            rec = dict(it=it, phase="scoring", deviance=dev, theta=[float(x) for x in theta], step_sigma=z_len)
            history.append(rec)
            if log:
                log(rec)
            it += 1
            if it >= steps - average_last:
                tail.append(u.clone())
            if z_len < scoring_tol:
                break
        k0 = it
        for it in range(k0, steps):
            if (it - k0) % cycle == 0:
                th_c = from_unconstrained(u, self.kinds)
                D = self._dtheta_du(th_c)
                Fu = D[:, None] * self.fisher(th_c, seed + 100_000 + it) * D[None, :]
                launches += 1
                lam, V = torch.linalg.eigh(Fu)
                lam = lam.clamp(min=1e-12 * float(lam.max()))
                S = V @ torch.diag(lam.rsqrt()) @ V.T  # u = u_c + S z
                u_c = u.clone()
                z = torch.zeros_like(u, requires_grad=True)
                opt = torch.optim.Adam([z], lr=1.0, betas=betas)
                lr0, c0 = None, it
            opt.zero_grad()
            theta = from_unconstrained(u_c + S @ z, self.kinds)
            dev, g_theta = self.loss(theta.detach(), seed + it)
            launches += 1
            theta.backward(g_theta)  # chain rule through the transform and the whitening
            if lr0 is None:
                # the quadratic model's minimum is z* = -g / 2; shrink it until its
                # u step is within max_du (a trust region: the model is local)
                z_star = -z.grad / 2.0
                shrink = min(1.0, max_du / max(float((S @ z_star).abs().max()), 1e-300))
                lr0 = max(lr_scale * float(z_star.abs().max()) * shrink, lr_final)
            for gparam in opt.param_groups:
                gparam["lr"] = lr_final + (lr0 - lr_final) * (1.0 - (it - c0) / cycle)
            z_old = z.detach().clone()
            opt.step()
            du = S @ (z.detach() - z_old)
            shrink = min(1.0, max_du / max(float(du.abs().max()), 1e-300))
            if shrink < 1.0:  # no step changes an unconstrained coordinate by more than max_du
                with torch.no_grad():
                    z.copy_(z_old + shrink * (z - z_old))
            u = (u_c + S @ z).detach()
            rec = dict(it=it, phase="adam", deviance=dev, theta=[float(x) for x in theta.detach()])
            history.append(rec)
            if log:
                log(rec)
            if it >= steps - average_last:
                tail.append(u.clone())
        self.tracker.sync()
        seconds = time.perf_counter() - t0
        u_avg = torch.stack(tail).mean(0) if tail else u
        theta_hat = from_unconstrained(u_avg, self.kinds)
        self.tracker.set_theta(theta_hat)
        return dict(theta=[float(x) for x in theta_hat], history=history, seconds=seconds, steps=steps,
                    scoring_steps=k0, launches=launches)


def main(argv=None):
    """Recover (L_abs, L_ray of the LXe, R of PTFE in LXe and GXe) from the hit
    maps of a grid of point sources generated with hidden values; prints one
    JSON line with the recovered values, the truth, the start and timings."""
    import argparse
    import json

    from . import geometry as g
    from .tracker import Tracker

    ap = argparse.ArgumentParser()
    ap.add_argument("--detector", choices=("darwin", "scaled"), default="darwin")
    ap.add_argument("--photons", type=int, default=1_000_000, help="photons per calibration source")
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--model-scale", type=int, default=2)
    ap.add_argument("--truth", type=float, nargs=4, default=(30_000.0, 350.0, 0.97, 0.80))
    ap.add_argument("--seed", type=int, default=7, help="seed of the source layout and of the target hit maps")
    ap.add_argument("--fit-seed", type=int, default=1000, help="first seed of the model launches of the fit")
    ap.add_argument("--layout", choices=("grid3d", "plane"), default="grid3d",
                    help="sources on a seeded subset of the 3-D grid nodes in the active LXe (default), or on a "
                         "grid in the plane y = 0")
    a = ap.parse_args(argv)
    t_build = time.perf_counter()
    if a.detector == "darwin":
        det = g.darwin()
        events = (g.grid_sources(det, a.photons, 256, spacing=100.0, margin=50.0, seed=a.seed)
                  if a.layout == "grid3d" else g.calibration_sources(a.photons))
    else:
        det = g.scaled_tpc()
        events = (g.grid_sources(det, a.photons, 64, spacing=50.0, margin=50.0, seed=a.seed)
                  if a.layout == "grid3d" else
                  g.calibration_sources(a.photons, n_x=8, n_z=8, spacing=50.0, z_center=-250.0))
    trk = Tracker(det)
    t_build = time.perf_counter() - t_build
    trk.set_adjoint([g.LXE], [0, 1])
    theta0 = trk.theta().tolist()
    # target: one realisation at the hidden values, with its own seed
    trk.upload_events(events)
    target = hit_maps(trk, a.truth, seed=a.seed)
    cal = Calibration(trk, events, target, model_scale=a.model_scale)
    dev_truth, _ = cal.loss(torch.tensor(a.truth, dtype=torch.float64), seed=a.seed + 1)
    res = cal.fit(theta0, steps=a.steps, seed=a.fit_seed)
    dev_fit, _ = cal.loss(torch.tensor(res["theta"], dtype=torch.float64), seed=a.seed + 1)
    cov = cal.covariance(res["theta"], seed=a.seed + 2)
    sigma = cov.diagonal().sqrt().tolist()
    st = deviation_stats(res["theta"], a.truth, cov)
    photons_per_iter = sum(n for _, n in events) * a.model_scale
    print(json.dumps(dict(
        detector=a.detector, layout=a.layout, sources=len(events), photons_per_source=a.photons,
        model_scale=a.model_scale,
        params=["L_abs_LXe_mm", "L_ray_LXe_mm", "R_PTFE_LXe", "R_PTFE_GXe"],
        truth=list(a.truth), start=theta0, recovered=res["theta"],
        rel_error=[(r - t) / t for r, t in zip(res["theta"], a.truth)], sigma=sigma,
        pull=st["pull"], chi2=st["chi2"], z_eigen=st["z_eigen"],
        fit_seed=a.fit_seed,
        deviance_at_truth=dev_truth, deviance_at_fit=dev_fit, cells=int(target.numel()),
        steps=a.steps, scoring_steps=res["scoring_steps"], launches=res["launches"], seconds_fit=res["seconds"],
        seconds_per_launch=res["seconds"] / res["launches"],
        photons_per_step=photons_per_iter, seconds_build=t_build,
        trajectory=[[round(x, 6) for x in h["theta"]] for h in res["history"][:: max(1, a.steps // 12)]])))


if __name__ == "__main__":
    main()
