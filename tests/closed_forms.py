"""Closed forms of polarised beams in layered set-ups, for the pins of the
oracle and the GPU tests alike.  Nothing here comes from either
implementation: the Fresnel amplitudes are solved from Maxwell's boundary
conditions, and the reflection series are summed exactly over the few paths
a beam can take between parallel interfaces.

Parallel interfaces share one plane of incidence, so a photon's
polarisation is fixed by its s fraction f = (eps . s)^2 alone: at an
interface it reflects with probability f R_s + (1 - f) R_p, and the branch
taken rescales the s and p amplitudes by (r_s, r_p) or (t_s, t_p) (the
coherent reading of the outgoing polarisation, Sec. 2.2).  A specular
mirror keeps f: the tangential field flips sign and the normal field is
kept, which preserves the modulus of both components."""
import math

import numpy as np

from paper_2203_14354_gb300 import geometry as g


def fresnel_bc(n1, n2, theta_deg):
    """r and t of the s and p waves at incidence theta from n1 into n2, from
    the continuity of the tangential components of E and H = n k x E across
    the interface (Born & Wolf, Sec. 1.5.1), solved as one linear system per
    polarisation.  p basis vectors are s x k of each wave.  Plane of
    incidence x-z, interface z = 0, incidence from z < 0.  Returns None past
    the critical angle."""
    th = math.radians(theta_deg)
    st = n1 / n2 * math.sin(th)
    if st >= 1.0:
        return None
    tt = math.asin(st)
    k = np.array([math.sin(th), 0.0, math.cos(th)])
    kr = np.array([math.sin(th), 0.0, -math.cos(th)])
    kt = np.array([math.sin(tt), 0.0, math.cos(tt)])
    s = np.array([0.0, -1.0, 0.0])
    out = {}
    for name, e_i, e_r, e_t in (("s", s, s, s), ("p", np.cross(s, k), np.cross(s, kr), np.cross(s, kt))):
        rows, rhs = [], []
        for comp in (0, 1):   # tangential x and y of E, then of H
            rows.append([e_r[comp], -e_t[comp]])
            rhs.append(-e_i[comp])
            rows.append([n1 * np.cross(kr, e_r)[comp], -n2 * np.cross(kt, e_t)[comp]])
            rhs.append(-n1 * np.cross(k, e_i)[comp])
        A, b = np.array(rows), np.array(rhs)
        sol, *_ = np.linalg.lstsq(A, b, rcond=None)
        assert np.allclose(A @ sol, b, atol=1e-12)
        out["r" + name], out["t" + name] = float(sol[0]), float(sol[1])
    return out


def refraction_angle(n1, n2, theta_deg):
    return math.degrees(math.asin(n1 / n2 * math.sin(math.radians(theta_deg))))


def _reflectance(f, c):
    return 1.0 if c is None else f * c["rs"] ** 2 + (1 - f) * c["rp"] ** 2


def _after(f, a_s, a_p):
    """s fraction after a branch that scales the amplitudes by (a_s, a_p)"""
    w = f * a_s ** 2 + (1 - f) * a_p ** 2
    return f * a_s ** 2 / w


def _reflected(f, c):
    return f if c is None else _after(f, c["rs"], c["rp"])


def _transmitted(f, c):
    return _after(f, c["ts"], c["tp"])


def top_fraction(n_lxe, n_gxe, n_q, theta_lxe_deg, f0, first="liquid", mirror_floor=None, tol=1e-13):
    """Fraction of a beam reaching the photocathode behind the quartz window
    of the layered set-up (LXe | liquid surface | GXe gap | quartz | top
    photocathode).  The beam starts in the LXe at angle theta_lxe from the
    vertical with s fraction f0, heading up (first = "liquid") or, with a
    specular mirror of reflectivity mirror_floor as the floor, down to the
    mirror (first = "mirror").  Without the mirror, light going down in the
    LXe ends on the bottom photocathode.  Sum over all paths until the
    remaining weight is below tol."""
    th_g = refraction_angle(n_lxe, n_gxe, theta_lxe_deg)
    up_liq = fresnel_bc(n_lxe, n_gxe, theta_lxe_deg)      # liquid surface from below
    down_liq = fresnel_bc(n_gxe, n_lxe, th_g)             # liquid surface from above
    up_q = fresnel_bc(n_gxe, n_q, th_g)                   # window from the gas
    top = 0.0
    # states: (where, weight, s fraction); where in {"liq_up", "q_up", "liq_down", "mirror"}
    stack = [("mirror" if first == "mirror" else "liq_up", 1.0, f0)]
    while stack:
        where, w, f = stack.pop()
        if w < tol:
            continue
        if where == "mirror":
            if mirror_floor is not None:
                stack.append(("liq_up", w * mirror_floor, f))
        elif where == "liq_up":
            r = _reflectance(f, up_liq)
            stack.append(("mirror", w * r, _reflected(f, up_liq)))
            if up_liq is not None:
                stack.append(("q_up", w * (1 - r), _transmitted(f, up_liq)))
        elif where == "q_up":
            r = _reflectance(f, up_q)
            top += w * (1 - r)
            stack.append(("liq_down", w * r, _reflected(f, up_q)))
        else:  # liq_down
            r = _reflectance(f, down_liq)
            stack.append(("q_up", w * r, _reflected(f, down_liq)))
            stack.append(("mirror", w * (1 - r), _transmitted(f, down_liq)))
    return top


def oblique_beam(n, theta_deg, psi, z0, up=True, spread=150.0, seed=3):
    """n photons at z0 with x, y uniform in +-spread, direction at theta from
    the vertical in the x-z plane (upwards or downwards), linear
    polarisation at angle psi from the s axis (y) towards p = s x k."""
    rng = np.random.default_rng(seed)
    p = np.zeros((n, 3), np.float32)
    p[:, 0] = rng.uniform(-spread, spread, n)
    p[:, 1] = rng.uniform(-spread, spread, n)
    p[:, 2] = z0
    th = math.radians(theta_deg)
    k = np.array([math.sin(th), 0.0, math.cos(th) if up else -math.cos(th)])
    s = np.array([0.0, 1.0, 0.0])
    pv = np.cross(s, k)
    pol = math.cos(psi) * s + math.sin(psi) * pv
    return p, np.tile(k.astype(np.float32), (n, 1)), np.tile(pol.astype(np.float32), (n, 1))


def mirror_floor_box(reflectivity=0.5, half=20000.0):
    """The layered set-up of the Sec. 3 worked examples with its bottom
    photocathode turned into a specular mirror (all reflections specular;
    the rest absorbed, so that light sent back down by the liquid surface
    is partly lost), and side walls far enough away that a beam bouncing
    between the floor and the liquid surface never reaches them."""
    det = g.layered_box(half=half)
    surfs = list(det.surfaces) + [g.Surface("mirror", g.REFLECTOR, reflectivity=reflectivity,
                                                     spec_frac=1.0)]
    surface = det.surface.copy()
    channel = det.channel.copy()
    floor = det.channel == 0
    surface[floor] = len(surfs) - 1
    channel[floor] = -1
    from dataclasses import replace
    return replace(det, surface=surface, channel=channel, surfaces=surfs)
