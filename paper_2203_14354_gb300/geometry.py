"""Procedural detector meshes and photon-source descriptions.

This module produces the *inputs* of the photon tracker: a triangle mesh with
per-triangle inner/outer material, surface and PMT channel, the material and
surface tables, the PMT table and a default photon source.  It holds none of
the tracking arithmetic (no sampling, no optics, no intersection) and imports
nothing from the CUDA path, so the CPU oracle's tests and the GPU path both
build their inputs from it.

The DARWIN CAD models are not public, so the detectors are generated from the
description of the paper:

* Sec. 2.1: cylindrical dual-phase TPC, PTFE side wall shaped as an extruded
  24-sided polygon inscribed in a 1300 mm circle, hex-packed 3-inch PMT arrays
  top and bottom, quartz entrance windows with the photocathode behind them and
  a photon-absorbing cap on all other sides, Z layout of Table 1 (photocathodes
  at +69 / -2693 mm, gate 0, liquid surface +2, cathode -2598 mm), electrodes
  as stainless-steel wire meshes.
* Table 2 / Sec. 2.2: refractive indices, absorption and Rayleigh lengths,
  PTFE and stainless-steel reflectivities.

Conventions (shared by every consumer of a mesh):

* Units are mm; vertices are snapped to a 1/4096 mm grid so that every
  coordinate below 4096 mm is exact in float32 and vertices shared by two
  primitives are bitwise identical (watertight seams).
* A triangle's geometric normal is (v1 - v0) x (v2 - v0); it points from
  ``mat_inner`` to ``mat_outer``.
* ``surface == SURF_NONE`` marks a bare dielectric boundary (Fresnel from the
  two refractive indices); otherwise the surface model decides the
  interaction.  ``channel`` is the PMT channel of a photocathode triangle, -1
  elsewhere.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SNAP = 4096.0  # grid 1/4096 mm: 12 fractional bits, exact in float32 below 4096 mm

# material indices used by the generated detectors
LXE, GXE, QUARTZ, OPAQUE = 0, 1, 2, 3

SURF_NONE = 0xFFFF
# surface model types (Sec. 2.2: explicit reflectivity, photocathode, and the
# thin effective-transparency electrode of the Geant4 model, Sec. 2.1)
ABSORBER, REFLECTOR, PHOTOCATHODE, ELECTRODE_T = 0, 1, 2, 3

# photon source kinds
SRC_VOLUME_POLYGON, SRC_POINT, SRC_SEGMENT, SRC_BALL, SRC_EXPLICIT = 0, 1, 2, 3, 4

INF = float("inf")


@dataclass
class Material:
    """Optical constants at 175 nm (the paper's Table 2).  A photon of
    wavelength wl (nm) sees the index n + dn_dlambda_per_nm * (wl - 175) and
    the Rayleigh length rayleigh_len_mm * (wl / 175) ** rayleigh_exp; the
    paper uses the 175 nm values for every photon (both 0)."""
    name: str
    n: float
    abs_len_mm: float = INF
    rayleigh_len_mm: float = INF
    dn_dlambda_per_nm: float = 0.0
    rayleigh_exp: float = 0.0


@dataclass
class Surface:
    name: str
    type: int
    reflectivity: float = 0.0
    spec_frac: float = 0.0
    qe: float = 0.0
    transparency: float = 0.0
    wire_reflectivity: float = 0.0
    wire_spec_frac: float = 0.0


@dataclass
class Source:
    """Where photons start.  Directions are isotropic and polarisations random
    linear for every kind except SRC_EXPLICIT (caller-given arrays)."""
    kind: int
    medium: int = LXE
    n_sides: int = 0          # VOLUME_POLYGON: polygon sides (0 = circle)
    radius: float = 0.0       # VOLUME_POLYGON: circumradius; BALL: radius
    phase: float = 0.0        # VOLUME_POLYGON: angle of vertex 0 (rad)
    z_min: float = 0.0
    z_max: float = 0.0
    center: tuple = (0.0, 0.0, 0.0)   # POINT / BALL centre, SEGMENT start
    p1: tuple = (0.0, 0.0, 0.0)       # SEGMENT end
    t0: float = 0.0
    # scintillation time profile: delay from the singlet component (tau_singlet)
    # with probability singlet_frac, else the triplet one; both 0 = no delay
    singlet_frac: float = 0.0
    tau_singlet_ns: float = 0.0
    tau_triplet_ns: float = 0.0
    # Gaussian emission spectrum: mean (0 = 175 nm) and full width at half
    # maximum (0 = one wavelength), nm
    wl_mean_nm: float = 0.0
    wl_fwhm_nm: float = 0.0

    def with_spectrum(self, spectrum):
        """This source with a Gaussian emission spectrum (mean_nm, fwhm_nm),
        e.g. LXE_SPECTRUM."""
        from dataclasses import replace
        return replace(self, wl_mean_nm=spectrum[0], wl_fwhm_nm=spectrum[1])

    def with_profile(self, profile):
        """This source with a scintillation time profile (singlet_frac,
        tau_singlet_ns, tau_triplet_ns), e.g. NR_PROFILE."""
        from dataclasses import replace
        return replace(self, singlet_frac=profile[0], tau_singlet_ns=profile[1], tau_triplet_ns=profile[2])


# Scintillation time profiles of LXe at 175 nm (Table 2 of the paper): singlet
# fraction, singlet and triplet time constants in ns, for nuclear and
# electronic recoils
NR_PROFILE = (0.66, 3.5, 24.0)
ER_PROFILE = (0.22, 3.5, 24.0)
# LXe scintillation spectrum (Sec. 2.2, Table 2): Gaussian, mean and FWHM in nm
LXE_SPECTRUM = (174.8, 10.2)


@dataclass
class Detector:
    name: str
    verts: np.ndarray        # float32 [nv, 3]
    tris: np.ndarray         # uint32 [nt, 3]
    mat_inner: np.ndarray    # uint8 [nt]
    mat_outer: np.ndarray    # uint8 [nt]
    surface: np.ndarray      # uint16 [nt]
    channel: np.ndarray      # int32 [nt]
    materials: list
    surfaces: list
    pmt_array: np.ndarray    # int32 [P]: 0 bottom, 1 top
    pmt_pos: np.ndarray      # float32 [P, 3] centre of the photocathode
    source: Source
    info: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_pmts(self) -> int:
        return int(self.pmt_array.shape[0])

    def tri_vertices(self) -> np.ndarray:
        """float32 [nt, 3, 3] vertex triplets in index order."""
        return self.verts[self.tris]


# ----------------------------------------------------------------------------
# mesh assembly
# ----------------------------------------------------------------------------
def _snap(x):
    return np.round(np.asarray(x, np.float64) * SNAP) / SNAP


class _Builder:
    """Collects oriented triangles; welds shared vertices by their snapped
    coordinates; keeps pre-indexed chunks (wire prisms) as they are."""

    def __init__(self):
        self._tri = []      # float64 [n, 3, 3]
        self._attr = []     # int64 [n, 4]
        self._idx_chunks = []  # (verts float64 [m,3], tris int64 [k,3], attr int64 [k,4])

    @staticmethod
    def _orient(tri, normal):
        tri = np.array(tri, np.float64).reshape(-1, 3, 3)
        if tri.shape[0] == 0:
            return tri
        nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
        want = np.broadcast_to(np.asarray(normal, np.float64), nrm.shape)
        flip = (nrm * want).sum(1) < 0
        tri[flip] = tri[flip][:, [0, 2, 1]]
        return tri

    def add(self, tri, normal, mat_in, mat_out, surf=SURF_NONE, chan=-1):
        tri = self._orient(tri, normal)
        if tri.shape[0] == 0:
            return
        a = np.empty((tri.shape[0], 4), np.int64)
        a[:, 0], a[:, 1], a[:, 2], a[:, 3] = mat_in, mat_out, surf, chan
        self._tri.append(tri)
        self._attr.append(a)

    def add_indexed(self, verts, tris, mat_in, mat_out, surf=SURF_NONE, chan=-1):
        a = np.empty((tris.shape[0], 4), np.int64)
        a[:, 0], a[:, 1], a[:, 2], a[:, 3] = mat_in, mat_out, surf, chan
        self._idx_chunks.append((np.asarray(verts, np.float64), np.asarray(tris, np.int64), a))

    def finish(self):
        verts_out, tris_out, attr_out = [], [], []
        nv = 0
        if self._tri:
            tri = np.concatenate(self._tri)
            attr = np.concatenate(self._attr)
            q = np.round(tri.reshape(-1, 3) * SNAP).astype(np.int64)
            uq, inv = np.unique(q, axis=0, return_inverse=True)
            idx = inv.reshape(-1, 3)
            verts_out.append(uq.astype(np.float64) / SNAP)
            tris_out.append(idx)
            attr_out.append(attr)
            nv = uq.shape[0]
        for v, t, a in self._idx_chunks:
            verts_out.append(_snap(v))
            tris_out.append(t + nv)
            attr_out.append(a)
            nv += v.shape[0]
        verts = np.concatenate(verts_out).astype(np.float32)
        tris = np.concatenate(tris_out)
        attr = np.concatenate(attr_out)
        # drop triangles that snapping collapsed (repeated index or zero area)
        v = verts.astype(np.float64)[tris]
        area2 = np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1)
        keep = (tris[:, 0] != tris[:, 1]) & (tris[:, 1] != tris[:, 2]) & (tris[:, 0] != tris[:, 2]) & (area2 > 0)
        tris, attr = tris[keep], attr[keep]
        return (verts, tris.astype(np.uint32), attr[:, 0].astype(np.uint8), attr[:, 1].astype(np.uint8),
                attr[:, 2].astype(np.uint16), attr[:, 3].astype(np.int32))


# ----------------------------------------------------------------------------
# primitives
# ----------------------------------------------------------------------------
def polygon_vertices(n_sides, radius, phase=0.0):
    k = np.arange(n_sides)
    ang = phase + 2.0 * math.pi * k / n_sides
    return np.stack([radius * np.cos(ang), radius * np.sin(ang)], 1)


def _circle(center, r, k_seg, phase=0.0):
    ang = phase + 2.0 * math.pi * np.arange(k_seg) / k_seg
    return np.stack([center[0] + r * np.cos(ang), center[1] + r * np.sin(ang)], 1)


def _fan(poly2, z, center2=None):
    """Triangles of a convex polygon fanned from its centre (or a given point)."""
    m = poly2.shape[0]
    c = poly2.mean(0) if center2 is None else np.asarray(center2, np.float64)
    tri = np.zeros((m, 3, 3))
    tri[:, 0, :2] = c
    tri[:, 1, :2] = poly2
    tri[:, 2, :2] = np.roll(poly2, -1, 0)
    tri[:, :, 2] = z
    return tri


def _disk(center2, r, k_seg, z, rings=4):
    """Disk of radius r as concentric rings (vertex counts k_seg * j / rings)
    around a small central fan: triangles of bounded aspect ratio instead of
    k_seg wedges meeting at the centre.  The rim is ``_circle(center2, r,
    k_seg)``, so it welds to any other primitive sharing that circle."""
    rings = max(1, min(rings, k_seg // 4))
    prev = _circle(center2, r / rings, max(4, k_seg // rings))
    tri = [_fan(prev, z, center2)]
    for j in range(2, rings + 1):
        cur = _circle(center2, r * j / rings, max(4, k_seg * j // rings))
        tri.append(_ring(cur, prev, z, center2))
        prev = cur
    return np.concatenate(tri)


def _subdivide(poly2, seg_len):
    """Polygon with every edge split into equal pieces no longer than
    seg_len; the split points of an edge depend only on its two endpoints
    (taken in a fixed order), so neighbouring polygons sharing the edge get
    identical points."""
    out = []
    m = len(poly2)
    for k in range(m):
        a, b = poly2[k], poly2[(k + 1) % m]
        out.append(a)
        L = float(np.hypot(*(b - a)))
        n = max(1, int(math.ceil(L / seg_len - 1e-9)))
        swap = tuple(a) > tuple(b)
        p, q = (b, a) if swap else (a, b)
        pts = [p + (q - p) * (i / n) for i in range(1, n)]
        if swap:
            pts = pts[::-1]
        out.extend(pts)
    return np.array(out, np.float64)


def _ring(outer2, inner2, z, center2):
    """Triangulate the region between a star-shaped outer polygon and an inner
    polygon (both around ``center2``) by merging their vertices by angle."""
    c = np.asarray(center2, np.float64)

    def sort_by_angle(p):
        a = np.arctan2(p[:, 1] - c[1], p[:, 0] - c[0]) % (2 * math.pi)
        o = np.argsort(a, kind="stable")
        return p[o], a[o]

    P, aP = sort_by_angle(outer2)
    Q, aQ = sort_by_angle(inner2)
    m, k = len(P), len(Q)
    # unwrap both angle sequences to start at aP[0]
    base = aP[0]
    aP = (aP - base) % (2 * math.pi)
    aQ = (aQ - base) % (2 * math.pi)
    oq = np.argsort(aQ, kind="stable")
    Q, aQ = Q[oq], aQ[oq]
    # the inner vertex preceding angle 0 closes the strip
    tris = []
    i = j = 0
    cur_p, cur_q = P[0], Q[-1]
    ap_next = lambda i: aP[i + 1] if i + 1 < m else 2 * math.pi
    aq_next = lambda j: aQ[j] if j < k else 2 * math.pi + aQ[0]
    while i < m or j < k:
        take_p = (j >= k) or (i < m and ap_next(i) <= aq_next(j))
        if take_p:
            nxt = P[(i + 1) % m]
            tris.append((cur_p, nxt, cur_q))
            cur_p = nxt
            i += 1
        else:
            nxt = Q[j]
            tris.append((cur_p, nxt, cur_q))
            cur_q = nxt
            j += 1
    out = np.zeros((len(tris), 3, 3))
    for t, (a, b, cc) in enumerate(tris):
        out[t, 0, :2], out[t, 1, :2], out[t, 2, :2] = a, b, cc
    out[:, :, 2] = z
    return out


def _clip_convex(subject, clip):
    """Sutherland-Hodgman: convex ``subject`` polygon clipped by convex
    counter-clockwise ``clip`` polygon (both [m, 2])."""
    out = [tuple(p) for p in subject]
    n = len(clip)
    for e in range(n):
        a, b = clip[e], clip[(e + 1) % n]
        ex, ey = b[0] - a[0], b[1] - a[1]
        inside = lambda p: ex * (p[1] - a[1]) - ey * (p[0] - a[0]) >= 0.0
        inp, out = out, []
        if not inp:
            break
        s = inp[-1]
        for p in inp:
            if inside(p):
                if not inside(s):
                    out.append(_seg_line(s, p, a, b))
                out.append(p)
            elif inside(s):
                out.append(_seg_line(s, p, a, b))
            s = p
    return np.array(out, np.float64).reshape(-1, 2)


def _seg_line(p, q, a, b):
    x1, y1 = p
    x2, y2 = q
    x3, y3 = a
    x4, y4 = b
    den = (x1 - x2) * (y3 - y4) - (y1 - y2) * (x3 - x4)
    t = ((x1 - x3) * (y3 - y4) - (y1 - y3) * (x3 - x4)) / den
    return (x1 + t * (x2 - x1), y1 + t * (y2 - y1))


def _inside_convex(pts, poly, margin=0.0):
    """Points [m,2] inside CCW convex polygon shrunk by ``margin``."""
    ok = np.ones(len(pts), bool)
    n = len(poly)
    for e in range(n):
        a, b = poly[e], poly[(e + 1) % n]
        d = b - a
        nrm = np.array([d[1], -d[0]]) / np.hypot(*d)  # outward normal of a CCW polygon
        ok &= ((pts - a) @ nrm) <= -margin
    return ok


def hex_lattice(pitch, extent):
    """Hex-packed centres (spacing ``pitch``) within radius ``extent``."""
    jmax = int(extent / (pitch * math.sqrt(3) / 2)) + 2
    pts = []
    for j in range(-jmax, jmax + 1):
        y = j * pitch * math.sqrt(3) / 2
        off = 0.5 * pitch * (j & 1)
        imax = int(extent / pitch) + 2
        for i in range(-imax, imax + 1):
            x = i * pitch + off
            if x * x + y * y <= extent * extent:
                pts.append((x, y))
    return np.array(pts, np.float64)


# ----------------------------------------------------------------------------
# detector parts
# ----------------------------------------------------------------------------
def hex_ring(centres, pitch):
    """Hexagonal ring of hex_lattice sites: the fewest neighbour steps from
    the site at the origin (0 for the centre, 1 for its 6 neighbours, ...)."""
    b = np.rint(centres[:, 1] / (pitch * math.sqrt(3) / 2))
    a = np.rint((centres[:, 0] - 0.5 * pitch * b) / pitch)
    return ((np.abs(a) + np.abs(b) + np.abs(a + b)) / 2).astype(int)


def _pmt_plate(b, wall2, z_plate, pitch, r_window, k_seg, facing, mat_xe, surf_plate, subdivide=False, holes=True,
               max_ring=None):
    """PTFE plate at ``z_plate`` filling the wall polygon, with a circular hole
    of radius ``r_window`` at every hex-lattice site whose window fits inside
    the wall (no holes if not ``holes``; only sites of hexagonal ring <=
    ``max_ring`` if given).  ``facing`` = +1 if the plate faces up (bottom
    array), -1 if it faces down (top array).  Returns the PMT centres (x, y)."""
    extent = np.abs(wall2).max() + pitch
    centres = hex_lattice(pitch, extent)
    # a PMT sits on every site whose window circle is inside the wall (0.5 mm clearance)
    has_pmt = _inside_convex(centres, wall2, margin=r_window + 0.5) & holes
    if max_ring is not None:
        has_pmt &= hex_ring(centres, pitch) <= max_ring
    hexagon = polygon_vertices(6, pitch / math.sqrt(3), math.pi / 6)  # flat-to-flat = pitch
    pmts, cells = [], []
    normal = (0.0, 0.0, -float(facing))  # plate normal points from Xe into PTFE
    seg_len = 2.0 * math.pi * r_window / k_seg   # the rim's segment length
    for c, pm in zip(centres, has_pmt):
        cell = _clip_convex(hexagon + c, wall2)
        if cell.shape[0] < 3:
            continue
        # snap before subdividing so that cells sharing an edge split it alike
        if subdivide:
            cell = _subdivide(_snap(cell), seg_len)
        cells.append(cell)
        if pm:
            rim = _circle(c, r_window, k_seg)
            b.add(_ring(cell, rim, z_plate, c), normal, mat_xe, OPAQUE, surf_plate)
            pmts.append(c)
        else:
            b.add(_fan(cell, z_plate), normal, mat_xe, OPAQUE, surf_plate)
    return np.array(pmts, np.float64).reshape(-1, 2), _boundary_points(cells, wall2)


def _pmt_windows(b, centres, z_front, thickness, facing, r_window, r_pc, k_seg, mat_xe,
                 surf_cap, surf_pc, chan0, rings=2, cone_h=0.0, surf_cone=SURF_NONE):
    """Quartz windows: front face in the xenon (bare dielectric boundary), side
    wall and back-face annulus covered by the absorbing cap, photocathode disk
    of radius ``r_pc`` on the back face (Sec. 2.1, Fig. 1).  With cone_h > 0
    a PTFE reflector of conical cross section sits on each window (Sec. 2.1):
    a cone from the photocathode radius on the front face to the window
    radius cone_h into the xenon, closed by a cylindrical collar at the
    window radius; the front face is then bare only inside r_pc, the annulus
    beyond it touches the PTFE (surface ``surf_cone``)."""
    z_back = z_front - facing * thickness
    for p, c in enumerate(centres):
        rim = _circle(c, r_window, k_seg)
        # front face, normal out of the quartz into the xenon
        if cone_h > 0.0:
            inner = _circle(c, r_pc, k_seg)
            b.add(_disk(c, r_pc, k_seg, z_front, rings), (0, 0, facing), QUARTZ, mat_xe)
            b.add(_ring(rim, inner, z_front, c), (0, 0, facing), QUARTZ, OPAQUE, surf_cone)
            z_top = z_front + facing * cone_h
            phi = np.arctan2(inner[:, 1] - c[1], inner[:, 0] - c[0]) + math.pi / k_seg
            phi = np.concatenate([phi, phi])
            # cone: from (r_pc, z_front) to (r_window, z_top); normal from the
            # xenon inside the opening into the PTFE
            a0 = np.concatenate([inner, np.full((k_seg, 1), z_front)], 1)
            a1 = np.concatenate([rim, np.full((k_seg, 1), z_top)], 1)
            a0n, a1n = np.roll(a0, -1, 0), np.roll(a1, -1, 0)
            cone = np.concatenate([np.stack([a0, a0n, a1n], 1), np.stack([a0, a1n, a1], 1)])
            nrm = np.stack([cone_h * np.cos(phi), cone_h * np.sin(phi),
                            np.full(phi.shape, -facing * (r_window - r_pc))], 1)
            b.add(cone, nrm, mat_xe, OPAQUE, surf_cone)
            # collar: cylinder at the window radius, xenon outside, PTFE inside
            r0 = np.concatenate([rim, np.full((k_seg, 1), z_front)], 1)
            r0n = np.roll(r0, -1, 0)
            collar = np.concatenate([np.stack([r0, r0n, a1n], 1), np.stack([r0, a1n, a1], 1)])
            b.add(collar, -np.stack([np.cos(phi), np.sin(phi), np.zeros_like(phi)], 1), mat_xe, OPAQUE,
                  surf_cone)
        else:
            b.add(_disk(c, r_window, k_seg, z_front, rings), (0, 0, facing), QUARTZ, mat_xe)
        # side wall
        r0 = np.concatenate([rim, np.full((k_seg, 1), z_front)], 1)
        r1 = np.concatenate([rim, np.full((k_seg, 1), z_back)], 1)
        r0n, r1n = np.roll(r0, -1, 0), np.roll(r1, -1, 0)
        side = np.concatenate([np.stack([r0, r0n, r1n], 1), np.stack([r0, r1n, r1], 1)])
        mid = side.mean(1)
        nrm = mid.copy()
        nrm[:, :2] -= c
        nrm[:, 2] = 0
        b.add(side, nrm, QUARTZ, OPAQUE, surf_cap)
        # back face: photocathode disk (+ cap annulus)
        back_n = (0, 0, -facing)
        if r_pc >= r_window:
            b.add(_disk(c, r_window, k_seg, z_back, rings), back_n, QUARTZ, OPAQUE, surf_pc, chan0 + p)
        else:
            inner = _circle(c, r_pc, k_seg)
            b.add(_disk(c, r_pc, k_seg, z_back, rings), back_n, QUARTZ, OPAQUE, surf_pc, chan0 + p)
            b.add(_ring(rim, inner, z_back, c), back_n, QUARTZ, OPAQUE, surf_cap)


def _wall(b, wall2, z0, z1, mat_xe, surf, bottom_pts=None, top_pts=None):
    """Side-wall panels of the extruded polygon between z0 and z1.  The bottom
    (top) edge of side k is split at ``bottom_pts[k]`` (``top_pts[k]``), the
    2-D points where the plate meeting the wall there has vertices, so the
    seam is conforming (no T-junction cracks)."""
    n = len(wall2)
    for k in range(n):
        a, c = wall2[k], wall2[(k + 1) % n]
        d = c - a
        L2 = float(d @ d)

        def chain(extra):
            pts = [a] + ([] if extra is None else list(extra[k])) + [c]
            pts = np.array(pts, np.float64)
            s = ((pts - a) @ d) / L2
            return pts[np.argsort(s, kind="stable")], np.sort(s)

        B, sb = chain(bottom_pts)
        T, st = chain(top_pts)
        tris = []
        i = j = 0
        while i < len(B) - 1 or j < len(T) - 1:
            adv_b = j >= len(T) - 1 or (i < len(B) - 1 and sb[i + 1] <= st[j + 1])
            if adv_b:
                tris.append(((*B[i], z0), (*B[i + 1], z0), (*T[j], z1)))
                i += 1
            else:
                tris.append(((*B[i], z0), (*T[j + 1], z1), (*T[j], z1)))
                j += 1
        mid = 0.5 * (a + c)
        b.add(np.array(tris, np.float64), (mid[0], mid[1], 0.0), mat_xe, OPAQUE, surf)


def _boundary_points(cells, wall2, tol=1e-6):
    """For every side of the wall polygon, the cell vertices lying on it
    (corners excluded), as 2-D points."""
    n = len(wall2)
    out = [[] for _ in range(n)]
    seen = [set() for _ in range(n)]
    for cell in cells:
        for p in cell:
            for k in range(n):
                a, c = wall2[k], wall2[(k + 1) % n]
                d = c - a
                L = math.hypot(*d)
                dist = abs(d[0] * (p[1] - a[1]) - d[1] * (p[0] - a[0])) / L
                s = ((p - a) @ d) / (L * L)
                if dist < max(tol * max(1.0, L), 2.0 / SNAP) and 1e-9 < s < 1 - 1e-9:
                    key = tuple(np.round(p * SNAP).astype(np.int64))
                    if key not in seen[k]:
                        seen[k].add(key)
                        out[k].append(p.copy())
    return out


def hex_wire_mesh(wall2, z, pitch, wire, margin=1.0):
    """Hexagonal wire mesh (flat-to-flat ``pitch``) of square-section wires of
    width ``wire`` in the plane ``z``, clipped to the wall polygon shrunk by
    ``margin``.  Each honeycomb edge is one prism of 4 faces (8 triangles),
    lengthened by wire/4 at both ends so that the open ends are covered by
    the neighbouring prisms at every junction.  Returns (verts [m,3],
    tris [k,3]) with outward-facing triangles."""
    a = pitch / math.sqrt(3)             # hexagon side
    extent = np.abs(wall2).max() + 2 * pitch
    jmax = int(extent / (pitch * math.sqrt(3) / 2)) + 2
    imax = int(extent / pitch) + 2
    jj, ii = np.meshgrid(np.arange(-jmax, jmax + 1), np.arange(-imax, imax + 1), indexing="ij")
    cx = ii * pitch + 0.5 * pitch * (jj & 1)
    cy = jj * pitch * math.sqrt(3) / 2
    A = np.stack([cx.ravel(), cy.ravel() + a], 1)   # top vertex of every cell
    dirs = np.array([[0.0, 1.0], [math.cos(-math.pi / 6), math.sin(-math.pi / 6)],
                     [math.cos(7 * math.pi / 6), math.sin(7 * math.pi / 6)]])
    P0 = np.repeat(A, 3, 0)
    P1 = P0 + a * np.tile(dirs, (A.shape[0], 1))
    keep = _inside_convex(P0, wall2, margin) & _inside_convex(P1, wall2, margin)
    P0, P1 = P0[keep], P1[keep]
    ns = P0.shape[0]
    u = (P1 - P0) / a
    ext = wire / 4.0
    P0 = P0 - ext * u
    P1 = P1 + ext * u
    v = np.stack([-u[:, 1], u[:, 0]], 1)
    h = wire / 2.0
    # cross-section corners (v, z): (+,+), (-,+), (-,-), (+,-) counter-clockwise about u
    cs = np.array([[1, 1], [-1, 1], [-1, -1], [1, -1]], np.float64) * h
    verts = np.zeros((ns, 8, 3))
    for k in range(4):
        for e, P in enumerate((P0, P1)):
            verts[:, 4 * e + k, :2] = P + cs[k, 0] * v
            verts[:, 4 * e + k, 2] = z + cs[k, 1]
    # faces: corner k -> k+1 at end 0 and end 1
    local = []
    for k in range(4):
        k1 = (k + 1) % 4
        a0, b0, a1, b1 = k, k1, 4 + k, 4 + k1
        local.append((a0, b0, b1))
        local.append((a0, b1, a1))
    local = np.array(local, np.int64)
    tris = (np.arange(ns)[:, None, None] * 8 + local[None]).reshape(-1, 3)
    verts = verts.reshape(-1, 3)
    # orient outward: compare with the vector from the prism axis to the face centre
    tv = verts[tris]
    nrm = np.cross(tv[:, 1] - tv[:, 0], tv[:, 2] - tv[:, 0])
    seg = np.repeat(np.arange(ns), 8)
    axis_mid = np.concatenate([(P0 + P1) / 2, np.full((ns, 1), z)], 1)[seg]
    outward = tv.mean(1) - axis_mid
    flip = (nrm * outward).sum(1) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts, tris


def parallel_wires(wall2, z, pitch, wire, r_end, along=0):
    """Plane of parallel wires (Sec. 2.1: stainless-steel wires of 200 um at
    5 or 7.5 mm pitch) running along x (along=0) or y (1) at height z,
    square-section prisms of width ``wire`` (8 triangles each, same
    construction as the hex meshes), each cut where it leaves the polygon
    wall2 scaled to circumradius ``r_end`` (the wire ends lie inside the
    frame).  Returns (verts [m,3], tris [k,3]), outward-facing."""
    R = float(np.abs(wall2).max())
    inner = wall2 * (r_end / R)
    offs = np.arange(-math.floor(r_end / pitch), math.floor(r_end / pitch) + 1) * pitch
    h = wire / 2.0
    verts, tris = [], []
    for o in offs:
        # chord of the inner polygon along the wire direction at offset o
        p = np.array([[-2 * R, o], [2 * R, o]]) if along == 0 else np.array([[o, -2 * R], [o, 2 * R]])
        seg = _clip_segment(p[0], p[1], inner)
        if seg is None or np.linalg.norm(seg[1] - seg[0]) < 10 * wire:
            continue
        P0, P1 = seg
        u = (P1 - P0) / np.linalg.norm(P1 - P0)
        v = np.array([-u[1], u[0]])
        cs = np.array([[1, 1], [-1, 1], [-1, -1], [1, -1]], np.float64) * h
        vv = np.zeros((8, 3))
        for k in range(4):
            for e, P in enumerate((P0, P1)):
                vv[4 * e + k, :2] = P + cs[k, 0] * v
                vv[4 * e + k, 2] = z + cs[k, 1]
        t = []
        for k in range(4):
            k1 = (k + 1) % 4
            t += [(k, k1, 4 + k1), (k, 4 + k1, 4 + k)]
        t = np.array(t, np.int64)
        tv = vv[t]
        nrm = np.cross(tv[:, 1] - tv[:, 0], tv[:, 2] - tv[:, 0])
        mid = np.array([*(P0 + P1) / 2, z])
        flip = (nrm * (tv.mean(1) - mid)).sum(1) < 0
        t[flip] = t[flip][:, [0, 2, 1]]
        tris.append(t + 8 * len(verts))
        verts.append(vv)
    if not verts:
        return np.zeros((0, 3)), np.zeros((0, 3), np.int64)
    return np.concatenate(verts), np.concatenate(tris)


def _clip_segment(a, b, poly):
    """Part of segment a-b inside the convex polygon (counter-clockwise), or None."""
    t0, t1 = 0.0, 1.0
    d = b - a
    n = poly.shape[0]
    for k in range(n):
        p, q = poly[k], poly[(k + 1) % n]
        e = q - p
        nrm = np.array([e[1], -e[0]])  # outward for a counter-clockwise polygon
        den = nrm @ d
        num = nrm @ (p - a)
        if abs(den) < 1e-15:
            if num < 0:
                return None
            continue
        t = num / den
        if den > 0:
            t1 = min(t1, t)
        else:
            t0 = max(t0, t)
        if t0 > t1:
            return None
    return a + t0 * d, a + t1 * d


def _frame(b, wall2, z_lo, z_hi, r_in, mat_xe, surf):
    """Electrode frame (Sec. 2.1: an extruded 24-sided polygon on which the
    wires are fixed): the annulus between the wall polygon and the polygon
    scaled to circumradius r_in, from z_lo to z_hi, opaque inside; its outer
    face is the wall itself."""
    R = float(np.abs(wall2).max())
    inner = wall2 * (r_in / R)
    c = (0.0, 0.0)
    b.add(_ring(wall2, inner, z_hi, c), (0, 0, -1), mat_xe, OPAQUE, surf)   # top face, normal into the frame
    b.add(_ring(wall2, inner, z_lo, c), (0, 0, 1), mat_xe, OPAQUE, surf)    # bottom face
    n = inner.shape[0]
    i0 = np.concatenate([inner, np.full((n, 1), z_lo)], 1)
    i1 = np.concatenate([inner, np.full((n, 1), z_hi)], 1)
    i0n, i1n = np.roll(i0, -1, 0), np.roll(i1, -1, 0)
    side = np.concatenate([np.stack([i0, i0n, i1n], 1), np.stack([i0, i1n, i1], 1)])
    nrm = side.mean(1)
    nrm[:, 2] = 0.0
    b.add(side, nrm, mat_xe, OPAQUE, surf)  # inner face, normal radially outwards = into the frame


# ----------------------------------------------------------------------------
# optical tables (Table 2 of the paper; workload values override it)
# ----------------------------------------------------------------------------
def default_materials(lxe_abs_mm=50_000.0, lxe_ray_mm=400.0, gxe_abs_mm=1e9, gxe_ray_mm=INF):
    return [
        Material("LXe", 1.69, lxe_abs_mm, lxe_ray_mm),
        Material("GXe", 1.00, gxe_abs_mm, gxe_ray_mm),
        Material("quartz", 1.60, INF, INF),
        Material("opaque", 1.00, INF, INF),
    ]


# ----------------------------------------------------------------------------
# detectors
# ----------------------------------------------------------------------------
def small_tpc(r_ptfe_lxe=0.95, r_ptfe_gxe=0.70, qe=0.3, lxe_abs_mm=50_000.0, lxe_ray_mm=400.0,
              wall_sides=64, k_seg=32):
    """Small dual-phase TPC: 100 mm radius PTFE cylinder (64-sided), 100 mm of
    LXe under a 5 mm GXe gap, 7 top + 7 bottom hex-packed PMT windows (64 mm
    diameter at 66 mm pitch, photocathode = whole back face; a 7-hex of 3-inch
    windows does not fit in 100 mm radius), Lambertian PTFE 0.95 (LXe) / 0.70
    (GXe), QE 0.3.  ~4.4k triangles.  Source: uniform in the LXe, isotropic."""
    R, z_bot, z_liq, z_top = 100.0, -100.0, 0.0, 5.0
    r_w, pitch, thick = 32.0, 66.0, 5.0
    mats = default_materials(lxe_abs_mm, lxe_ray_mm)
    S_PTFE_L, S_PTFE_G, S_CAP, S_PC = 0, 1, 2, 3
    surfs = [
        Surface("PTFE_LXe", REFLECTOR, r_ptfe_lxe, 0.0),
        Surface("PTFE_GXe", REFLECTOR, r_ptfe_gxe, 0.0),
        Surface("PMT_cap", ABSORBER),
        Surface("photocathode", PHOTOCATHODE, qe=qe),
    ]
    wall2 = polygon_vertices(wall_sides, R)
    b = _Builder()
    bot, bot_edge = _pmt_plate(b, wall2, z_bot, pitch, r_w, k_seg, +1, LXE, S_PTFE_L)
    top, top_edge = _pmt_plate(b, wall2, z_top, pitch, r_w, k_seg, -1, GXE, S_PTFE_G)
    _wall(b, wall2, z_bot, z_liq, LXE, S_PTFE_L, bottom_pts=bot_edge)
    _wall(b, wall2, z_liq, z_top, GXE, S_PTFE_G, top_pts=top_edge)
    b.add(_fan(wall2, z_liq, (0, 0)), (0, 0, 1), LXE, GXE)           # liquid surface
    _pmt_windows(b, bot, z_bot, thick, +1, r_w, r_w, k_seg, LXE, S_CAP, S_PC, 0, rings=2)
    _pmt_windows(b, top, z_top, thick, -1, r_w, r_w, k_seg, GXE, S_CAP, S_PC, len(bot), rings=2)
    src = Source(SRC_VOLUME_POLYGON, LXE, n_sides=wall_sides, radius=R, z_min=z_bot, z_max=z_liq)
    return _detector("small_tpc", b, mats, surfs, bot, top, z_bot - thick, z_top + thick, src,
                     dict(radius=R, wall_sides=wall_sides, z_liquid=z_liq))


def darwin(pitch_pmt=80.0, wire_um=216.0, mesh_pitch=5.0, electrodes=("gate", "anode", "cathode"),
           r_ptfe_lxe=0.95, r_ptfe_gxe=0.70, qe=0.3, lxe_abs_mm=50_000.0, lxe_ray_mm=400.0,
           r_ss=0.30, ss_spec_frac=2.0 / 3.0, k_seg=32, active_only=True, window_rings=2, plate_subdivide=False,
           ptfe_spec_frac=0.0, coated=(), r_coat=0.90, coat_spec_frac=0.85 / 0.90, single_phase=False,
           bottom_array=True, r_ptfe_bottom=0.99, gxe_abs_mm=1e9, gxe_ray_mm=INF, electrode_kind="mesh",
           pmt_cones=0.0):
    """DARWIN-scale dual-phase TPC (Sec. 2.1, Table 1): 24-sided PTFE wall
    inscribed in r = 1300 mm; gate z = 0 (LXe), liquid surface z = +2, anode
    z = +8 (GXe), cathode z = -2598; hex-packed 3-inch windows (76.2 mm, 5 mm
    quartz, 64 mm photocathode on the back face) with front faces at z = +64
    (top, facing down) and z = -2688 (bottom, facing up), photocathodes at
    +69 / -2693; electrodes as hexagonal stainless-steel wire meshes (square
    wires of ``wire_um``, flat-to-flat ``mesh_pitch``) with R = 0.30 and
    specular/diffuse ratio 2 (Table 2).  Source: uniform in the active LXe,
    z in [-2597, -1] (Sec. 3, average-LCE definition), isotropic.

    Design variants (Sec. 5):
    * ``coated``: names of electrodes whose wires carry an Al/MgF2 coating,
      total reflectivity ``r_coat`` of which ``coat_spec_frac`` specular
      (Sec. 5.1: 90 %, 85 of it specular);
    * ``single_phase``: LXe fills the detector up to the top array, with no
      liquid surface (Sec. 5.3); the PTFE above the gate then has the LXe
      reflectivity;
    * ``bottom_array=False``: the bottom array is replaced by a PTFE plate of
      reflectivity ``r_ptfe_bottom`` (Sec. 5.4: 99 %);
    * ``ptfe_spec_frac``: specular fraction of the PTFE reflection;
    * ``electrode_kind="wires"``: the paper's own baseline electrodes (Sec.
      2.1, Table 1) instead of the hex meshes: five planes of parallel
      200 um stainless-steel wires, top screen z = 54, anode z = 12 and gate
      z = 0 at 5 mm pitch, cathode z = -2598 and bottom screen z = -2678 at
      7.5 mm pitch, each fixed to a 24-gon frame 20 mm wide and 8 mm high
      (PTFE-covered on top, bare steel below; a surface entry of its own);
      ``electrodes`` is ignored;
    * ``pmt_cones``: height (mm) of a conical PTFE reflector on each window
      (Sec. 2.1; the paper gives no size: 0 = flat plates)."""
    R = 1300.0
    z_bot, z_cath, z_gate, z_liq, z_anode, z_top = -2688.0, -2598.0, 0.0, 2.0, 8.0, 64.0
    r_w, r_pc, thick = 38.1, 32.0, 5.0
    mats = default_materials(lxe_abs_mm, lxe_ray_mm, gxe_abs_mm, gxe_ray_mm)
    S_PTFE_L, S_PTFE_G, S_CAP, S_PC = 0, 1, 2, 3
    gas = LXE if single_phase else GXE
    surfs = [
        Surface("PTFE_LXe", REFLECTOR, r_ptfe_lxe, ptfe_spec_frac),
        Surface("PTFE_GXe", REFLECTOR, r_ptfe_lxe if single_phase else r_ptfe_gxe, ptfe_spec_frac),
        Surface("PMT_cap", ABSORBER),
        Surface("photocathode", PHOTOCATHODE, qe=qe),
    ]
    s_bottom = S_PTFE_L
    if not bottom_array:
        s_bottom = len(surfs)
        surfs.append(Surface("PTFE_bottom", REFLECTOR, r_ptfe_bottom, ptfe_spec_frac))
    wall2 = polygon_vertices(24, R)
    b = _Builder()
    bot, bot_edge = _pmt_plate(b, wall2, z_bot, pitch_pmt, r_w, k_seg, +1, LXE, s_bottom, plate_subdivide,
                               holes=bottom_array)
    top, top_edge = _pmt_plate(b, wall2, z_top, pitch_pmt, r_w, k_seg, -1, gas, S_PTFE_G, plate_subdivide)
    _wall(b, wall2, z_bot, z_liq, LXE, S_PTFE_L, bottom_pts=bot_edge)
    _wall(b, wall2, z_liq, z_top, gas, S_PTFE_G, top_pts=top_edge)
    if not single_phase:
        b.add(_fan(wall2, z_liq, (0, 0)), (0, 0, 1), LXE, GXE)
    _pmt_windows(b, bot, z_bot, thick, +1, r_w, r_pc, k_seg, LXE, S_CAP, S_PC, 0, rings=window_rings,
                 cone_h=pmt_cones, surf_cone=S_PTFE_L)
    _pmt_windows(b, top, z_top, thick, -1, r_w, r_pc, k_seg, gas, S_CAP, S_PC, len(bot), rings=window_rings,
                 cone_h=pmt_cones, surf_cone=S_PTFE_G)
    if electrode_kind == "wires":
        # (name, wire plane z, frame z range, xenon phase, pitch, frame surface)
        planes = (("screen_top", 54.0, (50.0, 58.0), gas, 5.0, S_PTFE_G),
                  ("anode", 12.0, (8.0, 16.0), gas, 5.0, S_PTFE_G),
                  ("gate", 0.0, (-9.0, -1.0), LXE, 5.0, S_PTFE_L),
                  ("cathode", -2598.0, (-2602.0, -2594.0), LXE, 7.5, None),
                  ("screen_bottom", -2678.0, (-2682.0, -2674.0), LXE, 7.5, None))
        # gate frame below the plane so that it stays in the liquid
        for name, zw, (f0, f1), mat, pitch, fsurf in planes:
            sid = len(surfs)
            if name in coated:
                surfs.append(Surface(f"{name}_AlMgF2", REFLECTOR, r_coat, coat_spec_frac))
            else:
                surfs.append(Surface(f"{name}_SS", REFLECTOR, r_ss, ss_spec_frac))
            v, t = parallel_wires(wall2, zw, pitch, 0.200, r_end=R - 10.0)
            b.add_indexed(v, t, OPAQUE, mat, sid)
            # the frame: its own surface entry (PTFE-covered above, bare or coated steel below)
            fid = len(surfs)
            base = surfs[fsurf] if fsurf is not None else surfs[sid]
            surfs.append(Surface(f"{name}_frame", REFLECTOR, base.reflectivity, base.spec_frac))
            _frame(b, wall2, f0, f1, R - 20.0, mat, fid)
        electrodes = tuple(p[0] for p in planes)
    zs = dict(gate=(z_gate, LXE), anode=(z_anode, gas), cathode=(z_cath, LXE))
    for name in (electrodes if electrode_kind == "mesh" else ()):
        ze, mat = zs[name]
        sid = len(surfs)
        if name in coated:
            surfs.append(Surface(f"{name}_AlMgF2", REFLECTOR, r_coat, coat_spec_frac))
        else:
            surfs.append(Surface(f"{name}_SS", REFLECTOR, r_ss, ss_spec_frac))
        v, t = hex_wire_mesh(wall2, ze, mesh_pitch, wire_um * 1e-3)
        b.add_indexed(v, t, OPAQUE, mat, sid)
    z0, z1 = (z_cath + 1.0, z_gate - 1.0) if active_only else (z_bot, z_liq)
    src = Source(SRC_VOLUME_POLYGON, LXE, n_sides=24, radius=R, z_min=z0, z_max=z1)
    return _detector("darwin", b, mats, surfs, bot, top, z_bot - thick, z_top + thick, src,
                     dict(radius=R, wall_sides=24, z_liquid=None if single_phase else z_liq,
                          electrodes=list(electrodes), coated=list(coated), single_phase=single_phase,
                          bottom_array=bottom_array))


# Best-guess optical constants of the paper's Table 2 (the workloads above use
# the benchmark optics instead): L_Rayleigh 36 cm in LXe, 500 m absorption and
# 200 m Rayleigh length in GXe, PTFE 99 % in LXe and 80 % in GXe with a
# specular/diffuse ratio of 0.05 (specular fraction 0.05 / 1.05).
PAPER_OPTICS = dict(lxe_abs_mm=50_000.0, lxe_ray_mm=360.0, gxe_abs_mm=500_000.0, gxe_ray_mm=200_000.0,
                    r_ptfe_lxe=0.99, r_ptfe_gxe=0.80, ptfe_spec_frac=0.05 / 1.05)


def _detector(name, b, mats, surfs, bot, top, z_pc_bot, z_pc_top, src, info):
    verts, tris, mi, mo, sf, ch = b.finish()
    pmt_array = np.concatenate([np.zeros(len(bot), np.int32), np.ones(len(top), np.int32)])
    pos = np.zeros((len(bot) + len(top), 3), np.float32)
    pos[:len(bot), :2] = bot
    pos[:len(bot), 2] = z_pc_bot
    pos[len(bot):, :2] = top
    pos[len(bot):, 2] = z_pc_top
    return Detector(name, verts, tris, mi, mo, sf, ch, mats, surfs, pmt_array, pos, src, info)


def scaled_tpc(r_ptfe_lxe=0.95, r_ptfe_gxe=0.70, qe=0.3, lxe_abs_mm=50_000.0, lxe_ray_mm=400.0,
               transparency=(0.95, 0.95, 0.97), r_wire=0.30, wire_spec_frac=2.0 / 3.0, k_seg=32):
    """The small TPC scaled x5 (radius 500 mm, 500 mm of LXe, 5 mm GXe gap)
    with 61 + 61 3-inch windows at 80 mm pitch and gate (z = -5, LXe), anode
    (z = +2.5, GXe) and cathode (z = -495, LXe) as thin effective-transparency
    disks (the Geant4 electrode model of Sec. 2.1)."""
    R, z_bot, z_liq, z_top = 500.0, -500.0, 0.0, 5.0
    r_w, r_pc, pitch, thick = 38.1, 32.0, 80.0, 5.0
    mats = default_materials(lxe_abs_mm, lxe_ray_mm)
    S_PTFE_L, S_PTFE_G, S_CAP, S_PC = 0, 1, 2, 3
    surfs = [
        Surface("PTFE_LXe", REFLECTOR, r_ptfe_lxe, 0.0),
        Surface("PTFE_GXe", REFLECTOR, r_ptfe_gxe, 0.0),
        Surface("PMT_cap", ABSORBER),
        Surface("photocathode", PHOTOCATHODE, qe=qe),
    ]
    wall2 = polygon_vertices(64, R)
    b = _Builder()
    # 61 windows per array: hexagonal rings 0..4 (1 + 6 + 12 + 18 + 24)
    bot, bot_edge = _pmt_plate(b, wall2, z_bot, pitch, r_w, k_seg, +1, LXE, S_PTFE_L, max_ring=4)
    top, top_edge = _pmt_plate(b, wall2, z_top, pitch, r_w, k_seg, -1, GXE, S_PTFE_G, max_ring=4)
    # the wall is split at every electrode plane so the disk rims weld to it
    _wall(b, wall2, z_bot, -495.0, LXE, S_PTFE_L, bottom_pts=bot_edge)
    _wall(b, wall2, -495.0, -5.0, LXE, S_PTFE_L)
    _wall(b, wall2, -5.0, z_liq, LXE, S_PTFE_L)
    _wall(b, wall2, z_liq, 2.5, GXE, S_PTFE_G)
    _wall(b, wall2, 2.5, z_top, GXE, S_PTFE_G, top_pts=top_edge)
    b.add(_fan(wall2, z_liq, (0, 0)), (0, 0, 1), LXE, GXE)
    for name, ze, mat, T in (("gate", -5.0, LXE, transparency[0]), ("anode", 2.5, GXE, transparency[1]),
                             ("cathode", -495.0, LXE, transparency[2])):
        sid = len(surfs)
        surfs.append(Surface(f"{name}_T", ELECTRODE_T, transparency=T, wire_reflectivity=r_wire,
                             wire_spec_frac=wire_spec_frac))
        b.add(_fan(wall2, ze, (0, 0)), (0, 0, 1), mat, mat, sid)
    _pmt_windows(b, bot, z_bot, thick, +1, r_w, r_pc, k_seg, LXE, S_CAP, S_PC, 0)
    _pmt_windows(b, top, z_top, thick, -1, r_w, r_pc, k_seg, GXE, S_CAP, S_PC, len(bot))
    src = Source(SRC_VOLUME_POLYGON, LXE, n_sides=64, radius=R, z_min=z_bot, z_max=z_liq)
    return _detector("scaled_tpc", b, mats, surfs, bot, top, z_bot - thick, z_top + thick, src,
                     dict(radius=R, wall_sides=64, z_liquid=z_liq))


# ----------------------------------------------------------------------------
# small test geometries (worked examples of Sec. 3 and closed-form checks)
# ----------------------------------------------------------------------------
def layered_box(half=500.0, z_bot=-100.0, z_liq=0.0, z_win=5.0, thick=5.0, with_gas=True):
    """Sec. 3 first check: photons sent straight up through the LXe/GXe surface
    into a quartz window whose back face is a photocathode (channel 1, "top");
    the bottom of the LXe is a photocathode too (channel 0, "bottom"); black
    side walls.  No absorption or scattering, PDE = 1.  ``with_gas=False``
    removes the gas layer (LXe directly under the window)."""
    mats = [Material("LXe", 1.69), Material("GXe", 1.00), Material("quartz", 1.60), Material("opaque", 1.0)]
    surfs = [Surface("black", ABSORBER), Surface("photocathode", PHOTOCATHODE, qe=1.0)]
    b = _Builder()
    sq = np.array([[-half, -half], [half, -half], [half, half], [-half, half]], np.float64)
    z_pc = z_win + thick
    # bottom photocathode (channel 0): faces up into the LXe
    b.add(_fan(sq, z_bot, (0, 0)), (0, 0, -1), LXE, OPAQUE, 1, 0)
    if with_gas:
        b.add(_fan(sq, z_liq, (0, 0)), (0, 0, 1), LXE, GXE)
        b.add(_fan(sq, z_win, (0, 0)), (0, 0, -1), QUARTZ, GXE)
        _wall(b, sq, z_bot, z_liq, LXE, 0)
        _wall(b, sq, z_liq, z_win, GXE, 0)
    else:
        b.add(_fan(sq, z_win, (0, 0)), (0, 0, -1), QUARTZ, LXE)
        _wall(b, sq, z_bot, z_win, LXE, 0)
    _wall(b, sq, z_win, z_pc, QUARTZ, 0)
    b.add(_fan(sq, z_pc, (0, 0)), (0, 0, 1), QUARTZ, OPAQUE, 1, 1)
    verts, tris, mi, mo, sf, ch = b.finish()
    src = Source(SRC_POINT, LXE, center=(0.0, 0.0, 0.5 * (z_bot + z_liq)))
    return Detector("layered_box", verts, tris, mi, mo, sf, ch, mats, surfs,
                    np.array([0, 1], np.int32), np.array([[0, 0, z_bot], [0, 0, z_pc]], np.float32), src,
                    dict(z_liquid=z_liq, z_window=z_win))


def icosphere(radius=100.0, subdiv=5, surface_type=PHOTOCATHODE, abs_len_mm=INF, ray_len_mm=INF, n_medium=1.0):
    """Closed triangulated sphere (20 * 4**subdiv triangles) filled with one
    medium; its inside is a photocathode (channel 0) with QE 1, so every photon
    reaching it is counted.  Used for the survival and escape-fraction checks."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
                  [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5],
                  [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    for _ in range(subdiv):
        edges = np.sort(np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]]), 1)
        ue, inv = np.unique(edges, axis=0, return_inverse=True)
        mid = v[ue[:, 0]] + v[ue[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m = inv.reshape(3, -1).T + len(v)
        v = np.concatenate([v, mid])
        a, bb, c = f[:, 0], f[:, 1], f[:, 2]
        ab, bc, ca = m[:, 0], m[:, 1], m[:, 2]
        f = np.concatenate([np.stack([a, ab, ca], 1), np.stack([bb, bc, ab], 1),
                            np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)])
    tri = v[f] * radius
    mats = [Material("medium", n_medium, abs_len_mm, ray_len_mm), Material("opaque", 1.0)]
    surfs = [Surface("sensor", surface_type, reflectivity=0.0, qe=1.0)]
    b = _Builder()
    b.add(tri, tri.mean(1), 0, 1, 0, 0)
    verts, tris, mi, mo, sf, ch = b.finish()
    src = Source(SRC_POINT, 0, center=(0.0, 0.0, 0.0))
    return Detector("icosphere", verts, tris, mi, mo, sf, ch, mats, surfs, np.array([0], np.int32),
                    np.zeros((1, 3), np.float32), src, dict(radius=radius))


def random_soup(n_tris, seed=0, extent=100.0, size=20.0):
    """Random triangles in a cube (for intersection tests): float32 vertices
    on the snap grid, attributes zero."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-extent, extent, (n_tris, 1, 3))
    tri = c + rng.uniform(-size, size, (n_tris, 3, 3))
    verts = (_snap(tri).reshape(-1, 3)).astype(np.float32)
    tris = np.arange(3 * n_tris, dtype=np.uint32).reshape(-1, 3)
    z8 = np.zeros(n_tris, np.uint8)
    return Detector("soup", verts, tris, z8, z8.copy(), np.full(n_tris, SURF_NONE, np.uint16),
                    np.full(n_tris, -1, np.int32), [Material("m", 1.0)], [], np.zeros(0, np.int32),
                    np.zeros((0, 3), np.float32), Source(SRC_POINT, 0))


def closed_edges_ok(det: Detector, mask=None) -> bool:
    """True if every edge of the selected triangles is shared by exactly two of
    them (a closed, conforming surface)."""
    t = det.tris if mask is None else det.tris[mask]
    e = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]).astype(np.int64), 1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    return bool(np.all(cnt == 2))


def electrode_box(transparency=0.9, r_wire=0.3, wire_spec_frac=0.0, half=500.0, z_bot=-100.0, z_el=0.0,
                  z_top=100.0, mat_n=1.69):
    """LXe box with photocathodes (QE 1) as floor (channel 0) and ceiling
    (channel 1), black side walls and one thin effective-transparency
    electrode plane at ``z_el`` (the Geant4 electrode model, Sec. 2.1)."""
    mats = [Material("LXe", mat_n), Material("opaque", 1.0)]
    surfs = [Surface("black", ABSORBER), Surface("photocathode", PHOTOCATHODE, qe=1.0),
             Surface("electrode", ELECTRODE_T, transparency=transparency, wire_reflectivity=r_wire,
                     wire_spec_frac=wire_spec_frac)]
    sq = np.array([[-half, -half], [half, -half], [half, half], [-half, half]], np.float64)
    b = _Builder()
    b.add(_fan(sq, z_bot, (0, 0)), (0, 0, -1), 0, 1, 1, 0)
    b.add(_fan(sq, z_top, (0, 0)), (0, 0, 1), 0, 1, 1, 1)
    b.add(_fan(sq, z_el, (0, 0)), (0, 0, 1), 0, 0, 2)
    _wall(b, sq, z_bot, z_el, 0, 0)
    _wall(b, sq, z_el, z_top, 0, 0)
    verts, tris, mi, mo, sf, ch = b.finish()
    mo[mo == OPAQUE] = 1
    src = Source(SRC_POINT, 0, center=(0.0, 0.0, 0.5 * (z_bot + z_el)))
    return Detector("electrode_box", verts, tris, mi, mo, sf, ch, mats, surfs, np.array([0, 1], np.int32),
                    np.array([[0, 0, z_bot], [0, 0, z_top]], np.float32), src, dict())


def reflector_box(reflectivity=0.8, spec_frac=1.0, half=500.0, z_bot=-100.0, z_top=100.0, mat_n=1.69):
    """LXe box with a reflecting floor (surface 1), a photocathode ceiling with
    QE 1 (channel 0) and black side walls; for the reflectivity checks."""
    mats = [Material("LXe", mat_n), Material("opaque", 1.0)]
    surfs = [Surface("black", ABSORBER), Surface("floor", REFLECTOR, reflectivity, spec_frac),
             Surface("photocathode", PHOTOCATHODE, qe=1.0)]
    sq = np.array([[-half, -half], [half, -half], [half, half], [-half, half]], np.float64)
    b = _Builder()
    b.add(_fan(sq, z_bot, (0, 0)), (0, 0, -1), 0, 1, 1)
    b.add(_fan(sq, z_top, (0, 0)), (0, 0, 1), 0, 1, 2, 0)
    _wall(b, sq, z_bot, z_top, 0, 0)
    verts, tris, mi, mo, sf, ch = b.finish()
    mo[mo == OPAQUE] = 1
    src = Source(SRC_POINT, 0, center=(0.0, 0.0, 0.0))
    return Detector("reflector_box", verts, tris, mi, mo, sf, ch, mats, surfs, np.array([1], np.int32),
                    np.array([[0, 0, z_top]], np.float32), src, dict())


def darwin_events(seed=0, n_s1=4096, n_s2=512, s1_range=(1e2, 1e5), s2_range=(1e5, 1e6), radius=1300.0,
                  z_active=(-2597.0, -1.0), z_gap=(2.01, 7.85)):
    """Batched events in the DARWIN-scale detector: S1-like point sources
    uniform in the active LXe (inside the 24-gon, z in z_active) with photon
    counts log-uniform in s1_range, and S2-like sources uniform along a
    vertical segment in the gas gap between the liquid surface (z = +2) and
    the anode (z = +8) at (x, y) uniform in the 24-gon, photon counts
    log-uniform in s2_range (Sec. 1: S1 scintillation at the interaction
    point, S2 light in the gas).  Returns a list of (Source, n_photons)."""
    rng = np.random.default_rng(seed)
    poly = polygon_vertices(24, radius)

    def xy(n):
        out = []
        while len(out) < n:
            p = rng.uniform(-radius, radius, (2 * n, 2))
            out.extend(p[_inside_convex(p, poly, margin=1.0)].tolist())
        return np.array(out[:n])

    ev = []
    p1 = xy(n_s1)
    z1 = rng.uniform(*z_active, n_s1)
    c1 = np.exp(rng.uniform(np.log(s1_range[0]), np.log(s1_range[1]), n_s1)).astype(np.int64)
    for (x, y), z, n in zip(p1, z1, c1):
        ev.append((Source(SRC_POINT, LXE, center=(float(x), float(y), float(z))), int(n)))
    p2 = xy(n_s2)
    c2 = np.exp(rng.uniform(np.log(s2_range[0]), np.log(s2_range[1]), n_s2)).astype(np.int64)
    for (x, y), n in zip(p2, c2):
        ev.append((Source(SRC_SEGMENT, GXE, center=(float(x), float(y), z_gap[0]),
                          p1=(float(x), float(y), z_gap[1])), int(n)))
    return ev


def calibration_sources(n_photons, n_x=16, n_z=16, spacing=100.0, z_center=-1299.0, medium=LXE):
    """Point sources for a calibration fit: an n_x by n_z grid with ``spacing``
    mm pitch in the vertical plane y = 0, centred on (0, 0, z_center), each
    emitting ``n_photons`` isotropically (the LCE(R, Z) maps of Sec. 3 sample
    the active volume on such a grid).  The defaults give 256 sources on a
    10 cm grid around the middle of the DARWIN-scale drift volume.  Returns a
    list of (Source, n_photons)."""
    xs = (np.arange(n_x) - (n_x - 1) / 2.0) * spacing
    zs = z_center + (np.arange(n_z) - (n_z - 1) / 2.0) * spacing
    return [(Source(SRC_POINT, medium, center=(float(x), 0.0, float(z))), int(n_photons)) for z in zs for x in xs]


def grid_sources(det, n_photons, n_sources=256, spacing=100.0, margin=50.0, seed=0, medium=LXE):
    """Point sources for a calibration fit on a 3-D grid: the nodes of a
    cubic grid of pitch ``spacing`` (mm, aligned with the origin) inside the
    detector's active volume -- the regular-polygon prism of its volume
    source (the LXe between cathode and gate inside the wall) -- at least
    ``margin`` mm from every wall side and from the prism's bottom and top;
    a seeded random subset of ``n_sources`` of them (all if fewer), each
    emitting ``n_photons``.  The DARWIN-scale detector has about 12 000 such
    nodes at 10 cm.  Returns a list of (Source, n_photons), ordered by
    (z, y, x)."""
    s = det.source
    if s.kind != SRC_VOLUME_POLYGON:
        raise ValueError("grid_sources needs a detector whose source is its active volume (a polygon prism)")
    n = max(int(s.n_sides), 3) if s.n_sides else 0
    r_out = float(s.radius)
    ext = r_out + spacing
    ax = np.arange(np.floor(-ext / spacing), np.ceil(ext / spacing) + 1) * spacing
    az = np.arange(np.ceil((s.z_min + margin) / spacing), np.floor((s.z_max - margin) / spacing) + 1) * spacing
    z, y, x = np.meshgrid(az, ax, ax, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    if n:
        apothem = r_out * math.cos(math.pi / n)
        ok = np.ones(x.size, bool)
        for k in range(n):   # side k's outward normal, half-way between vertices k and k + 1
            a = s.phase + 2.0 * math.pi * (k + 0.5) / n
            ok &= x * math.cos(a) + y * math.sin(a) <= apothem - margin
    else:
        ok = x * x + y * y <= (r_out - margin) ** 2
    x, y, z = x[ok], y[ok], z[ok]
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(x.size, min(n_sources, x.size), replace=False))
    return [(Source(SRC_POINT, medium, center=(float(x[i]), float(y[i]), float(z[i]))), int(n_photons))
            for i in pick]
