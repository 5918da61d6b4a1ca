"""Synthetic C-section spar: geometry, ply frames, layup and box partition.

The spar runs along x.  Its cross-section (in the y-z plane) is a C opening
toward +y: a web of height ``web`` between the inner faces of two flanges of
width ``flange`` (measured from the web's inner face), joined to the web by
quarter-circle corners of inner radius ``radius``.  The laminate of
``n_plies`` plies of thickness ``t`` grows outward from the inner surface.

The mesh is structured in index space, like the box beam: node (i, j, k) has
i along x (clamped face i = 0, loaded face i = NX), j along the arc length of
the cross-section (from the tip of the bottom flange to the tip of the top
flange) and k through the thickness (ply k between node layers k and k + 1).
Node (i, j, k) sits at (x_i, c_j + k t n_j), with c_j the j-th point of the
inner surface curve and n_j its outward unit normal there.  Corner nodes lie
on the circle arcs at equal angle steps, so the corners are refined by taking
a smaller arc step than on the straight segments.

Ply frames: every element carries three orthonormal axes, rows of a 3x3
array: a0 = the spar axis x (fibre direction at angle 0), a1 = the unit
tangent of the cross-section curve (fibre direction at angle 90), a2 = a0 x a1,
the outward laminate normal.  The tangent of an element is the chord of its
two inner-surface nodes (on an arc, the tangent at the mid angle).

This module holds geometry and seeded inputs only, none of the method's
arithmetic.  Units: N, mm, MPa.
"""
import math
from dataclasses import dataclass, field, replace
from typing import Tuple

import numpy as np

from .configs import material_constants
from .generators import layup_angles


@dataclass(frozen=True)
class SectionConfig:
    name: str
    length: float = 1000.0       # spar length along x
    web: float = 200.0           # web height between the flanges' inner faces
    flange: float = 60.0         # flange width from the web's inner face
    radius: float = 8.0          # inner corner radius
    n_plies: int = 32
    t: float = 0.25              # ply (element) thickness
    h_len: float = 4.0           # element size along x
    h_arc: float = 4.0           # element size along the straight segments
    h_corner: float = 1.0        # element size along the corner arcs (mid-surface)
    xparts: Tuple[int, ...] = ()     # element widths of the non-overlapping boxes along x
    sparts: Tuple[int, ...] = ()     # element widths along the arc
    overlap: int = 1
    oversampling: int = 3
    n_loc: int = 16
    n_loc_max: int = 0           # > n_loc: per-subdomain counts from n_loc to this (n_loc_per_subdomain)
    layup_seed: int = 0
    noise_sd_deg: float = 0.0    # per-ply Gaussian angle noise (as for the beams)
    noise_seed: int = 1
    traction: float = 1.0
    material: Tuple[float, ...] = field(default_factory=material_constants)
    kind: str = "section"

    # ---- mesh sizes
    @property
    def segments(self):
        """Element counts of (flange, corner, web, corner, flange) along the arc."""
        straight_f = self.flange - self.radius
        straight_w = self.web - 2.0 * self.radius
        arc_mid = 0.5 * math.pi * (self.radius + 0.5 * self.n_plies * self.t)
        nf = max(1, int(round(straight_f / self.h_arc)))
        nc = max(1, int(round(arc_mid / self.h_corner)))
        nw = max(1, int(round(straight_w / self.h_arc)))
        return (nf, nc, nw, nc, nf)

    @property
    def NX(self) -> int:
        return max(1, int(round(self.length / self.h_len)))

    @property
    def NY(self) -> int:
        return int(sum(self.segments))

    @property
    def NZ(self) -> int:
        return self.n_plies

    # box-beam attribute names, for code that reads them generically
    @property
    def hx(self) -> float:
        return self.length / self.NX

    @property
    def hy(self) -> float:
        return self.h_arc

    @property
    def n_nodes(self) -> int:
        return (self.NX + 1) * (self.NY + 1) * (self.NZ + 1)

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes

    @property
    def sx(self) -> int:
        return len(self.xparts)

    @property
    def sy(self) -> int:
        return len(self.sparts)

    @property
    def n_sub(self) -> int:
        return self.sx * self.sy

    @property
    def boxes(self):
        """Non-overlapping element boxes (x0, x1, y0, y1), subdomain a sy + b."""
        xc = np.concatenate([[0], np.cumsum(self.xparts)]).astype(int)
        yc = np.concatenate([[0], np.cumsum(self.sparts)]).astype(int)
        if xc[-1] != self.NX or yc[-1] != self.NY:
            raise ValueError(f"{self.name}: parts sum to {xc[-1]} x {yc[-1]}, mesh is {self.NX} x {self.NY}")
        return tuple((int(xc[a]), int(xc[a + 1]), int(yc[b]), int(yc[b + 1]))
                     for a in range(self.sx) for b in range(self.sy))

    def with_(self, **kw) -> "SectionConfig":
        return replace(self, **kw)


def _inner_curve(cfg):
    """Points c_j (y, z) of the inner surface and outward normals n_j, j = 0..NY."""
    nf, nc, nw, _, _ = cfg.segments
    F, W, r = cfg.flange, cfg.web, cfg.radius
    pts, nrm = [], []

    def add(p, n):
        pts.append(p)
        nrm.append(n)
    # bottom flange: tip (F, -W/2) toward the corner start (r, -W/2); normal -z
    for a in range(nf):
        add((F + (r - F) * a / nf, -0.5 * W), (0.0, -1.0))
    # bottom corner: centre (r, -W/2 + r), angle -pi/2 -> -pi
    cy, cz = r, -0.5 * W + r
    for a in range(nc):
        ph = -0.5 * math.pi - 0.5 * math.pi * a / nc
        add((cy + r * math.cos(ph), cz + r * math.sin(ph)), (math.cos(ph), math.sin(ph)))
    # web: (0, -W/2 + r) -> (0, W/2 - r); normal -y
    for a in range(nw):
        add((0.0, -0.5 * W + r + (W - 2.0 * r) * a / nw), (-1.0, 0.0))
    # top corner: centre (r, W/2 - r), angle pi -> pi/2
    cy, cz = r, 0.5 * W - r
    for a in range(nc):
        ph = math.pi - 0.5 * math.pi * a / nc
        add((cy + r * math.cos(ph), cz + r * math.sin(ph)), (math.cos(ph), math.sin(ph)))
    # top flange: (r, W/2) -> tip (F, W/2); normal +z, last node included
    for a in range(nf + 1):
        add((r + (F - r) * a / nf, 0.5 * W), (0.0, 1.0))
    return np.array(pts, dtype=np.float64), np.array(nrm, dtype=np.float64)


def section_nodes(cfg) -> np.ndarray:
    """Node coordinates, shape (NX + 1, NY + 1, NZ + 1, 3)."""
    c, n = _inner_curve(cfg)
    x = cfg.length * np.arange(cfg.NX + 1) / cfg.NX
    k = np.arange(cfg.NZ + 1) * cfg.t
    out = np.empty((cfg.NX + 1, cfg.NY + 1, cfg.NZ + 1, 3))
    out[..., 0] = x[:, None, None]
    out[..., 1] = (c[:, 0][None, :, None] + k[None, None, :] * n[:, 0][None, :, None])
    out[..., 2] = (c[:, 1][None, :, None] + k[None, None, :] * n[:, 1][None, :, None])
    return out


def section_frames(cfg) -> np.ndarray:
    """Ply frames per element, shape (NX, NY, NZ, 3, 3); rows a0, a1, a2."""
    c, _ = _inner_curve(cfg)
    d = c[1:] - c[:-1]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    fr = np.zeros((cfg.NY, 3, 3))
    fr[:, 0, 0] = 1.0
    fr[:, 1, 1], fr[:, 1, 2] = d[:, 0], d[:, 1]
    fr[:, 2, 1], fr[:, 2, 2] = -d[:, 1], d[:, 0]
    return np.broadcast_to(fr[None, :, None], (cfg.NX, cfg.NY, cfg.NZ, 3, 3)).copy()


def omega_star_sizes(cfg):
    """DoFs of every oversampling box (node box of the grown element box x full thickness)."""
    out = []
    for (x0, x1, y0, y1) in cfg.boxes:
        m = cfg.oversampling
        a0, a1 = max(0, x0 - m), min(cfg.NX, x1 + m)
        b0, b1 = max(0, y0 - m), min(cfg.NY, y1 + m)
        out.append(3 * (a1 - a0 + 1) * (b1 - b0 + 1) * (cfg.NZ + 1))
    return np.array(out)


def n_loc_per_subdomain(cfg):
    """Eigenpairs per subdomain: cfg.n_loc everywhere, or, with n_loc_max above
    it, counts growing linearly with the oversampling domain's DoF count from
    n_loc (the smallest domain) to n_loc_max (the largest), rounded to the
    nearest integer.  Interior subdomains need more eigenvectors for the same
    local error (Sec. 5.3), and the domains cut short by the clamped end, the
    free end or a flange tip are the small ones."""
    sizes = omega_star_sizes(cfg)
    if cfg.n_loc_max <= cfg.n_loc or sizes.max() == sizes.min():
        return np.full(len(sizes), cfg.n_loc, dtype=np.int32)
    frac = (sizes - sizes.min()) / float(sizes.max() - sizes.min())
    return (cfg.n_loc + np.floor((cfg.n_loc_max - cfg.n_loc) * frac + 0.5)).astype(np.int32)


SECTIONS = {
    # C-section spar of 1 m: web 200 mm, flanges 60 mm, inner radius 8 mm, 32 plies
    # of 0.25 mm; 4 mm elements along x and the straight segments, ~1 mm on the
    # corner arcs (19 per corner): 250 x 110 x 32 elements, 2,758,239 DoF.
    # 16 x 16 boxes, graded along x (1 element at the clamped end, ~21 in the
    # span) and along the arc (short boxes at the flange tips, three per corner,
    # six on the web); overlap 1, oversampling 3: oversampling domains of
    # 4,455 to 41,580 DoF (mean 29,570); 16 to 31 eigenpairs per subdomain,
    # growing with the domain's size.
    "c4": SectionConfig("c4", xparts=(1, 2, 4, 8, 12, 20, 20, 20, 20, 21, 21, 21, 21, 21, 21, 17),
                        sparts=(5, 8, 7, 6, 6, 8, 7, 8, 8, 7, 8, 6, 6, 7, 8, 5), n_loc=16, n_loc_max=31),
    # test sections: curved corners, clamped / floating / interior subdomains
    "s1": SectionConfig("s1", length=24.0, web=12.0, flange=8.0, radius=2.0, n_plies=4, t=0.5,
                        h_len=3.0, h_arc=2.0, h_corner=1.0, xparts=(3, 5), sparts=(5, 5, 5, 5),
                        overlap=1, oversampling=2, n_loc=8),
    "s2": SectionConfig("s2", length=40.0, web=16.0, flange=10.0, radius=3.0, n_plies=6, t=0.5,
                        h_len=2.5, h_arc=2.0, h_corner=1.0, xparts=(4, 4, 8), sparts=(6, 8, 7, 6),
                        overlap=1, oversampling=3, n_loc=12, noise_sd_deg=1.0),
}
