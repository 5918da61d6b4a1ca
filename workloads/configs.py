"""Workload descriptions for the laminated-beam problems.

Units: N, mm, MPa.  The beam occupies [0, NX*hx] x [0, NY*hy] x [0, NZ*t] with
one trilinear hexahedron per ply through the thickness (Sec. 5.1 of the paper
uses one element per ply).  The x = 0 face is clamped and the x = L face carries
a uniform compressive traction of magnitude ``traction`` (MPa).

Sizes are the ones of the five benchmark workloads:

* ``c1``  24 x 4 x 12 elements, 12 plies, 2 x 1 subdomains, overlap 1,
  oversampling 2, n_loc = 8.
* ``c2``  192 x 12 x 39 elements, 39 plies with 1 degree Gaussian ply noise,
  16 x 2 subdomains, overlap 2, oversampling 4, n_loc = 20.
* ``c3``  384 x 24 x 48 elements, 48 plies, 32 x 2 subdomains, overlap 2,
  oversampling 4, n_loc = 24 (mixed precision workload).
* ``c5``  the c1 beam with a per-sample wrinkle field of ply-angle
  perturbation (learned warm-start workload).

``p2`` has c2-sized subdomains but only six of them (profiling).
``a1``, ``a4``, ``a8``, ``a15``: the c1 topology with in-plane element edges of 1, 4, 8
and 15 ply thicknesses (the element aspect-ratio study of Sec. 5.3).
Smaller ``t*`` workloads are test cases that span several layers, ragged
partitions and both clamped and floating subdomains.
"""
from dataclasses import dataclass, field, replace
from typing import Tuple

# Orthotropic ply constants (MPa and dimensionless Poisson ratios):
# E11, E22, E33, G12, G13, G23, nu12, nu13, nu23.
_PLY = (162000.0, 10000.0, 10000.0, 5200.0, 5200.0, 3500.0, 0.35, 0.35, 0.5)


def material_constants() -> Tuple[float, ...]:
    """The nine engineering constants (E11, E22, E33, G12, G13, G23, nu12, nu13, nu23)."""
    return _PLY


@dataclass(frozen=True)
class BeamConfig:
    name: str
    NX: int
    NY: int
    NZ: int
    hx: float = 2.0
    hy: float = 2.0
    t: float = 0.25              # ply (element) thickness
    sx: int = 2                  # subdomains along x
    sy: int = 1                  # subdomains along y
    overlap: int = 1             # o: element layers added to each non-overlapping box
    oversampling: int = 2        # o*: element layers, counted from the non-overlapping box
    n_loc: int = 8               # eigenvectors per subdomain
    layup_seed: int = 0          # offset into the (0, 90, 45, -45) cycle
    noise_sd_deg: float = 0.0    # per-ply Gaussian angle noise
    noise_seed: int = 1
    traction: float = 1.0        # compressive traction on x = L (MPa)
    material: Tuple[float, ...] = field(default=_PLY)

    @property
    def n_nodes(self) -> int:
        return (self.NX + 1) * (self.NY + 1) * (self.NZ + 1)

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes

    @property
    def n_sub(self) -> int:
        return self.sx * self.sy

    def with_(self, **kw) -> "BeamConfig":
        return replace(self, **kw)


CONFIGS = {
    "c1": BeamConfig("c1", 24, 4, 12, sx=2, sy=1, overlap=1, oversampling=2, n_loc=8),
    "c2": BeamConfig("c2", 192, 12, 39, sx=16, sy=2, overlap=2, oversampling=4, n_loc=20,
                     noise_sd_deg=1.0, noise_seed=1),
    "c3": BeamConfig("c3", 384, 24, 48, sx=32, sy=2, overlap=2, oversampling=4, n_loc=24),
    "c5": BeamConfig("c5", 24, 4, 12, sx=2, sy=1, overlap=1, oversampling=2, n_loc=8),
    # profiling case: c2-sized subdomains (one interior), six subdomains in all
    "p2": BeamConfig("p2", 36, 12, 39, sx=3, sy=2, overlap=2, oversampling=4, n_loc=20,
                     noise_sd_deg=1.0, noise_seed=1),
    # test cases: a few layers, ragged partitions, clamped / floating / interior subdomains
    "t1": BeamConfig("t1", 8, 2, 3, sx=2, sy=1, overlap=1, oversampling=1, n_loc=6),
    "t2": BeamConfig("t2", 12, 4, 4, sx=3, sy=2, overlap=1, oversampling=2, n_loc=10),
    "t3": BeamConfig("t3", 20, 6, 6, sx=3, sy=2, overlap=1, oversampling=3, n_loc=12,
                     noise_sd_deg=1.0),
    "t4": BeamConfig("t4", 40, 6, 12, sx=4, sy=2, overlap=2, oversampling=4, n_loc=20,
                     noise_sd_deg=1.0),
}
# element aspect-ratio sweep (Sec. 5.3): in-plane element edge = aspect ratio x ply
# thickness, the c1 beam's topology, oversampling 4, the 8 smallest eigenpairs
ASPECT_RATIOS = (1, 4, 8, 15)
for _ar in ASPECT_RATIOS:
    CONFIGS[f"a{_ar}"] = BeamConfig(f"a{_ar}", 24, 4, 12, hx=0.25 * _ar, hy=0.25 * _ar, sx=2, sy=1, overlap=1,
                                    oversampling=4, n_loc=8)


def get_config(name: str):
    """A box-beam workload (``BeamConfig``) or a C-section one (``SectionConfig``)."""
    if name in CONFIGS:
        return CONFIGS[name]
    from .section import SECTIONS
    return SECTIONS[name]
