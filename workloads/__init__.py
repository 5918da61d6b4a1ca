"""Seeded synthetic inputs for the MS-GFEM local stage.

This package holds only workload descriptions and seeded random inputs
(laminate layups, ply-angle noise, wrinkle fields) and the geometry of the
curved C-section spar (node coordinates, ply frames, subdomain boxes).  It contains none of the
method's arithmetic: no stiffness, no partition of unity, no eigensolver.  It
is the one module shared by the CPU oracle (``oracle/``) and the GPU product
path (``paper_2211_13893_gb300``).
"""
from .configs import BeamConfig, CONFIGS, get_config, material_constants  # noqa: F401
from .generators import layup_angles, ply_angles, element_angles, wrinkle_field  # noqa: F401
from .section import SectionConfig, SECTIONS, section_nodes, section_frames  # noqa: F401
