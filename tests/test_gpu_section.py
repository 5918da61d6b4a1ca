"""GPU parity on the curved C-section spar: general hexahedra with per-element
ply frames, explicit subdomain boxes, geometric 3-2-1 pins on floating curved
subdomains and the end-face load on curved quads, against the FP64 oracle
(eigenvalues 1e-8 / mixed 1e-5 relative, eigenvector spans at spectral gaps,
coarse dimension exact, energy error within 1 % of the oracle's)."""
import pytest

from test_gpu_local import run_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["s1", "s2"])
def test_section_parity_fp64(name):
    run_case(name)


@pytest.mark.parametrize("name", ["s1", "s2"])
def test_section_parity_mixed(name):
    run_case(name, precision=1, tol_lam=1e-5, tol_angle=1e-4)
