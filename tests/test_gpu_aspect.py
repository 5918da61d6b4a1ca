"""The element aspect-ratio study (Sec. 5.3): in-plane element edges of 1, 4, 8
and 15 ply thicknesses on the c1 topology with oversampling 4, the 8 smallest
eigenpairs.  Flat elements raise the condition numbers of the local matrices,
which the paper observes to cost its ARPACK / sparse-LU eigensolves accuracy.
The GPU local stage is held to the same parity bars against the (dense, exact
up to rounding) oracle at every aspect ratio: every eigenvalue 1e-8 relative
in FP64 and 1e-5 in mixed precision, eigenvector spans at gaps, psi_j and u^G
in the energy norm, the energy error within 1 %.  Beyond n_loc = 8 the wanted
eigenvalues of the aspect-ratio-15 mesh span seven orders of magnitude (1/lambda
from 256 to 1.6e-5 at n_loc = 12) and the block Krylov solver stalls above its
tolerance (ENOCONV, also with 1000 block steps), the GPU counterpart of the
paper's plateau of 1/lambda at aspect ratios of 15 and more."""
import pytest

from test_gpu_local import run_case
from workloads.configs import ASPECT_RATIOS

pytestmark = pytest.mark.gpu


def _tol_res(ar):
    # the relative eigen-residual ||S x - lambda T x|| / (||S x|| + lambda ||T x||) of pairs
    # converged to the solver's energy-norm tolerance grows with the condition number; at
    # aspect ratio 15 it reaches ~5e-5 (the paper's loss of accuracy with flat elements)
    return 1e-4 if ar >= 15 else 1e-5


@pytest.mark.parametrize("ar", ASPECT_RATIOS)
def test_aspect_ratio_fp64(ar):
    run_case(f"a{ar}", tol_res=_tol_res(ar))


@pytest.mark.parametrize("ar", ASPECT_RATIOS)
def test_aspect_ratio_mixed(ar):
    run_case(f"a{ar}", precision=1, tol_lam=1e-5, tol_angle=1e-4, tol_res=_tol_res(ar))
