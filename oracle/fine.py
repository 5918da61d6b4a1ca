"""Fine-scale FE solution u_h of A u = b with the clamped DoFs removed
(Eq. fe_matrix_system; h = 0, so u^p = 0 in Eq. bilinear).

The paper computes u_h with GenEO-preconditioned CG at a tight tolerance
(Sec. 5.3); here a direct factorisation is used instead, exact up to roundoff:
a banded Cholesky (LAPACK pbtrf through SciPy) in the natural node order, whose
bandwidth is 3 (NY+1)(NZ+1) + O(NZ).
"""
import numpy as np
import scipy.linalg as sla


def free_dofs(mesh):
    mask = np.ones(mesh.n_dof, dtype=bool)
    mask[mesh.dirichlet_dofs()] = False
    return np.nonzero(mask)[0]


def to_lower_banded(M):
    """LAPACK lower band storage ab[i - j, j] = M[i, j] of a symmetric sparse matrix."""
    C = M.tocoo()
    low = C.row >= C.col
    r, c, v = C.row[low], C.col[low], C.data[low]
    kd = int((r - c).max()) if len(r) else 0
    ab = np.zeros((kd + 1, M.shape[0]))
    np.add.at(ab, (r - c, c), v)
    return ab


def solve_fine(mesh, A, b):
    """u_h on all DoFs (zero on the clamped face)."""
    fd = free_dofs(mesh)
    Aff = A[fd][:, fd]
    ab = to_lower_banded(Aff)
    cb = sla.cholesky_banded(ab, lower=True)
    u = np.zeros(mesh.n_dof)
    u[fd] = sla.cho_solve_banded((cb, True), b[fd])
    return u


def energy_norm(A, v):
    return float(np.sqrt(max(v @ (A @ v), 0.0)))
