"""Element-wise assembly of the stiffness (Eq. element_stiffness) and of its
restriction a_D to a mesh-resolved subdomain D (Eq. restricted_bilinear_form).

All elements of the beam are congruent bricks, so the element matrix depends
only on the ply angle; it is computed once per distinct angle value.
"""
import numpy as np
import scipy.sparse as sp

from .element import brick_corners, hex_stiffness
from .material import rotated_tensor


class ElementCache:
    """K_e as a function of the fibre angle for the bricks of one mesh."""

    def __init__(self, mesh, E):
        self.mesh, self.E, self._cache = mesh, tuple(E), {}
        self.X = brick_corners(0.0, 0.0, 0.0, mesh.hx, mesh.hy, mesh.t)

    def __call__(self, theta):
        key = float(theta)
        if key not in self._cache:
            self._cache[key] = hex_stiffness(self.X, rotated_tensor(self.E, key))
        return self._cache[key]


def assemble_box(mesh, angles, E, ex0, ex1, ey0, ey1, node_index=None, n_dof=None, cache=None):
    """Stiffness a_D of the element box [ex0, ex1) x [ey0, ey1) x [0, NZ).

    ``angles`` has shape (NX, NY, NZ).  With ``node_index`` (global node id ->
    local id, -1 outside) the matrix is returned in that local numbering.
    """
    cache = cache or ElementCache(mesh, E)
    ii, jj, kk = np.meshgrid(np.arange(ex0, ex1), np.arange(ey0, ey1), np.arange(mesh.NZ), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    dofs = mesh.element_dofs(ii, jj, kk)                       # (ne, 24)
    if node_index is not None:
        nodes = dofs // 3
        dofs = 3 * node_index[nodes] + dofs % 3
        assert (dofs >= 0).all()
    th = angles[ii, jj, kk]
    rows, cols, vals = [], [], []
    for t in np.unique(th):
        sel = np.nonzero(th == t)[0]
        Ke = cache(t)
        d = dofs[sel]
        rows.append(np.repeat(d, 24, axis=1).ravel())
        cols.append(np.tile(d, (1, 24)).ravel())
        vals.append(np.broadcast_to(Ke.ravel(), (len(sel), 576)).ravel())
    n = n_dof if n_dof is not None else mesh.n_dof
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A.tocsr()


def assemble_global(mesh, angles, E, cache=None):
    return assemble_box(mesh, angles, E, 0, mesh.NX, 0, mesh.NY, cache=cache)
