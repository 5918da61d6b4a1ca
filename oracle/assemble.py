"""Element-wise assembly of the stiffness (Eq. element_stiffness) and of its
restriction a_D to a mesh-resolved subdomain D (Eq. restricted_bilinear_form).

All elements of the box beam are congruent bricks, so the element matrix
depends only on the ply angle; it is computed once per distinct angle value.
On a general hexahedral mesh (the curved C-section) every element has its own
corners and ply frame; its matrix is computed from them, and elements whose
corners (up to a translation), frame and angle are identical share it.
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


class GeneralElementCache:
    """K_e of element (i, j, k) of a ``HexMesh``: its corners, frame and angle."""

    def __init__(self, mesh, E):
        self.mesh, self.E, self._cache = mesh, tuple(E), {}

    def element(self, i, j, k, theta):
        X = self.mesh.element_corners(i, j, k)
        F = self.mesh.frames[i, j, k]
        key = ((X - X[0]).tobytes(), F.tobytes(), float(theta))
        if key not in self._cache:
            self._cache[key] = hex_stiffness(X, rotated_tensor(self.E, float(theta), F))
        return self._cache[key]


def make_cache(mesh, E):
    return GeneralElementCache(mesh, E) if getattr(mesh, "general", False) else ElementCache(mesh, E)


def _assemble_general(mesh, angles, ii, jj, kk, dofs, n, cache):
    rows, cols, vals = [], [], []
    for e in range(len(ii)):
        Ke = cache.element(ii[e], jj[e], kk[e], angles[ii[e], jj[e], kk[e]])
        d = dofs[e]
        rows.append(np.repeat(d, 24))
        cols.append(np.tile(d, 24))
        vals.append(Ke.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A.tocsr()


def assemble_box(mesh, angles, E, ex0, ex1, ey0, ey1, node_index=None, n_dof=None, cache=None):
    """Stiffness a_D of the element box [ex0, ex1) x [ey0, ey1) x [0, NZ).

    ``angles`` has shape (NX, NY, NZ).  With ``node_index`` (global node id ->
    local id, -1 outside) the matrix is returned in that local numbering.
    """
    cache = cache or make_cache(mesh, E)
    ii, jj, kk = np.meshgrid(np.arange(ex0, ex1), np.arange(ey0, ey1), np.arange(mesh.NZ), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    dofs = mesh.element_dofs(ii, jj, kk)                       # (ne, 24)
    if node_index is not None:
        nodes = dofs // 3
        dofs = 3 * node_index[nodes] + dofs % 3
        assert (dofs >= 0).all()
    n = n_dof if n_dof is not None else mesh.n_dof
    if getattr(mesh, "general", False):
        return _assemble_general(mesh, angles, ii, jj, kk, dofs, n, cache)
    th = angles[ii, jj, kk]
    rows, cols, vals = [], [], []
    for t in np.unique(th):
        sel = np.nonzero(th == t)[0]
        Ke = cache(t)
        d = dofs[sel]
        rows.append(np.repeat(d, 24, axis=1).ravel())
        cols.append(np.tile(d, (1, 24)).ravel())
        vals.append(np.broadcast_to(Ke.ravel(), (len(sel), 576)).ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A.tocsr()


def assemble_global(mesh, angles, E, cache=None):
    return assemble_box(mesh, angles, E, 0, mesh.NX, 0, mesh.NY, cache=cache)
