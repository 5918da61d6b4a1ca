"""Relative L2 errors of the displacement and strain fields (Sec. 5.4).

The paper measures a coarse approximation u_H against the fine-scale u_h by

    e_d   = ||u_h - u_H||_2 / ||u_h||_2,
    e_eps = ||eps(u_h) - eps(u_H)||_2 / ||eps(u_h)||_2.

It does not say whether ||.||_2 is the Euclidean norm of the DoF vector or the
norm of L2(Omega).  Here it is the L2(Omega) norm of the finite element fields:
each element's integral of |v|^2 (displacement) and of eps(v) : eps(v) (strain,
the Frobenius norm of the symmetric gradient, i.e. shear components counted
as tensor entries, not engineering strains), by 2x2x2 Gauss-Legendre
quadrature through the trilinear map of the element's corners.  The rule is
exact for the squared displacement on bricks and on the extruded elements of
the C-section, whose Jacobian determinant is linear in each in-plane reference
coordinate (the integrand stays of degree 3 in each variable).

Test infrastructure: this module is imported by tests only.
"""
import numpy as np

from .element import gauss_points, shape_gradients_ref, shape_values


def _corners_and_dofs(mesh):
    NX, NY, NZ = mesh.NX, mesh.NY, mesh.NZ
    ii, jj, kk = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    nodes = mesh.element_nodes(ii, jj, kk)                 # (ne, 8), CORNERS order
    X = mesh.coords(nodes.ravel()).reshape(nodes.shape + (3,))
    return X, nodes


def field_norms(mesh, v):
    """(int |v|^2 dx, int eps(v) : eps(v) dx) of the nodal field v (3 per node)."""
    X, nodes = _corners_and_dofs(mesh)
    vals = np.asarray(v, dtype=np.float64).reshape(-1, 3)[nodes]       # (ne, 8, 3)
    pts, wts = gauss_points(2)
    disp = np.zeros(len(X))
    strain = np.zeros(len(X))
    for xi, w in zip(pts, wts):
        dN_dxi = shape_gradients_ref(xi)                   # (8, 3)
        N = shape_values(xi)                               # (8,)
        J = np.einsum("eai,ar->eir", X, dN_dxi)            # dx_i / dxi_r
        detJ = np.linalg.det(J)
        dN_dx = np.einsum("ar,eri->eai", dN_dxi, np.linalg.inv(J))
        u = np.einsum("a,eac->ec", N, vals)
        G = np.einsum("eac,eaj->ecj", vals, dN_dx)        # du_c / dx_j
        eps = 0.5 * (G + np.transpose(G, (0, 2, 1)))
        disp += w * detJ * np.einsum("ec,ec->e", u, u)
        strain += w * detJ * np.einsum("eij,eij->e", eps, eps)
    return disp.sum(), strain.sum()


def l2_errors(mesh, u_ref, u):
    """(e_d, e_eps) of the approximation u against the reference u_ref."""
    u_ref = np.asarray(u_ref, dtype=np.float64)
    d0, s0 = field_norms(mesh, u_ref - np.asarray(u, dtype=np.float64))
    d1, s1 = field_norms(mesh, u_ref)
    return np.sqrt(d0 / d1), np.sqrt(s0 / s1)

