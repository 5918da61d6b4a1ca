"""Trilinear hexahedron (Q1) stiffness.

a_e(u, v) = int_e sigma(u) : eps(v) dx (Eq. weak_form restricted to one element,
Eq. element_stiffness), evaluated with 2x2x2 Gauss-Legendre quadrature.  The
integrand is written with the fourth-order tensor directly,

    K[a i, b k] = sum_g sum_{j,l} C_ijkl dN_a/dx_j dN_b/dx_l det J w_g,

so no Voigt strain-displacement matrix is involved.  Local node a sits at the
reference corner ``CORNERS[a]``; local DoF index is 3 a + component.

The paper uses "reduced integration to avoid shear-locking" (Sec. 5.1) without
saying which; a uniform one-point rule makes the element rank-deficient and
the local problems singular, so full 2x2x2 integration is used here.
"""
import numpy as np

CORNERS = np.array([(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1),
                    (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1)], dtype=np.float64)


def shape_gradients_ref(xi):
    """dN_a/dxi_r at reference point xi for N_a = prod_r (1 + c_ar xi_r) / 8."""
    g = np.empty((8, 3))
    for a in range(8):
        c = CORNERS[a]
        f = 1.0 + c * xi
        g[a, 0] = c[0] * f[1] * f[2] / 8.0
        g[a, 1] = f[0] * c[1] * f[2] / 8.0
        g[a, 2] = f[0] * f[1] * c[2] / 8.0
    return g


def shape_values(xi):
    return np.array([np.prod(1.0 + CORNERS[a] * xi) / 8.0 for a in range(8)])


def gauss_points(n):
    x, w = np.polynomial.legendre.leggauss(n)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                pts.append((x[i], x[j], x[k]))
                wts.append(w[i] * w[j] * w[k])
    return np.array(pts), np.array(wts)


def hex_stiffness(X, C, order=2):
    """24x24 stiffness of a hexahedron with corner coordinates X (8x3) and tensor C."""
    K = np.zeros((8, 3, 8, 3))
    pts, wts = gauss_points(order)
    for xi, w in zip(pts, wts):
        dN_dxi = shape_gradients_ref(xi)
        J = X.T @ dN_dxi                       # J[i, r] = dx_i / dxi_r
        detJ = np.linalg.det(J)
        dN_dx = dN_dxi @ np.linalg.inv(J)      # dN_a/dx_j
        K += np.einsum("aj,ijkl,bl->aibk", dN_dx, C, dN_dx) * detJ * w
    return K.reshape(24, 24)


def brick_corners(x0, y0, z0, hx, hy, hz):
    """Corner coordinates of an axis-aligned brick in the ``CORNERS`` order."""
    base = np.array([x0, y0, z0])
    h = np.array([hx, hy, hz])
    return base + (CORNERS + 1.0) / 2.0 * h
