"""The A-harmonic local eigenproblem and the local particular function.

On Omega*_j with free DoFs F = B1 u B2 (B3 removed, phi_3 = 0), let
K = A_{Omega*}[F, F] with blocks A11, A12, A22 and B = D_mu A_{Omega*} D_mu,
which vanishes outside B1 x B1 because mu = 0 on B2 (Sec. 4.3).  The mixed
eigenproblem (Eq. bilinearAharmonic / Eq. algebraicAharmonic) constrains
phi to ker [A11 A12] = range E with E = [-A11^{-1} A12; I]; substituting
phi = E x and testing with E gives the reduced symmetric pencil

    S x = lambda T x,   S = E^T K E = A22 - A21 A11^{-1} A12,   T = E^T B E,

which is Eq. AHarmonicGeneralizeEigenProblem written on V_A.  Its n_loc
smallest eigenvalues and phi = E x (normalised phi^T B phi = 1) are wanted.

Dense-reduced solution: form S and T, Cholesky L L^T = S + sigma T
(sigma = 1e-2, SPD also on floating subdomains because T > 0 on rigid modes),
eigenvalues nu of L^{-1} T L^{-T}, lambda = 1/nu - sigma; each eigenvalue is
then reported as the Rayleigh quotient x^T S x / x^T T x of its vector.

Particular function (Eq. up_r): psi in V_{h,DI}: A11 psi_1 = b_1, psi_2 = 0,
psi_3 = 0; psi^d = 0 because the Dirichlet data are zero (Eq. up_d).
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assemble import assemble_box
from .partition import dof_classes


@dataclass
class LocalProblem:
    sub: object
    nodes: np.ndarray       # global node ids of Omega*_j
    n_star: int             # DoFs on Omega*_j
    I1: np.ndarray          # local DoF indices of B1
    I2: np.ndarray          # local DoF indices of B2
    I3: np.ndarray          # local DoF indices of B3
    A: sp.csr_matrix        # A_{Omega*_j} (all local DoFs)
    mu: np.ndarray          # PoU per local DoF
    b: np.ndarray           # restriction of the global load to local DoFs

    @property
    def A11(self):
        return self.A[self.I1][:, self.I1]

    @property
    def A12(self):
        return self.A[self.I1][:, self.I2]

    @property
    def A22(self):
        return self.A[self.I2][:, self.I2]

    @property
    def B11(self):
        d = sp.diags(self.mu[self.I1])
        return (d @ self.A11 @ d).tocsr()


def local_problem(mesh, angles, E, sub, mu_global, load, cache=None):
    nodes, b1, b2, b3 = dof_classes(mesh, sub)
    node_index = -np.ones(mesh.n_nodes, dtype=np.int64)
    node_index[nodes] = np.arange(len(nodes))
    n = 3 * len(nodes)
    A = assemble_box(mesh, angles, E, *sub.star, node_index=node_index, n_dof=n, cache=cache)

    def dofs(mask):
        return (3 * np.nonzero(mask)[0][:, None] + np.arange(3)).ravel()
    gd = (3 * nodes[:, None] + np.arange(3)).ravel()
    return LocalProblem(sub, nodes, n, dofs(b1), dofs(b2), dofs(b3), A,
                        np.repeat(mu_global[nodes], 3), load[gd].copy())


def _factor(M):
    return spla.splu(sp.csc_matrix(M), permc_spec="MMD_AT_PLUS_A")


def reduced_pencil(lp):
    """Dense S, T and P = A11^{-1} A12 of the reduced pencil."""
    lu = _factor(lp.A11)
    A12 = lp.A12.toarray()
    P = lu.solve(A12)
    S = lp.A22.toarray() - A12.T @ P
    T = P.T @ (lp.B11 @ P)
    return 0.5 * (S + S.T), 0.5 * (T + T.T), P


def extend(lp, P, X):
    """phi = E x on all local DoFs (B3 entries zero)."""
    phi = np.zeros((lp.n_star, X.shape[1]))
    phi[lp.I1] = -P @ X
    phi[lp.I2] = X
    return phi


def local_eigs_dense(lp, n_loc, sigma=1e-2):
    """n_loc smallest eigenpairs (lambda ascending, phi on local DoFs)."""
    n2 = len(lp.I2)
    if n2 == 0:
        return np.zeros(0), np.zeros((lp.n_star, 0))
    S, T, P = reduced_pencil(lp)
    L = np.linalg.cholesky(S + sigma * T)
    C = sla.solve_triangular(L, sla.solve_triangular(L, T, lower=True).T, lower=True)
    nu, Y = np.linalg.eigh(0.5 * (C + C.T))
    order = np.argsort(nu)[::-1][:min(n_loc, n2)]
    X = sla.solve_triangular(L.T, Y[:, order], lower=False)
    tn = np.einsum("ik,ik->k", X, T @ X)
    # nu = 0 (x in ker T) is lambda = infinity; such vectors vanish under the PoU
    inf = tn <= 1e-13 * tn.max()
    X = X / np.sqrt(np.where(inf, np.einsum("ik,ik->k", X, X), tn))
    lam = np.where(inf, np.inf, np.einsum("ik,ik->k", X, S @ X))
    srt = np.argsort(lam)
    return lam[srt], extend(lp, P, X[:, srt])


def particular(lp):
    """psi_j on local DoFs: A11 psi_1 = b_1 and zero on B2, B3."""
    psi = np.zeros(lp.n_star)
    b1 = lp.b[lp.I1]
    if np.any(b1 != 0.0):
        psi[lp.I1] = _factor(lp.A11).solve(b1)
    return psi
