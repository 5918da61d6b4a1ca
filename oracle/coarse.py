"""MS-GFEM coarse space, coarse Galerkin problem and energy error.

Sec. 4.3-4.4: each local eigenvector is multiplied by the partition of unity
(Xi_j phi = D_mu phi, extended by zero, Eq. AHarmonic_coarse_space); the
weighted vectors are re-orthogonalised by Gram-Schmidt; the PoU-weighted
particular function Xi_j psi_j is Gram-Schmidt orthogonalised against them,
normalised and appended.  The Gram-Schmidt inner product is a(., .), which on
PoU-weighted vectors (zero on the cut boundary of Omega_j) equals
a_{Omega*_j}; the paper does not name the inner product, and the coarse span,
hence u^G, does not depend on it.

Coarse problem (Eq. GFEM_coarse_approximation): A^H = V^T A V, b^H = V^T b,
u^G = V c.  ``variant="ii"`` is the paper's implementation (psi appended to
the basis, Sec. 4.4); ``variant="i"`` is the theory form u^G = u^p + u_H with
u^p = sum_j R_j^T Xi_j psi_j fixed (Eqs. global_particular_function,
GFEM_coarse_approximation).  The energy error is ||u_h - u^G||_a / ||u_h||_a
with ||v||_a = sqrt(a(v, v)) (Theorem 1).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from workloads import element_angles

from .arpack import local_eigs_arpack
from .assemble import assemble_global, make_cache
from .fine import energy_norm, solve_fine
from .local import local_eigs_dense, local_problem, particular
from .mesh import make_mesh
from .partition import partition_of_unity, subdomains


def gram_schmidt(A, vectors, drop_tol=1e-10):
    """Modified Gram-Schmidt (two passes) in the inner product u^T A v; a vector
    whose A-norm falls below drop_tol times its initial norm is dropped."""
    Q, AQ = [], []
    for v in vectors:
        v = v.copy()
        n0 = np.sqrt(max(v @ (A @ v), 0.0))
        if n0 == 0.0:
            continue
        for _ in range(2):
            for q, aq in zip(Q, AQ):
                v -= (aq @ v) * q
        Av = A @ v
        n = np.sqrt(max(v @ Av, 0.0))
        if n <= drop_tol * n0:
            continue
        Q.append(v / n)
        AQ.append(Av / n)
    return Q


def coarse_solve(AH, bH, rel_cut=1e-14):
    """Cholesky of A^H; on a non-positive or tiny pivot, a symmetric eigen pseudo-inverse."""
    try:
        L = np.linalg.cholesky(AH)
        if np.min(np.diag(L)) ** 2 > rel_cut * np.max(np.diag(AH)):
            return sla.cho_solve((L, True), bH)
    except np.linalg.LinAlgError:
        pass
    w, U = np.linalg.eigh(AH)
    keep = w > rel_cut * w.max()
    return U[:, keep] @ ((U[:, keep].T @ bH) / w[keep])


@dataclass
class MSGFEMResult:
    lam: list = field(default_factory=list)        # per subdomain, ascending
    phi: list = field(default_factory=list)        # per subdomain, local DoFs x n_loc
    basis_counts: list = field(default_factory=list)
    V: sp.csc_matrix = None
    AH: np.ndarray = None
    bH: np.ndarray = None
    uG: np.ndarray = None
    uh: np.ndarray = None
    energy_error: float = None
    A: sp.csr_matrix = None
    b: np.ndarray = None
    problems: list = field(default_factory=list)


def run_msgfem(cfg, angles=None, n_loc=None, variant="ii", solver="dense", uh=None,
               keep_problems=False, threshold=None, load=None):
    """MS-GFEM with n_loc eigenvectors per subdomain, or, with ``threshold`` t,
    the eigenvectors with 1 / lambda > t among the n_loc computed (Sec. 5.5,
    Sec. 5.6: the local basis sizes m_j follow from a threshold on the
    reciprocal eigenvalues).  n_loc may also be a sequence with one count per
    subdomain: the m_j of Eq. AHarmonic_coarse_space chosen for each subdomain
    (Sec. 5.3: interior subdomains need more eigenvectors).  ``load``: nodal
    forces replacing the end-face traction as the right-hand side b."""
    mesh = make_mesh(cfg)
    E = cfg.material
    if angles is None:
        angles = element_angles(cfg)
    n_loc = cfg.n_loc if n_loc is None else n_loc
    cache = make_cache(mesh, E)
    A = assemble_global(mesh, angles, E, cache=cache)
    b = mesh.compression_load(cfg.traction) if load is None else np.asarray(load, dtype=np.float64).copy()
    subs = subdomains(cfg)
    mus = partition_of_unity(mesh, subs, cfg.overlap)
    res = MSGFEMResult(A=A, b=b)
    cols, up = [], np.zeros(mesh.n_dof)
    eig = local_eigs_dense if solver == "dense" else local_eigs_arpack
    for s in subs:
        lp = local_problem(mesh, angles, E, s, mus[s.index], b, cache=cache)
        lam, phi = eig(lp, n_loc if np.ndim(n_loc) == 0 else int(n_loc[s.index]))
        psi = particular(lp)
        res.lam.append(lam)
        res.phi.append(phi)
        if keep_problems:
            res.problems.append(lp)
        m_j = phi.shape[1]
        if threshold is not None:
            m_j = int(np.sum(lam * threshold < 1.0))
        weighted = [lp.mu * phi[:, k] for k in range(m_j)]
        psi_w = lp.mu * psi
        if variant == "ii":
            vecs = weighted + ([psi_w] if np.any(psi_w != 0.0) else [])
        else:
            vecs = weighted
            gd = (3 * lp.nodes[:, None] + np.arange(3)).ravel()
            up[gd] += psi_w
        Q = gram_schmidt(lp.A, vecs)
        res.basis_counts.append(len(Q))
        gd = (3 * lp.nodes[:, None] + np.arange(3)).ravel()
        for q in Q:
            col = np.zeros(mesh.n_dof)
            col[gd] = q
            cols.append(col)
    V = sp.csc_matrix(np.stack(cols, axis=1)) if cols else sp.csc_matrix((mesh.n_dof, 0))
    AH = (V.T @ (A @ V)).toarray() if V.shape[1] else np.zeros((0, 0))
    AH = 0.5 * (AH + AH.T)
    rhs = b - A @ up
    bH = V.T @ rhs
    c = coarse_solve(AH, bH) if V.shape[1] else np.zeros(0)
    res.V, res.AH, res.bH = V, AH, bH
    res.uG = up + V @ c
    if uh is None:
        uh = solve_fine(mesh, A, b)
    res.uh = uh
    res.energy_error = energy_norm(A, uh - res.uG) / energy_norm(A, uh)
    return res
