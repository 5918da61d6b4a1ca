"""The GenEO local eigenproblem and coarse space (Sec. 2.3), the comparison
method of the paper: no oversampling and no A-harmonic constraint.

On Omega_j with its free DoFs F (the clamped face removed), the local
problem of Eq. bilinearGeneralizeEigenProblem,

    a_{Omega_j}(phi, v) = lambda a_{Omega_j}(Xi_j phi, Xi_j v)   for all v,

is K phi = lambda B phi with K = A_{Omega_j}[F, F] (Neumann on the cut
boundary) and B = D_mu K D_mu.  The partition of unity vanishes on the cut
boundary C of Omega_j and is positive on the other free DoFs I, so B lives on
I x I; the C rows give phi_C = -K_CC^{-1} K_CI phi_I and the problem becomes
the symmetric definite pencil

    (K_II - K_IC K_CC^{-1} K_CI) phi_I = lambda B_II phi_I,

B_II = D_mu K_II D_mu being positive definite (K_II is K with C clamped).  Its
smallest eigenpairs are wanted (six zeros, the rigid motions, on a subdomain
away from the clamped face).  The coarse space is Eq. coarse_space,
V_H = span{R_j^T Xi_j phi_{j,k}}, and the coarse approximation the Galerkin
projection onto it (Sec. 2.4: GenEO used as a GFEM), without a particular
function.

The local problem reuses the MS-GFEM local problem of oracle.local with the
oversampling domain taken equal to Omega_j: its B1 is I and its B2 is C.
Test infrastructure: imported by tests only.
"""
from dataclasses import replace

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from workloads import element_angles

from .assemble import assemble_global, make_cache
from .coarse import coarse_solve, gram_schmidt
from .fine import energy_norm, solve_fine
from .local import _factor, local_problem
from .mesh import make_mesh
from .partition import partition_of_unity, subdomains


def geneo_problem(mesh, angles, E, sub, mu_global, load, cache=None):
    """The local problem on Omega_j (a LocalProblem with star = omega)."""
    return local_problem(mesh, angles, E, replace(sub, star=sub.omega), mu_global, load, cache)


def geneo_eigs(gp, n_loc):
    """n_loc smallest eigenpairs (lambda ascending, phi on the local DoFs of
    Omega_j, normalised phi^T B phi = 1)."""
    I, Cb = gp.I1, gp.I2
    KII = gp.A[I][:, I].toarray()
    if len(Cb):
        KIC = gp.A[I][:, Cb]
        Y = _factor(gp.A[Cb][:, Cb]).solve(KIC.T.toarray())        # K_CC^{-1} K_CI
        S = KII - KIC @ Y
    else:
        Y = np.zeros((0, len(I)))
        S = KII
    S = 0.5 * (S + S.T)
    d = gp.mu[I]
    B = d[:, None] * KII * d[None, :]
    k = min(n_loc, len(I))
    lam, X = sla.eigh(S, 0.5 * (B + B.T), subset_by_index=[0, k - 1])
    phi = np.zeros((gp.n_star, k))
    phi[I] = X
    phi[Cb] = -Y @ X
    return lam, phi


def geneo_basis(cfg, angles=None, n_loc=None):
    """The GenEO coarse basis V (columns on all DoFs, Gram-Schmidt in a(., .) per
    subdomain), the eigenvalues per subdomain, and the mesh, A and b it was
    built for."""
    mesh = make_mesh(cfg)
    E = cfg.material
    angles = element_angles(cfg) if angles is None else angles
    n_loc = cfg.n_loc if n_loc is None else n_loc
    cache = make_cache(mesh, E)
    A = assemble_global(mesh, angles, E, cache=cache)
    b = mesh.compression_load(cfg.traction)
    subs = subdomains(cfg)
    mus = partition_of_unity(mesh, subs, cfg.overlap)
    cols, lams = [], []
    for s in subs:
        gp = geneo_problem(mesh, angles, E, s, mus[s.index], b, cache)
        lam, phi = geneo_eigs(gp, n_loc)
        lams.append(lam)
        gd = (3 * gp.nodes[:, None] + np.arange(3)).ravel()
        for q in gram_schmidt(gp.A, [gp.mu * phi[:, k] for k in range(phi.shape[1])]):
            col = np.zeros(mesh.n_dof)
            col[gd] = q
            cols.append(col)
    return sp.csc_matrix(np.stack(cols, axis=1)), lams, mesh, A, b


def run_geneo(cfg, angles=None, n_loc=None, uh=None):
    """GenEO coarse approximation with n_loc eigenvectors per subdomain:
    (eigenvalues per subdomain, u_H, u_h, energy error ||u_h - u_H||_a / ||u_h||_a)."""
    V, lams, mesh, A, b = geneo_basis(cfg, angles, n_loc)
    AH = (V.T @ (A @ V)).toarray()
    c = coarse_solve(0.5 * (AH + AH.T), V.T @ b)
    uH = V @ c
    if uh is None:
        uh = solve_fine(mesh, A, b)
    return lams, uH, uh, energy_norm(A, uh - uH) / energy_norm(A, uh)
