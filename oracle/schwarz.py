"""Two-level additive Schwarz preconditioned CG (Sec. 2.3; Sec. 5.4's reference
solver), the fine-scale solve that a coarse space preconditions.

On the free DoFs (clamped face removed) the preconditioner is

    M^{-1} r = V A_0^{-1} V^T r + sum_j R_j^T A_j^{-1} R_j r,

with R_j the restriction to the DoFs of V_{h,0}(Omega_j) (nodes of Omega_j off
its cut boundary and off the clamped face), A_j = R_j A R_j^T (local Dirichlet
problems on the overlapping subdomains), V the coarse basis (GenEO or MS-GFEM,
columns on all DoFs, zero on the clamped face) and A_0 = V^T A V.  Without V
it is the one-level method.  CG follows the textbook recurrence; the extreme
eigenvalues of the preconditioned operator are estimated from its coefficients
through the Lanczos tridiagonal matrix (the standard CG-Lanczos relation).

Test infrastructure: imported by tests only.
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fine import free_dofs
from .local import _factor
from .partition import dof_classes


@dataclass
class PCGResult:
    u: np.ndarray            # solution on all DoFs
    iterations: int
    residuals: list          # ||r_k||_2 / ||b||_2 per iteration (free DoFs)
    kappa: float             # Lanczos estimate of lambda_max / lambda_min of M^{-1} A
    lam_min: float
    lam_max: float


class TwoLevelSchwarz:
    """M^{-1} on the free DoFs of mesh for the global matrix A."""

    def __init__(self, mesh, A, subs, V=None):
        from dataclasses import replace
        self.fd = free_dofs(mesh)
        pos = -np.ones(mesh.n_dof, dtype=np.int64)
        pos[self.fd] = np.arange(len(self.fd))
        self.pos = pos
        self.Aff = A[self.fd][:, self.fd].tocsr()
        self.local = []
        for s in subs:
            nodes, b1, _, _ = dof_classes(mesh, replace(s, star=s.omega))
            g = (3 * nodes[b1][:, None] + np.arange(3)).ravel()      # global DoFs of V_h,0(Omega_j)
            idx = pos[g]
            assert (idx >= 0).all()
            self.local.append((idx, _factor(self.Aff[idx][:, idx])))
        self.V = None
        if V is not None and V.shape[1]:
            Vf = sp.csr_matrix(V)[self.fd]
            A0 = (Vf.T @ (self.Aff @ Vf)).toarray()
            self.V = Vf
            self.A0 = sla.cho_factor(0.5 * (A0 + A0.T))

    def apply(self, r):
        z = np.zeros_like(r)
        for idx, lu in self.local:
            z[idx] += lu.solve(r[idx])
        if self.V is not None:
            z += self.V @ sla.cho_solve(self.A0, self.V.T @ r)
        return z


def pcg(mesh, A, b, prec, x0=None, rtol=1e-10, max_iter=2000):
    """Preconditioned CG for A u = b on the free DoFs, from x0 (all DoFs) or zero."""
    fd = prec.fd
    Aff = prec.Aff
    bf = b[fd]
    x = np.zeros(len(fd)) if x0 is None else x0[fd].copy()
    r = bf - Aff @ x
    z = prec.apply(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(bf)
    res = [np.linalg.norm(r) / nb]
    alphas, betas = [], []
    it = 0
    while res[-1] > rtol and it < max_iter:
        q = Aff @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = prec.apply(r)
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        alphas.append(alpha)
        betas.append(beta)
        it += 1
        res.append(np.linalg.norm(r) / nb)
    # Lanczos tridiagonal of M^{-1} A from the CG coefficients
    k = len(alphas)
    if k:
        d = np.array([1.0 / alphas[0]] + [1.0 / alphas[i] + betas[i - 1] / alphas[i - 1] for i in range(1, k)])
        e = np.array([np.sqrt(betas[i]) / alphas[i] for i in range(k - 1)])
        ev = sla.eigvalsh_tridiagonal(d, e)
        lmin, lmax = ev[0], ev[-1]
    else:
        lmin = lmax = 1.0
    u = np.zeros(mesh.n_dof)
    u[fd] = x
    return PCGResult(u, it, res, lmax / lmin, lmin, lmax)
