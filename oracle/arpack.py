"""The paper's own local solver: ARPACK shift-invert on the saddle-point pencil.

Sec. 4.5: the local GEVP is solved with ARPACK in symmetric shift-invert mode
with a sparse LU (UMFPACK) as the subdomain solver, applied to the matrix form
of Eq. algebraicAharmonic,

    [A11 A12 A11] [phi1]          [B11 0 0] [phi1]
    [A21 A22 A21] [phi2] = lambda [0   0 0] [phi2]
    [A11 A12 0  ] [p   ]          [0   0 0] [p   ].

Here SciPy's ``eigsh`` (ARPACK) and ``splu`` (SuperLU, standing in for
UMFPACK) are used with the shift sigma = -1e-2; eigenvectors come back
normalised phi^T B phi = 1.  This is the timed CPU baseline of the local stage.

The Lanczos start vector is a seeded Gaussian vector: a single-vector Krylov
method sees each copy of a multiple eigenvalue (the six rigid zeros of a
floating subdomain) only through rounding, so with ARPACK's own random start
the number of zeros found could vary from call to call.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def saddle_pencil(lp):
    A11, A12, A22 = lp.A11, lp.A12, lp.A22
    M = sp.bmat([[A11, A12, A11], [A12.T, A22, A12.T], [A11, A12, None]], format="csc")
    n1, n2 = A11.shape[0], A22.shape[0]
    Bm = sp.block_diag([lp.B11, sp.csr_matrix((n2, n2)), sp.csr_matrix((n1, n1))], format="csc")
    return M, Bm


def local_eigs_arpack(lp, n_loc, sigma=-1e-2, tol=1e-12, seed=0):
    n1, n2 = len(lp.I1), len(lp.I2)
    if n2 == 0:
        return np.zeros(0), np.zeros((lp.n_star, 0))
    M, Bm = saddle_pencil(lp)
    lu = spla.splu((M - sigma * Bm).tocsc())
    op = spla.LinearOperator(M.shape, matvec=lu.solve, dtype=np.float64)
    k = min(n_loc, n2)
    v0 = np.random.default_rng(seed).standard_normal(M.shape[0])
    lam, V = spla.eigsh(M, k=k, M=Bm, sigma=sigma, which="LM", OPinv=op, tol=tol, v0=v0,
                        ncv=min(M.shape[0] - 1, max(2 * k + 1, k + 20)))
    srt = np.argsort(lam)
    lam, V = lam[srt], V[:, srt]
    phi = np.zeros((lp.n_star, k))
    phi[lp.I1] = V[:n1]
    phi[lp.I2] = V[n1:n1 + n2]
    bn = np.einsum("ik,ik->k", phi[lp.I1], lp.B11 @ phi[lp.I1])
    return lam, phi / np.sqrt(bn)
