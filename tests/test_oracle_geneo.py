"""Pins of the GenEO comparison oracle (oracle/geneo.py, Sec. 2.3, Eq.
bilinearGeneralizeEigenProblem): the finite eigenvalues of the full pencil
(K, D_mu K D_mu) by dense QZ equal the reduced ones; every eigenpair satisfies
the unreduced problem and the basis is B-orthonormal; a subdomain away from
the clamped face has exactly six zero eigenvalues spanning the rigid motions
of Omega_j; all eigenvectors reproduce u_h exactly; nested coarse spaces give
a non-increasing energy error; with o* = o the MS-GFEM local space differs
(the A-harmonic constraint), so the two eigenvalue sets differ."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.assemble import make_cache
from oracle.geneo import geneo_eigs, geneo_problem, run_geneo
from oracle.mesh import make_mesh
from oracle.partition import partition_of_unity, subdomains
from workloads import element_angles, get_config


def problems(name):
    cfg = get_config(name)
    m = make_mesh(cfg)
    ang = element_angles(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(m, subs, cfg.overlap)
    b = m.compression_load(cfg.traction)
    cache = make_cache(m, cfg.material)
    return cfg, m, [geneo_problem(m, ang, cfg.material, s, mus[s.index], b, cache) for s in subs]


def _pencil(gp):
    F = np.concatenate([gp.I1, gp.I2])
    K = gp.A[F][:, F].toarray()
    d = gp.mu[F]
    return F, K, d[:, None] * K * d[None, :]


@pytest.mark.parametrize("name", ["t1", "t2"])
def test_brute_force_qz(name):
    cfg, m, gps = problems(name)
    for gp in gps:
        _, K, B = _pencil(gp)
        alpha, beta = sla.eigvals(K, B, homogeneous_eigvals=True)
        lam, _ = geneo_eigs(gp, cfg.n_loc)
        scale = max(abs(lam[-1]), 1.0)
        fin = np.abs(beta) > 1e-10 * np.abs(alpha).max()
        lq = (alpha[fin] / beta[fin]).real
        lq = np.sort(lq[np.abs(lq) < 1e5 * scale])
        assert np.allclose(lq[:len(lam)], lam, rtol=1e-7, atol=1e-9 * scale)


@pytest.mark.parametrize("name", ["t2", "c1", "s1"])
def test_eigenpairs_solve_the_unreduced_problem(name):
    cfg, m, gps = problems(name)
    for gp in gps:
        lam, phi = geneo_eigs(gp, cfg.n_loc)
        F, K, B = _pencil(gp)
        P = phi[F]
        assert np.all(phi[gp.I3] == 0.0)
        scale = np.abs(K).max() * np.abs(P).max()
        R = K @ P - (B @ P) * lam[None, :]
        assert np.abs(R).max() < 1e-9 * scale * max(1.0, np.abs(lam).max())
        assert np.allclose(P.T @ B @ P, np.eye(len(lam)), atol=1e-9)
        assert np.all(np.diff(lam) >= -1e-12 * abs(lam[-1]))


def test_rigid_motions_of_a_floating_subdomain():
    cfg, m, gps = problems("c1")
    clamped, floating = gps
    lam0, _ = geneo_eigs(clamped, cfg.n_loc)
    lam1, phi1 = geneo_eigs(floating, cfg.n_loc)
    assert len(clamped.I3) > 0 and lam0[0] > 1e-6 * lam0[-1]
    assert len(floating.I3) == 0
    assert np.abs(lam1[:6]).max() < 1e-10 * lam1[-1] and lam1[6] > 1e-4 * lam1[-1]
    X = m.coords(floating.nodes)
    Xc = X - X.mean(axis=0)
    R = np.zeros((floating.n_star, 6))
    for c in range(3):
        R[c::3, c] = 1.0
    for r, axis in enumerate(np.eye(3)):
        R[:, 3 + r] = np.cross(axis, Xc).reshape(-1)
    coef, *_ = np.linalg.lstsq(phi1[:, :6], R, rcond=None)
    assert np.abs(phi1[:, :6] @ coef - R).max() < 1e-8 * np.abs(R).max()


@pytest.mark.parametrize("name", ["t1", "t2"])
def test_full_local_spaces_reproduce_uh(name):
    cfg = get_config(name)
    _, _, gps = problems(name)
    n_all = max(len(gp.I1) for gp in gps)
    _, _, _, err = run_geneo(cfg, n_loc=n_all)
    assert err < 1e-10


def test_energy_error_non_increasing_in_n_loc():
    cfg = get_config("t2")
    errs = []
    uh = None
    for n in (2, 6, 12, 20):
        _, _, uh, err = run_geneo(cfg, n_loc=n, uh=uh)
        errs.append(err)
    assert all(b <= a * (1 + 1e-10) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0]


def test_geneo_and_msgfem_local_problems_differ():
    """Without oversampling the two methods still solve different eigenproblems:
    GenEO eliminates the cut boundary (Neumann there), MS-GFEM the interior
    (A-harmonic); the spectra of one subdomain are not the same."""
    from oracle.local import local_eigs_dense
    cfg, m, gps = problems("t2")
    for gp in gps:
        lg, _ = geneo_eigs(gp, 10)
        lm, _ = local_eigs_dense(gp, 10)
        nz = (lg > 1e-8 * lg[-1]) & (lm > 1e-8 * lm[-1])      # the rigid zeros are common
        assert nz.sum() >= 4 and not np.allclose(lg[nz], lm[nz], rtol=1e-3)


@pytest.mark.parametrize("name", ["t3", "c1"])
def test_msgfem_beats_geneo_at_equal_n_loc(name):
    """Sec. 2.4: GenEO local spaces used as a GFEM converge poorly in m_j; the
    MS-GFEM space (oversampling, A-harmonic, particular function) is far more
    accurate at the same number of local eigenvectors."""
    from oracle.coarse import run_msgfem
    cfg = get_config(name)
    ref = run_msgfem(cfg, n_loc=8)
    _, _, _, err = run_geneo(cfg, n_loc=8, uh=ref.uh)
    assert ref.energy_error < 0.5 * err
