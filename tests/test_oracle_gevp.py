"""Pins of the oracle's local eigenproblem, particular function and coarse
Galerkin solve (Secs. 3.3, 4.3, 4.4 of the paper)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle.arpack import local_eigs_arpack, saddle_pencil
from oracle.assemble import make_cache
from oracle.coarse import run_msgfem
from oracle.local import local_eigs_dense, local_problem, particular
from oracle.mesh import make_mesh
from oracle.partition import partition_of_unity, subdomains
from workloads import element_angles, get_config


def problems(name, **kw):
    cfg = get_config(name).with_(**kw) if kw else get_config(name)
    m = make_mesh(cfg)
    ang = element_angles(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(m, subs, cfg.overlap)
    b = m.compression_load(cfg.traction)
    cache = make_cache(m, cfg.material)
    return cfg, m, [local_problem(m, ang, cfg.material, s, mus[s.index], b, cache) for s in subs]


def rigid_modes_local(m, lp):
    X = m.coords(lp.nodes)
    c = X.mean(0)
    R = []
    for a in range(3):
        v = np.zeros_like(X)
        v[:, a] = 1.0
        R.append(v.ravel())
    for w in np.eye(3):
        R.append(np.cross(w, X - c).ravel())
    return np.array(R).T


@pytest.mark.parametrize("name", ["t1", "t2"])
def test_brute_force_saddle_qz(name):
    """The finite eigenvalues of the full saddle-point pencil (Eq.
    algebraicAharmonic), found by dense QZ, equal the dense-reduced eigenvalues."""
    cfg, m, lps = problems(name)
    for lp in lps:
        M, Bm = saddle_pencil(lp)
        w = sla.eigvals(M.toarray(), Bm.toarray(), homogeneous_eigvals=True)
        alpha, beta = w
        lam, _ = local_eigs_dense(lp, cfg.n_loc)
        k = len(lam)
        scale = max(abs(lam[-1]), 1.0)
        # the pencil is singular (B has a large null space); its infinite
        # eigenvalues come out of QZ as huge or ill-determined values
        fin = np.abs(beta) > 1e-10 * np.abs(alpha).max()
        lq = (alpha[fin] / beta[fin]).real
        lq = np.sort(lq[np.abs(lq) < 1e5 * scale])
        assert np.allclose(lq[:k], lam, rtol=1e-7, atol=1e-9 * scale)


@pytest.mark.parametrize("name", ["t2", "t3", "c1"])
def test_eigenpairs_satisfy_saddle_form(name):
    """Each phi is A-harmonic (third block row), satisfies the first two block
    rows with a multiplier p, and the basis is B-orthonormal."""
    cfg, m, lps = problems(name)
    for lp in lps:
        lam, phi = local_eigs_dense(lp, cfg.n_loc)
        A11, A12, A22, B11 = lp.A11, lp.A12, lp.A22, lp.B11
        lu = spla.splu(A11.tocsc())
        p1, p2 = phi[lp.I1], phi[lp.I2]
        scale = spla.norm(lp.A, 1) * np.abs(phi).max()
        assert np.abs(A11 @ p1 + A12 @ p2).max() < 1e-10 * scale
        for k in range(len(lam)):
            p = lu.solve(lam[k] * (B11 @ p1[:, k])) - p1[:, k] - lu.solve(A12 @ p2[:, k])
            row2 = A12.T @ p1[:, k] + A22 @ p2[:, k] + A12.T @ p
            assert np.abs(row2).max() < 1e-9 * scale * max(1.0, abs(lam[k]))
        G = p1.T @ (B11 @ p1)
        assert np.allclose(G, np.eye(len(lam)), atol=1e-10)


def test_rigid_modes_on_floating_subdomains():
    """A subdomain whose oversampling domain misses Gamma_D has six zero
    eigenvalues whose eigenvectors span the rigid-body modes (Sec. 5.2); the
    clamped subdomain has none."""
    cfg, m, lps = problems("c1")
    lam0, _ = local_eigs_dense(lps[0], cfg.n_loc)
    lam1, phi1 = local_eigs_dense(lps[1], cfg.n_loc)
    assert lam0[0] > 1e-3 and len(lps[0].I3) > 0
    assert len(lps[1].I3) == 0
    assert np.abs(lam1[:6]).max() < 1e-10 * lam1[-1] and lam1[6] > 1e-3
    R = rigid_modes_local(m, lps[1])
    coef, *_ = np.linalg.lstsq(phi1[:, :6], R, rcond=None)
    assert np.abs(phi1[:, :6] @ coef - R).max() < 1e-8 * np.abs(R).max()


@pytest.mark.parametrize("name", ["t2", "c1", "s1"])
def test_arpack_baseline_agrees(name):
    cfg, m, lps = problems(name)
    for lp in lps:
        ld, _ = local_eigs_dense(lp, cfg.n_loc)
        la, _ = local_eigs_arpack(lp, cfg.n_loc)
        top = abs(ld[-1])
        rigid = np.abs(ld) < 1e-8 * top
        assert np.abs(la[rigid]).max(initial=0) < 1e-9 * top
        assert np.allclose(la[~rigid], ld[~rigid], rtol=1e-9)


def test_particular_function():
    cfg, m, lps = problems("t2")
    for lp in lps:
        psi = particular(lp)
        touches_load = lp.sub.star[1] == cfg.NX
        assert np.any(psi != 0) == touches_load
        assert (psi[lp.I2] == 0).all() and (psi[lp.I3] == 0).all()
        if touches_load:
            r = lp.A11 @ psi[lp.I1] - lp.b[lp.I1]
            assert np.abs(r).max() < 1e-10 * np.abs(lp.b).max()


def test_oversampling_accelerates_decay():
    """Larger o* gives faster decay of 1/lambda (Theorem 2, Sec. 5.2)."""
    inv = []
    for o_star in (2, 4):
        cfg, m, lps = problems("t4", oversampling=o_star)
        lam, _ = local_eigs_dense(lps[2], 24)
        inv.append(1.0 / lam[8:24])
    assert (inv[1] < inv[0]).all()


@pytest.mark.parametrize("name", ["t1", "t2", "s1"])
def test_full_local_space_reproduces_fine_solution(name):
    """With n_loc = n2 the local spaces contain u_h|Omega* - psi_j, so the coarse
    Galerkin solution equals u_h up to roundoff (Eqs. global_particular_function,
    GFEM_coarse_approximation)."""
    cfg, m, lps = problems(name)
    n2 = max(len(lp.I2) for lp in lps)
    assert run_msgfem(cfg, n_loc=n2).energy_error < 1e-10


def test_energy_error_monotone_and_variant_order():
    """Nested coarse spaces: the energy error cannot increase with n_loc, and
    appending psi to the basis (the paper's implementation) is no worse than a
    fixed particular function (Galerkin optimality)."""
    cfg = get_config("t2")
    ref = run_msgfem(cfg)
    prev = np.inf
    for n in (2, 4, 6, 8, 10, 12):
        e2 = run_msgfem(cfg, n_loc=n, uh=ref.uh).energy_error
        e1 = run_msgfem(cfg, n_loc=n, uh=ref.uh, variant="i").energy_error
        assert e2 <= prev * (1 + 1e-12)
        assert e2 <= e1 * (1 + 1e-12)
        prev = e2


def test_pou_weighted_basis_is_a_orthonormal():
    """b-normalised eigenvectors stay orthonormal in a(., .) after the PoU
    multiplication, since phi^T B phi = a(Xi phi, Xi phi)."""
    cfg, m, lps = problems("c1")
    for lp in lps:
        _, phi = local_eigs_dense(lp, cfg.n_loc)
        W = lp.mu[:, None] * phi
        assert np.allclose(W.T @ (lp.A @ W), np.eye(phi.shape[1]), atol=1e-10)


def test_threshold_selection_nested_and_exhaustive():
    """Threshold t on 1 / lambda (Sec. 5.5): a t below every 1 / lambda keeps all
    n_loc vectors (same result as n_loc); lowering t can only enlarge the local
    spaces, so the energy error cannot increase; per-subdomain sizes follow the
    eigenvalues."""
    cfg = get_config("t2")
    full = run_msgfem(cfg)
    lam_all = np.concatenate(full.lam)
    t_small = 0.5 / lam_all.max()
    same = run_msgfem(cfg, threshold=t_small, uh=full.uh)
    assert same.basis_counts == full.basis_counts and same.energy_error == full.energy_error
    prev = np.inf
    for t in (1e-1, 3e-2, 1e-2, 3e-3):
        r = run_msgfem(cfg, threshold=t, uh=full.uh)
        for lam, cnt, sub_full in zip(r.lam, r.basis_counts, full.basis_counts):
            assert cnt <= sub_full
        assert r.energy_error <= prev * (1 + 1e-12)
        prev = r.energy_error


def test_per_subdomain_sizes_nested():
    """One n_loc per subdomain (the m_j of Eq. AHarmonic_coarse_space): every
    subdomain gets exactly its own count of eigenpairs, and raising any single
    subdomain's count enlarges the coarse space, so the Galerkin energy error
    cannot increase (a count read from the wrong subdomain breaks one of the
    two); the largest counts everywhere give the uniform result."""
    cfg = get_config("t2")
    base = [4, 7, 5, 9, 6, 8]
    ref = run_msgfem(cfg, n_loc=base)
    assert [len(lam) for lam in ref.lam] == base
    assert [phi.shape[1] for phi in ref.phi] == base
    for j in range(len(base)):
        up = list(base)
        up[j] += 3
        r = run_msgfem(cfg, n_loc=up, uh=ref.uh)
        assert [len(lam) for lam in r.lam] == up
        assert r.basis_counts[j] > ref.basis_counts[j]
        assert r.energy_error <= ref.energy_error * (1 + 1e-12)
        assert r.energy_error < ref.energy_error * (1 - 1e-6)
    top = run_msgfem(cfg, n_loc=[cfg.n_loc] * len(base), uh=ref.uh)
    assert top.energy_error == run_msgfem(cfg, uh=ref.uh).energy_error
