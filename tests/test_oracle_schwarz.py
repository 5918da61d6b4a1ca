"""Pins of the two-level additive Schwarz PCG oracle (oracle/schwarz.py; Sec.
2.3's preconditioner, Sec. 5.4's reference solver): the preconditioner is
symmetric positive definite; PCG reaches the direct solution u_h; the CG-Lanczos
estimate of the extreme eigenvalues of M^{-1} A matches a dense eigensolve of
the preconditioned operator; a coarse space lowers the condition number and the
iteration count against the one-level method; more GenEO modes per subdomain
lower the condition number (Eq. condition_bound's trend); starting from the
MS-GFEM coarse solution u^G saves iterations."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.coarse import run_msgfem
from oracle.fine import energy_norm
from oracle.geneo import geneo_basis
from oracle.partition import subdomains
from oracle.schwarz import TwoLevelSchwarz, pcg
from workloads import get_config


def _setup(name, n_loc=None, coarse="msgfem"):
    cfg = get_config(name)
    if coarse == "geneo":
        V, _, mesh, A, b = geneo_basis(cfg, n_loc=n_loc)
        ref = run_msgfem(cfg, n_loc=n_loc)
    else:
        ref = run_msgfem(cfg, n_loc=n_loc)
        from oracle.mesh import make_mesh
        mesh, A, b, V = make_mesh(cfg), ref.A, ref.b, ref.V
    return cfg, mesh, A, b, V, ref


def test_preconditioner_is_spd():
    cfg, mesh, A, b, V, _ = _setup("t2")
    prec = TwoLevelSchwarz(mesh, A, subdomains(cfg), V)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal((2, len(prec.fd)))
    assert np.isclose(x @ prec.apply(y), y @ prec.apply(x), rtol=1e-10)
    for _ in range(3):
        v = rng.standard_normal(len(prec.fd))
        assert v @ prec.apply(v) > 0.0


@pytest.mark.parametrize("name", ["t2", "c1"])
def test_pcg_reaches_the_direct_solution(name):
    cfg, mesh, A, b, V, ref = _setup(name)
    prec = TwoLevelSchwarz(mesh, A, subdomains(cfg), V)
    out = pcg(mesh, A, b, prec, rtol=1e-12)
    assert out.residuals[-1] <= 1e-12
    assert energy_norm(A, out.u - ref.uh) <= 1e-9 * energy_norm(A, ref.uh)


def test_lanczos_estimate_matches_dense_spectrum():
    cfg, mesh, A, b, V, _ = _setup("t2")
    prec = TwoLevelSchwarz(mesh, A, subdomains(cfg), V)
    n = len(prec.fd)
    Minv = np.stack([prec.apply(e) for e in np.eye(n)], axis=1)
    Aff = prec.Aff.toarray()
    ev = np.sort(sla.eigvals(Minv @ Aff).real)
    # a random right-hand side excites every eigenvector (the end load does not)
    rhs = np.zeros(mesh.n_dof)
    rhs[prec.fd] = np.random.default_rng(1).standard_normal(n)
    out = pcg(mesh, A, rhs, prec, rtol=1e-13)
    assert np.isclose(out.lam_max, ev[-1], rtol=1e-6) and np.isclose(out.lam_min, ev[0], rtol=1e-5)


def test_coarse_space_lowers_condition_and_iterations():
    cfg, mesh, A, b, V, _ = _setup("c1")
    subs = subdomains(cfg)
    one = pcg(mesh, A, b, TwoLevelSchwarz(mesh, A, subs, None), rtol=1e-10)
    two = pcg(mesh, A, b, TwoLevelSchwarz(mesh, A, subs, V), rtol=1e-10)
    assert two.kappa < 0.5 * one.kappa and two.iterations < one.iterations


def test_more_geneo_modes_lower_the_condition_number():
    kappas = []
    for n in (2, 8, 16):
        cfg, mesh, A, b, V, _ = _setup("t3", n_loc=n, coarse="geneo")
        kappas.append(pcg(mesh, A, b, TwoLevelSchwarz(mesh, A, subdomains(cfg), V), rtol=1e-10).kappa)
    assert kappas[2] < kappas[1] < kappas[0], kappas


def test_start_from_the_coarse_solution():
    cfg, mesh, A, b, V, ref = _setup("c1")
    prec = TwoLevelSchwarz(mesh, A, subdomains(cfg), V)
    cold = pcg(mesh, A, b, prec, rtol=1e-10)
    warm = pcg(mesh, A, b, prec, x0=ref.uG, rtol=1e-10)
    assert warm.iterations < cold.iterations
    assert energy_norm(A, warm.u - ref.uh) <= 1e-8 * energy_norm(A, ref.uh)
