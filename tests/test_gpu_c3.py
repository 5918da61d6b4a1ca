"""The largest beam, c3 (384 x 24 x 48, 1,414,875 DoF, 64 subdomains, n_loc =
24), in the bench's launch configuration, FP64 and mixed precision.

The oracle cannot solve all 64 local problems in seconds, so parity is
checked on three sampled subdomains (clamped, floating interior, loaded end)
against tests/golden/c3_sample_eigs.json (written by
tests/golden/make_c3_golden.py, which calls only oracle/): the DoF classes and
every eigenvalue (1e-8 relative FP64, 1e-5 mixed); and the GPU eigenpairs of
those subdomains solve the oracle's own pencil: for phi = E x the reduced
residual E^T (K phi - lambda B phi) = S x - lambda T x, formed with the
oracle's sparse matrices and one sparse A11 factorisation, is below 1e-6 of
||S x|| + lambda ||T x||.  For the whole problem: mixed eigenvalues against
FP64 (1e-5 each), the coarse dimensions, and the global energy errors of both
coarse solutions against a fine solution u_h computed on the GPU by the
two-level Schwarz PCG (msgfem_schwarz_solve with the FP64 MS-GFEM coarse
space, residual 1e-10): mixed within 1 % of FP64 at equal n_loc."""
import ctypes as C
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from parity_util import assert_eigs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c3_sample_eigs.json")


def _run(cfg, ang, precision):
    from paper_2211_13893_gb300 import MSGFEM
    m = MSGFEM.from_config(cfg, ang, seed=1234, precision=precision)
    lam = m.local_spaces(cfg.n_loc)
    nc = m.coarse_assemble()
    u = torch.empty(m.n_dof, dtype=torch.float64, device="cuda")
    m.solve(u_out=u)
    return m, lam, nc, u


def _energy(m, u, ref):
    e = C.c_double(-1.0)
    assert m.lib.msgfem_energy_error_noalloc(m.h, u.data_ptr(), ref.data_ptr(), C.addressof(e)) == 0
    return e.value


def _pencil_residuals(cfg, samples, m, lam):
    """Largest relative reduced residual of the GPU's non-rigid eigenpairs in the oracle's pencil."""
    from oracle.assemble import make_cache
    from oracle.local import _factor, local_problem
    from oracle.mesh import make_mesh
    from oracle.partition import partition_of_unity, subdomains
    from workloads import element_angles
    mesh = make_mesh(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(mesh, subs, cfg.overlap)
    b = mesh.compression_load(cfg.traction)
    cache = make_cache(mesh, cfg.material)
    ang = element_angles(cfg)
    worst = 0.0
    for j in samples:
        lp = local_problem(mesh, ang, cfg.material, subs[j], mus[j], b, cache)
        phi, _ = m.basis(j)
        lu = _factor(lp.A11)
        A11, A12, A22, B11 = lp.A11, lp.A12, lp.A22, lp.B11
        p1, p2 = phi[lp.I1], phi[lp.I2]
        top = max(np.abs(lam[j]).max(), 1.0)
        for k in range(phi.shape[1]):
            if abs(lam[j][k]) <= 1e-8 * top:
                continue
            q1 = A11 @ p1[:, k] + A12 @ p2[:, k]                 # (K phi)_1, zero for an A-harmonic phi
            Sx = A12.T @ p1[:, k] + A22 @ p2[:, k] - A12.T @ lu.solve(q1)
            Tx = -(A12.T @ lu.solve(B11 @ p1[:, k]))
            r = np.linalg.norm(Sx - lam[j][k] * Tx) / (np.linalg.norm(Sx) + abs(lam[j][k]) * np.linalg.norm(Tx))
            worst = max(worst, r)
    return worst


def test_c3_fp64_mixed_and_gpu_fine_solution():
    from paper_2211_13893_gb300 import MSGFEM
    from dataclasses import replace
    from workloads import element_angles, get_config
    gold = json.load(open(GOLD))
    cfg = get_config("c3")
    ang = torch.tensor(element_angles(cfg).reshape(-1), dtype=torch.float64, device="cuda")
    samples = [int(k) for k in gold["samples"]]
    m64, lam64, nc64, u64 = _run(cfg, ang, 0)
    for j in samples:
        rec = gold["samples"][str(j)]
        inf = m64.info(j)
        assert (inf["n_star_dof"], inf["n1"], inf["n2"], inf["n3"]) == (rec["n_star_dof"], rec["n1"], rec["n2"],
                                                                           rec["n3"])
        assert_eigs(lam64[j], rec["lambda"], 1e-8, j)
    assert _pencil_residuals(cfg, samples, m64, lam64) <= 1e-6
    # the fine solution u_h on the GPU: Schwarz PCG with FP32 Dirichlet factors on Omega_j
    # and the FP64 MS-GFEM coarse space, started from u^G
    hl = MSGFEM.from_config(replace(cfg, oversampling=cfg.overlap), ang, seed=1234, precision=1)
    uh = torch.empty(m64.n_dof, dtype=torch.float64, device="cuda")
    _, info = hl.schwarz_solve(m64, u0=u64, rtol=1e-10, u_out=uh)
    hl.close()
    assert info["residual"] <= 1e-10
    e64 = _energy(m64, u64, uh)
    m64.close()
    m32, lam32, nc32, u32 = _run(cfg, ang, 1)
    for j in samples:
        assert_eigs(lam32[j], gold["samples"][str(j)]["lambda"], 1e-5, j)
    for j in range(m32.N):
        assert_eigs(lam32[j], lam64[j], 1e-5, j)
    assert nc32 == nc64
    e32 = _energy(m32, u32, uh)
    assert 0.0 < e64 < 1.0 and abs(e32 - e64) <= 0.01 * e64, (e32, e64)
    assert 0.0 <= _energy(m32, u32, u64) <= 1e-5
    m32.close()
