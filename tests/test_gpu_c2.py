"""Parity at the benchmark's full size: the c2 beam (192x12x39, 301,080 DoF,
32 subdomains, n_loc = 20) in the bench's launch configuration, against the
oracle results stored in tests/golden/c2_oracle.json and the oracle's coarse
solution in tests/golden/c2_oracle_uG.npy (both written by
tests/golden/make_c2_golden.py, which calls only oracle/).

Checked: each of the 32 x 20 eigenvalues (1e-8 relative to itself in FP64,
1e-5 mixed; rigid zeros absolutely at that fraction of the largest), the
coarse dimension, the coarse solution u^G against the oracle's in the global
energy norm (1e-8 FP64, 1e-5 mixed), and the relative energy error of u^G
within 1 % of the oracle's.  The energy error is formed directly with the
oracle's assembled A and load b: A u_h = b gives
||u_h - u||_a^2 = ||u_h||_a^2 - 2 b^T u + u^T A u for any u, with ||u_h||_a
from the golden file.
"""
import json
import os

import numpy as np
import pytest

from parity_util import assert_eigs, energy_error_direct, energy_rel

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GOLD = os.path.join(HERE, "c2_oracle.json")
GOLD_UG = os.path.join(HERE, "c2_oracle_uG.npy")


@pytest.fixture(scope="module")
def oracle_c2():
    from oracle.assemble import assemble_global, make_cache
    from oracle.mesh import make_mesh
    from workloads import element_angles, get_config
    cfg = get_config("c2")
    mesh = make_mesh(cfg)
    A = assemble_global(mesh, element_angles(cfg), cfg.material, cache=make_cache(mesh, cfg.material))
    return cfg, json.load(open(GOLD)), np.load(GOLD_UG), A, mesh.compression_load(cfg.traction)


@pytest.mark.parametrize("precision,tol,factor_kernel", [(0, 1e-8, 0), (1, 1e-5, 0), (1, 1e-5, 1)])
def test_c2_full_size(oracle_c2, precision, tol, factor_kernel):
    """FP64, mixed with the FMA factor kernel, mixed with the tensor-core one."""
    from paper_2211_13893_gb300 import MSGFEM
    from workloads import element_angles
    cfg, gold, uG_or, A, b = oracle_c2
    ang = torch.tensor(element_angles(cfg).reshape(-1), dtype=torch.float64, device="cuda")
    m = MSGFEM.from_config(cfg, ang, seed=1234, precision=precision, factor_kernel=factor_kernel)
    lam = m.local_spaces(cfg.n_loc)
    nc = m.coarse_assemble()
    uG, _ = m.solve()
    m.close()
    ref = np.array(gold["lam"])
    for j in range(ref.shape[0]):
        assert_eigs(lam[j], ref[j], tol, j)
    assert nc == sum(gold["basis_counts"])
    assert energy_rel(A, uG, uG_or) <= tol, energy_rel(A, uG, uG_or)
    err = energy_error_direct(A, b, gold["uh_energy"] ** 2, uG)
    assert abs(err - gold["energy_error"]) <= 0.01 * gold["energy_error"], (err, gold["energy_error"])
