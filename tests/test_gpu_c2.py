"""Parity at the benchmark's full size: the c2 beam (192x12x39, 301,080 DoF,
32 subdomains, n_loc = 20) in the bench's launch configuration, against the
oracle results stored in tests/golden/c2_oracle.json (written by
tests/golden/make_c2_golden.py, which calls only oracle/).

Checked: all 32 x 20 eigenvalues (1e-8 relative to the subdomain's largest
wanted eigenvalue in FP64, 1e-5 mixed), the coarse dimension, and the relative
energy error of u^G within 1 % of the oracle's.  The energy error uses
Galerkin orthogonality: u^G is the A-orthogonal projection of u_h onto the
coarse space, so ||u_h - u^G||_a^2 = b^T u_h - b^T u^G, with b^T u_h =
||u_h||_a^2 from the golden file and b the consistent load vector.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_oracle.json")


def _run(precision):
    from oracle.mesh import BeamMesh
    from paper_2211_13893_gb300 import MSGFEM
    from workloads import element_angles, get_config
    if not os.path.exists(GOLD):
        pytest.skip("tests/golden/c2_oracle.json not generated")
    gold = json.load(open(GOLD))
    cfg = get_config("c2")
    ang = torch.tensor(element_angles(cfg).reshape(-1), dtype=torch.float64, device="cuda")
    m = MSGFEM.from_config(cfg, ang, seed=1234, precision=precision)
    lam = m.local_spaces(cfg.n_loc)
    nc = m.coarse_assemble()
    uG, _ = m.solve()
    m.close()
    b = BeamMesh.from_config(cfg).compression_load(cfg.traction)
    e2 = (gold["uh_energy"] ** 2 - float(b @ uG)) / gold["uh_energy"] ** 2
    return gold, lam, nc, np.sqrt(max(e2, 0.0))


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-5)])
def test_c2_full_size(precision, tol):
    gold, lam, nc, err = _run(precision)
    ref = np.array(gold["lam"])
    for j in range(ref.shape[0]):
        scale = max(abs(ref[j, -1]), 1e-2)
        assert np.abs(lam[j] - ref[j]).max() <= tol * scale, (j, lam[j], ref[j])
    assert nc == sum(gold["basis_counts"])
    assert abs(err - gold["energy_error"]) <= 0.01 * gold["energy_error"], (err, gold["energy_error"])
