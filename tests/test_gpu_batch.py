"""Batched instances: one handle holding S copies of the mesh and partition,
each with its own element angles (msgfem_options.instances).  Every
instance's eigenvalues match the oracle's for that instance's angles, the
warm-start plumbing addresses each instance's own perturbation field, and the
coarse problem is refused for a batched handle."""
import numpy as np
import pytest

from parity_util import assert_eigs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _fields(cfg, samples):
    from workloads import element_angles, wrinkle_field
    d = np.stack([wrinkle_field(cfg, s) for s in samples])
    return element_angles(cfg)[None] + d, d


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-5)])
def test_batched_instances_match_oracle(precision, tol):
    from oracle.coarse import run_msgfem
    from paper_2211_13893_gb300 import MSGFEM, MsgfemError
    from workloads import get_config
    cfg = get_config("c5")
    samples = [3, 11, 27]
    ang, _ = _fields(cfg, samples)
    S = len(samples)
    m = MSGFEM.from_config(cfg, ang.reshape(-1), seed=9, precision=precision, instances=S)
    assert m.N == S * cfg.n_sub
    lam = m.local_spaces(cfg.n_loc)
    for i in range(S):
        ref = run_msgfem(cfg, angles=ang[i], solver="dense")
        for j in range(cfg.n_sub):
            assert_eigs(lam[i * cfg.n_sub + j], np.asarray(ref.lam[j])[:cfg.n_loc], tol, (i, j))
    with pytest.raises(MsgfemError):
        m.coarse_assemble()
    m.close()


def test_batched_warm_features_follow_instances():
    from paper_2211_13893_gb300 import MSGFEM
    from workloads import get_config
    cfg = get_config("c5")
    ang, d = _fields(cfg, [1, 2])
    m = MSGFEM.from_config(cfg, ang.reshape(-1), instances=2)
    m.local_spaces(cfg.n_loc)
    nf = m.warm_features(None, 1.0, None, 0)
    feat = torch.empty((m.N, nf), dtype=torch.float32, device="cuda")
    m.warm_features(torch.tensor(d.reshape(-1), device="cuda"), 0.5, feat, nf)
    f = feat.cpu().numpy()
    info = [m.basis(j)[1] for j in range(m.N)]   # (I0, I1, J0, J1) node boxes
    for j in range(m.N):
        i = j // cfg.n_sub
        I0, I1, J0, J1 = info[j]
        expect = 0.5 * d[i, I0:I1, J0:J1, :].reshape(-1)
        assert np.allclose(f[j, :expect.size], expect, rtol=1e-6, atol=1e-6)
        assert np.all(f[j, expect.size:] == 0.0)
    m.close()
