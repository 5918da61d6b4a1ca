"""One n_loc per subdomain (msgfem_local_spaces_var: the local basis sizes m_j
of Eq. AHarmonic_coarse_space chosen subdomain by subdomain, Sec. 5.3, Sec.
5.5) against the oracle run with the same counts: every subdomain's
eigenvalues one by one (1e-8 relative in FP64, 1e-5 mixed; rigid zeros
absolutely), NaN beyond its own count, its eigenvector spans at spectral gaps,
its particular function through the coarse dimension, u^G in the energy norm
(1e-8 / 1e-5) and the energy error within 1 %.  The counts are drawn per
subdomain and moved down to the nearest spectral gap of the oracle's
spectrum, so that each local space is well defined.  Also: a checkpoint of
such a stage resumes bit for bit, the threshold variant keeps at most the
counts, and counts outside 1 .. 31 are refused with the handle still usable.
"""
import functools

import numpy as np
import pytest

from oracle.coarse import run_msgfem
from parity_util import assert_eigs, energy_rel
from test_gpu_local import gap_sizes, max_sin_angle
from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


def _counts(cfg, ext_lam, seed=5):
    """Per-subdomain counts in 7 .. n_loc (the workload's own count, up to which
    its uniform runs meet the residual bound), each lowered to the nearest gap
    (drawn again while they are all equal)."""
    for s in range(seed, seed + 20):
        rng = np.random.default_rng(s)
        out = []
        for lam in ext_lam:
            target = int(rng.integers(7, cfg.n_loc + 1))
            gaps = [m for m in gap_sizes(np.asarray(lam), target) if m >= 7]
            out.append(gaps[-1] if gaps else target)
        if len(set(out)) > 1:
            break
    return np.array(out, dtype=np.int32)


@functools.lru_cache(maxsize=None)
def _oracle(name):
    """The oracle's spectra (one beyond every count), the counts, and its run
    with those counts."""
    cfg = get_config(name)
    ang = element_angles(cfg)
    ext = run_msgfem(cfg, angles=ang, n_loc=cfg.n_loc + 1)
    counts = _counts(cfg, ext.lam)
    return ext, counts, run_msgfem(cfg, angles=ang, n_loc=counts, uh=ext.uh)


@pytest.mark.parametrize("name,precision", [("t2", 0), ("t4", 0), ("t4", 1), ("c1", 1)])
def test_per_subdomain_counts_match_oracle(name, precision):
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config(name)
    ang = element_angles(cfg)
    ext, counts, ref = _oracle(name)
    assert len(set(counts.tolist())) > 1, counts
    tol = 1e-8 if precision == 0 else 1e-5
    m = MSGFEM.from_config(cfg, ang, seed=7, precision=precision)
    lam = m.local_spaces(counts)
    assert lam.shape == (m.N, counts.max())
    nc = m.coarse_assemble()
    uG, err = m.solve(u_ref=ext.uh)
    for j in range(m.N):
        n = int(counts[j])
        assert_eigs(lam[j, :n], ext.lam[j], tol, (name, j))
        assert np.all(np.isnan(lam[j, n:])), (name, j, lam[j])
        info = m.info(j)
        assert info["n_loc"] == n and info["residual"] < 1e-5, (name, j, info)
        assert info["basis_size"] == ref.basis_counts[j], (name, j, info, ref.basis_counts[j])
        phi, _ = m.basis(j)
        assert phi.shape[1] == counts.max() and np.all(phi[:, n:] == 0.0)
        for mm in gap_sizes(np.asarray(ext.lam[j]), n):
            s = max_sin_angle(ext.phi[j][:, :mm], phi[:, :mm])
            assert s < (1e-5 if precision == 0 else 1e-4), (name, j, mm, s)
    assert nc == sum(ref.basis_counts)
    assert energy_rel(ref.A, uG, ref.uG) <= tol, (name, energy_rel(ref.A, uG, ref.uG))
    assert abs(err - ref.energy_error) <= 0.01 * ref.energy_error, (err, ref.energy_error)
    m.close()


def test_per_subdomain_counts_checkpoint_and_threshold(tmp_path):
    """Export / import with NaN-padded eigenvalue rows resumes bit for bit;
    the threshold variant keeps at most each subdomain's count."""
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("t2")
    ang = element_angles(cfg)
    counts = np.array([7, 12, 9, 10, 8, 11], dtype=np.int32)
    a = MSGFEM.from_config(cfg, ang, seed=4)
    assert a.N == len(counts)
    lam = a.local_spaces(counts).copy()
    nc = a.coarse_assemble()
    ua, _ = a.solve()
    for j in range(a.N):
        phi, lj = a.export_local(j)
        assert np.array_equal(lj, lam[j], equal_nan=True)
        assert np.all(phi[:, counts[j]:counts.max()] == 0.0)
    a.save_local(tmp_path / "local")
    t = 0.5 / np.nanmax(lam)
    assert a.coarse_assemble(threshold=t) == nc                 # t below every 1 / lambda keeps all
    for tt in (3e-2, 1e-2):
        a.coarse_assemble(threshold=tt)
        for j in range(a.N):
            assert a.info(j)["basis_size"] <= counts[j] + 1
    a.close()
    b = MSGFEM.from_config(cfg, ang, seed=99)
    b.load_local(tmp_path / "local")
    assert [b.info(j)["n_loc"] for j in range(b.N)] == counts.tolist()
    assert b.coarse_assemble() == nc
    ub, _ = b.solve()
    assert np.array_equal(ub, ua)
    b.close()


def test_per_subdomain_counts_refused():
    """Counts of 0 or above 31 (the eigenvectors and the particular function
    share 32 basis columns) are EINVAL; a list of the wrong length is refused
    by the binding; the handle still runs a local stage afterwards."""
    from paper_2211_13893_gb300 import MSGFEM
    from paper_2211_13893_gb300.msgfem import MsgfemError
    cfg = get_config("t2")
    m = MSGFEM.from_config(cfg, element_angles(cfg), seed=4)
    for bad in ([0, 8, 8, 8, 8, 8], [8, 8, 32, 8, 8, 8]):
        with pytest.raises(MsgfemError) as e:
            m.local_spaces(np.array(bad))
        assert e.value.code == 1 and "1 .. 31" in str(e.value), e.value
    with pytest.raises(ValueError):
        m.local_spaces([8, 8])
    lam = m.local_spaces(cfg.n_loc)
    assert np.all(np.isfinite(lam))
    m.close()


def test_per_subdomain_counts_from_device_memory():
    """The counts may live in device memory: the same counts and eigenvalues as
    from a host array (a second local stage on the same handle)."""
    import torch
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("t2")
    counts = np.array([8, 10, 7, 9, 10, 8], dtype=np.int32)
    m = MSGFEM.from_config(cfg, element_angles(cfg), seed=4)
    a = m.local_spaces(counts).copy()
    b = m.local_spaces(torch.tensor(counts, device="cuda"))
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12, equal_nan=True)
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert [m.info(j)["n_loc"] for j in range(m.N)] == counts.tolist()
    m.close()
