"""Checkpoint / resume of the local stage (msgfem_export_local /
msgfem_import_local; the offline / online reuse of local bases, Sec. 6): a
second handle that imports the exported local spaces, here through a file,
assembles the same coarse problem and gives the same coarse solution, bit for
bit, without an eigensolve; the exported eigenvectors are those of
msgfem_get_basis; threshold selection works on imported eigenvalues."""
import numpy as np
import pytest

from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["t2", "s1"])
def test_resume_from_exported_local_spaces(name, tmp_path):
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config(name)
    ang = element_angles(cfg)
    a = MSGFEM.from_config(cfg, ang, seed=4)
    lam = a.local_spaces(cfg.n_loc).copy()
    nc = a.coarse_assemble()
    ua, _ = a.solve()
    for j in range(a.N):
        phi, lj = a.export_local(j)
        basis, _ = a.basis(j)
        assert np.array_equal(phi[:, :cfg.n_loc], basis) and np.array_equal(lj, lam[j])
    a.save_local(tmp_path / "local")
    nt = a.coarse_assemble(threshold=0.05)
    ut, _ = a.solve()
    a.close()
    b = MSGFEM.from_config(cfg, ang, seed=99)
    b.load_local(tmp_path / "local")
    assert b.coarse_assemble() == nc
    ub, _ = b.solve()
    assert np.array_equal(ub, ua)
    assert b.coarse_assemble(threshold=0.05) == nt
    ub2, _ = b.solve()
    assert np.array_equal(ub2, ut)
    assert all(b.info(j)["iterations"] == 0 for j in range(b.N))
    b.close()


def test_checkpoint_of_another_decomposition_is_refused(tmp_path):
    """A checkpoint written with another oversampling (same mesh, same number of
    subdomains and DoFs) is refused before the library reads it, and so are
    arrays whose shapes do not match the handle's oversampling domains."""
    from dataclasses import replace
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("t2")
    ang = element_angles(cfg)
    a = MSGFEM.from_config(cfg, ang, seed=4)
    a.local_spaces(cfg.n_loc)
    a.save_local(tmp_path / "local")
    out = [a.export_local(j) for j in range(a.N)]
    a.close()
    b = MSGFEM.from_config(replace(cfg, oversampling=cfg.oversampling + 1), ang, seed=4)
    with pytest.raises(ValueError):
        b.load_local(tmp_path / "local")
    lam = np.stack([o[1] for o in out])
    with pytest.raises(ValueError):
        b.import_local(lam, [o[0] for o in out])
    with pytest.raises(ValueError):
        b.import_local(lam[:, :3], [o[0] for o in out])
    b.close()
