"""msgfem_plan (include/msgfem.h): the device storage of a workload planned on
the host, through the built library, with no GPU.  Checked against the layout
of the layer blocks written out here from the oracle's DoF classes (per layer
K keeps B1 + B2, A11 keeps B1, each padded to 64 rows; D, E and Linv blocks
plus the compact solve buffers of 32 and 8 columns, each part 256-byte
aligned), and for the wave split, ENOMEM and invalid descriptors."""
import numpy as np
import pytest

from workloads import get_config


@pytest.fixture(scope="module")
def plan():
    from paper_2211_13893_gb300.build import build
    build()
    from paper_2211_13893_gb300.msgfem import plan as p
    return p


def _align(n):
    return (n + 255) // 256 * 256


def expected_bytes(cfg, word):
    from oracle.mesh import make_mesh
    from oracle.partition import dof_classes, subdomains
    mesh = make_mesh(cfg)
    nz = cfg.NZ + 1
    out = []
    for sub in subdomains(cfg):
        _, b1, b2, _ = dof_classes(mesh, sub)
        per_layer = len(b1) // nz
        nK = 3 * int((b1 | b2).sum()) // nz
        nA = 3 * int(b1.sum()) // nz
        assert per_layer * nz == len(b1)
        bK, bA = (max(-(-n // 64), 1) * 64 for n in (nK, nA))
        parts = [bK * bK * (2 * nz - 1), bK * bK * nz, bA * bA * (2 * nz - 1), bA * bA * nz,
                 nz * bK * 32, nz * bA * 32, bK * 32, bA * 32, nz * bK * 8, nz * bA * 8, bK * 8, bA * 8]
        out.append(sum(_align(p * word) for p in parts))
    return np.array(out)


@pytest.mark.parametrize("name", ["t2", "c1", "s2", "c2"])
@pytest.mark.parametrize("precision", [0, 1])
def test_storage_matches_the_layout(plan, name, precision):
    cfg = get_config(name)
    exp = expected_bytes(cfg, 8 if precision == 0 else 4)
    got = plan(cfg, precision=precision)
    mib = 1048576.0
    assert got["status"] == "OK" and got["waves"] == 1 and got["n_subdomains"] == len(exp)
    assert got["blocks_mb"] * mib == exp.sum() and got["largest_mb"] * mib == exp.max()
    assert got["pool_mb"] == got["blocks_mb"]
    assert got["n_dof"] == cfg.n_dof


def test_waves_and_errors(plan):
    cfg = get_config("s2")
    full = plan(cfg)
    for budget in (full["largest_mb"], full["blocks_mb"] / 3):
        w = plan(cfg, wave_mb=budget)
        assert w["status"] == "OK" and w["waves"] >= 2 and w["pool_mb"] <= budget
    bad = plan(cfg, wave_mb=0.99 * full["largest_mb"])
    assert bad["status"] == "ENOMEM" and bad["waves"] == 0 and bad["largest_mb"] == full["largest_mb"]
    assert plan(cfg, precision=5)["status"] == "EINVAL"
    assert plan(cfg.with_(overlap=0))["status"] == "EINVAL"
    batched = plan(get_config("t2"), instances=3)
    assert batched["n_subdomains"] == 3 * plan(get_config("t2"))["n_subdomains"]


def test_c4_spar_needs_mixed_precision_or_waves(plan):
    """The 2.76M-DoF C-section: its FP64 factors (about 303 GiB) exceed the
    GB300's HBM (~278 GiB), the FP32 factors of the mixed path take half."""
    cfg = get_config("c4")
    f64, f32 = plan(cfg), plan(cfg, precision=1)
    assert f64["n_subdomains"] == 256 and f64["max_star_dof"] == 41580
    assert f64["blocks_mb"] > 284208.0 > f32["blocks_mb"]
    assert abs(f32["blocks_mb"] / f64["blocks_mb"] - 0.5) < 0.01
