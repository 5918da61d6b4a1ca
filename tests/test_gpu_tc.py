"""The tensor-core tile kernel of the FP32 factorisation (msgfem_options.
factor_kernel = 1: TMA-staged operands, tcgen05.mma in split TF32 with the
accumulator in tensor memory) against the oracle, with the same bars as the
FMA kernel's mixed-precision parity: every eigenvalue to 1e-5 relative,
spans at spectral gaps to 1e-4, psi_j and u^G in the energy norm, the energy
error within 1 %.  Cases with one-tile and multi-tile layers, both
factorisation schedules, curved sections (s2) and the c1 beam (layers of four
64-row tiles); the full-size c2 case (eleven tiles per layer) is in
test_gpu_c2.py.  And the autotuner's accuracy gate: the tensor-core factor of
a subdomain differs from the FMA kernel's by at most twice as much as the FMA
kernel's two schedules (two summation orders) differ from each other."""
import pytest

from test_gpu_local import run_case
from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,schedule", [("t2", 0), ("c1", 0), ("c1", 1), ("s2", 0), ("s2", 1)])
def test_tensor_core_factorisation_parity(name, schedule):
    run_case(name, precision=1, tol_lam=1e-5, tol_angle=1e-4, factor_kernel=1, factor_schedule=schedule)


@pytest.mark.parametrize("name", ["t4", "c1"])
def test_autotuner_gate_of_the_tensor_core_factor(name):
    """Both kernels are timed; the tensor-core factor agrees with the FMA
    kernel's to FP32-GEMM level (1e-5, Frobenius) and is adopted only when it
    is within twice the FMA kernel's own schedule-to-schedule difference."""
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config(name)
    m = MSGFEM.from_config(cfg, element_angles(cfg), seed=7, precision=1)
    m.local_spaces(cfg.n_loc)
    t = m.autotune()
    lam = m.local_spaces(cfg.n_loc)          # the chosen kernel still converges
    m.close()
    assert 0.0 <= t["fma_factor_diff"] <= 1e-5, t
    assert 0.0 < t["tc_factor_diff"] <= 1e-5, t
    assert min(x for row in t["factor_ms_tc"] for x in row if x > 0) > 0
    if t["tc_factor_diff"] > 2.0 * t["fma_factor_diff"]:
        assert t["factor_kernel"] == 0, t
    assert lam.shape == (m.N, cfg.n_loc)
