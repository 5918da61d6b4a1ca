"""The tensor-core tile kernel of the FP32 factorisation (msgfem_options.
factor_kernel = 1: TMA-staged operands, tcgen05.mma in split TF32 with the
accumulator in tensor memory) against the oracle, with the same bars as the
FMA kernel's mixed-precision parity: every eigenvalue to 1e-5 relative,
spans at spectral gaps to 1e-4, psi_j and u^G in the energy norm, the energy
error within 1 %.  Cases with one-tile and multi-tile layers, both
factorisation schedules, curved sections (s2) and the c1 beam (layers of four
64-row tiles); the full-size c2 case (eleven tiles per layer) is in
test_gpu_c2.py.  And the autotuner's accuracy gate: the
tensor-core factor of a subdomain agrees with the FMA kernel's to 1e-4 in
the Frobenius norm."""
import pytest

from test_gpu_local import run_case
from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,schedule", [("t2", 0), ("c1", 0), ("c1", 1), ("s2", 0), ("s2", 1)])
def test_tensor_core_factorisation_parity(name, schedule):
    run_case(name, precision=1, tol_lam=1e-5, tol_angle=1e-4, factor_kernel=1, factor_schedule=schedule)


def test_autotuner_gate_accepts_the_tensor_core_factor():
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("t4")
    m = MSGFEM.from_config(cfg, element_angles(cfg), seed=7, precision=1)
    m.local_spaces(cfg.n_loc)
    t = m.autotune()
    m.close()
    assert 0.0 <= t["tc_factor_diff"] <= 1e-4, t
    assert min(x for row in t["factor_ms_tc"] for x in row if x > 0) > 0
