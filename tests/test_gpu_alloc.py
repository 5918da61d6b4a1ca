"""msgfem_options.dev_alloc / dev_free: a handle that takes all its device
memory from the caller's allocator (PyTorch's caching allocator here) gives the
same results, bit for bit, as a handle on cudaMalloc, gives every block back at
destroy with the size it was allocated with, and a descriptor with only one of
the two callbacks is refused."""
import ctypes as C

import numpy as np
import pytest

from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


def test_caller_allocator():
    import torch
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("t2")
    ang = element_angles(cfg)
    live, calls = {}, [0]

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n, device=torch.cuda.current_device())
        live[p] = n
        calls[0] += 1
        return p

    def free(p, n):
        assert live.pop(p) == n
        torch.cuda.caching_allocator_delete(p)

    def run(**kw):
        m = MSGFEM.from_config(cfg, ang, seed=5, **kw)
        lam = m.local_spaces(cfg.n_loc).copy()
        m.coarse_assemble()
        u, _ = m.solve()
        phi, _ = m.basis(1)
        tune = m.autotune(reps=1)                 # replaces task lists: frees and allocates
        lam2 = m.local_spaces(cfg.n_loc).copy()
        m.close()
        return lam, u, phi, lam2, tune

    ref = run()
    got = run(allocator=(alloc, free))
    assert calls[0] > 20 and not live
    for a, b in zip(ref[:3], got[:3]):
        assert np.array_equal(a, b)
    # after the autotuner (whose timing-based choice of solve kernel may differ
    # between the two handles) the eigenvalues agree to rounding
    assert np.allclose(got[3], ref[3], rtol=1e-10, atol=1e-12 * np.abs(ref[3]).max())


def test_one_callback_is_refused():
    from paper_2211_13893_gb300 import msgfem
    lib = msgfem.load_library()
    cfg = get_config("t1")
    ang = np.ascontiguousarray(element_angles(cfg), dtype=np.float64).reshape(-1)
    E = np.ascontiguousarray(cfg.material, dtype=np.float64)
    cb = msgfem.DEV_ALLOC(lambda n, ctx: None)
    opt = msgfem.Options()
    opt.dev_alloc = C.cast(cb, C.c_void_p).value
    mesh = msgfem.Mesh(cfg.NX, cfg.NY, cfg.NZ, cfg.hx, cfg.hy, cfg.t, cfg.traction, None)
    plies = msgfem.Plies(E.ctypes.data, ang.ctypes.data, None)
    part = msgfem.Partition(cfg.sx, cfg.sy, 0, None)
    h = C.c_void_p()
    st = lib.msgfem_setup(C.byref(mesh), C.byref(plies), C.byref(part), cfg.overlap, cfg.oversampling,
                          C.byref(opt), C.byref(h))
    assert st == 1 and b"together" in lib.msgfem_last_error(h)
    lib.msgfem_destroy(h)
