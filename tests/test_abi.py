"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no GPU needed: no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    txt = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(msgfem_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2211_13893_gb300.build import build
    return build()


def test_header_lists_the_entry_points():
    syms = declared_symbols()
    for s in ("msgfem_setup", "msgfem_local_spaces", "msgfem_coarse_assemble", "msgfem_solve", "msgfem_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (msgfem_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_library_loads_with_binding(lib_path):
    import ctypes
    from paper_2211_13893_gb300 import msgfem
    lib = msgfem.load_library(lib_path)
    for s in declared_symbols():
        assert isinstance(getattr(lib, s), ctypes._CFuncPtr)
    assert set(msgfem.EXPORTS) <= set(declared_symbols())
    assert lib.msgfem_num_subdomains(None) == 0
    assert lib.msgfem_last_error(None) == b"null handle"


def test_setup_rejects_bad_descriptors(lib_path):
    """Argument validation happens before any CUDA call."""
    import ctypes as C
    import numpy as np
    from paper_2211_13893_gb300 import msgfem
    lib = msgfem.load_library(lib_path)
    E = np.ones(9)
    ang = np.zeros(8)
    h = C.c_void_p()
    plies = msgfem.Plies(E.ctypes.data, ang.ctypes.data)
    opt = msgfem.Options()
    for mesh, part, o, os_ in [((0, 2, 2), (1, 1), 1, 1), ((2, 2, 2), (3, 1), 1, 1), ((2, 2, 2), (1, 1), 0, 1),
                               ((2, 2, 2), (1, 1), 2, 1)]:
        m = msgfem.Mesh(*mesh, 1.0, 1.0, 1.0, 1.0)
        p = msgfem.Partition(*part)
        st = lib.msgfem_setup(C.byref(m), C.byref(plies), C.byref(p), o, os_, C.byref(opt), C.byref(h))
        assert st == 1 and not h.value
    # explicit boxes announced without an array; a box mesh without a brick size
    p = msgfem.Partition(1, 1, 2, None)
    m = msgfem.Mesh(2, 2, 2, 1.0, 1.0, 1.0, 1.0)
    assert lib.msgfem_setup(C.byref(m), C.byref(plies), C.byref(p), 1, 1, C.byref(opt), C.byref(h)) == 1
    m = msgfem.Mesh(2, 2, 2, 0.0, 1.0, 1.0, 1.0, None)
    p = msgfem.Partition(1, 1)
    assert lib.msgfem_setup(C.byref(m), C.byref(plies), C.byref(p), 1, 1, C.byref(opt), C.byref(h)) == 1
    assert not h.value


def test_setup_rejects_non_finite_inputs(lib_path):
    """A NaN traction, brick size, material constant or nodal load is refused
    (EINVAL) before any device memory is touched."""
    import ctypes as C
    import numpy as np
    from paper_2211_13893_gb300 import msgfem
    lib = msgfem.load_library(lib_path)
    ang = np.zeros(8)
    h = C.c_void_p()
    opt = msgfem.Options()
    p = msgfem.Partition(1, 1)
    E = np.ones(9)
    plies = msgfem.Plies(E.ctypes.data, ang.ctypes.data)
    for tr, hx in [(np.nan, 1.0), (1.0, np.inf)]:
        m = msgfem.Mesh(2, 2, 2, hx, 1.0, 1.0, tr)
        assert lib.msgfem_setup(C.byref(m), C.byref(plies), C.byref(p), 1, 1, C.byref(opt), C.byref(h)) == 1
        assert not h.value
    Ebad = np.ones(9)
    Ebad[4] = np.nan
    m = msgfem.Mesh(2, 2, 2, 1.0, 1.0, 1.0, 1.0)
    bad = msgfem.Plies(Ebad.ctypes.data, ang.ctypes.data)
    assert lib.msgfem_setup(C.byref(m), C.byref(bad), C.byref(p), 1, 1, C.byref(opt), C.byref(h)) == 1
    assert not h.value
    load = np.zeros(27 * 3)
    load[40] = np.nan
    m = msgfem.Mesh(2, 2, 2, 1.0, 1.0, 1.0, 1.0, None, load.ctypes.data)
    st = lib.msgfem_setup(C.byref(m), C.byref(plies), C.byref(p), 1, 1, C.byref(opt), C.byref(h))
    assert st == 1 and b"non-finite" in lib.msgfem_last_error(h)
    lib.msgfem_destroy(h)
