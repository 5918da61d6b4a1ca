"""ctypes wrapper of the host test harness (host_shim.cpp + the library's
setup.cpp, compiled with the host C++ compiler; no GPU, no CUDA calls).

Test infrastructure: it exposes the library's own host-side set-up (DoF
classes, partition of unity, nodal loads, 3-2-1 pins, waves) and its static
task schedules to CPU tests, which compare the former with the oracle and run
the latter through a race check and a host execution of the tile-task
semantics.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2211_13893_gb300", "csrc")
SOURCES = [os.path.join(HERE, "host_shim.cpp"), os.path.join(CSRC, "setup.cpp"), os.path.join(CSRC, "hexmesh.cpp")]
HEADERS = [os.path.join(CSRC, "internal.h"), os.path.join(ROOT, "include", "msgfem.h")]
LIB = os.path.join(HERE, "_build", "libhostcheck.so")

SC_FACTOR, SC_SOLVE_K, SC_SOLVE_A, SC_SOLVE_K8, SC_SOLVE_A8, SC_COARSE_FACTOR, SC_COARSE_SOLVE = range(7)
SOLVES = (SC_SOLVE_K, SC_SOLVE_A, SC_SOLVE_K8, SC_SOLVE_A8)
TILE, PST, KB = 64, 32, 8
SUB_FIELDS = ("I0", "I1", "J0", "J1", "oI0", "oI1", "oJ0", "oJ1", "nxn", "nyn", "nzn", "npl", "nnode", "nfull",
              "nK", "nA", "bK", "bA", "floating", "loaded", "pin0", "pin1", "pin2", "pin3", "pin4", "pin5",
              "n1", "n2", "n3")


def cuda_include():
    """Directory holding cuda_runtime.h (the set-up code includes it for types only), or None."""
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


def build():
    """Compile the harness if a source is newer than the library; returns its path."""
    inc = cuda_include()
    cxx = shutil.which("g++") or shutil.which("c++")
    if inc is None or cxx is None:
        raise RuntimeError("host harness needs a C++ compiler and the CUDA headers")
    stamp = max(os.path.getmtime(p) for p in SOURCES + HEADERS)
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= stamp:
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([cxx, "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", inc, *SOURCES, "-o", tmp], check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, ip, dp, i, d = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int, C.c_double
        L.hc_create.restype = vp
        L.hc_create.argtypes = [i, i, i, d, d, d, d, i, i, i, i, i, vp, vp, i, i, vp]
        L.hc_status.argtypes = [vp]
        L.hc_error.restype = C.c_char_p
        L.hc_error.argtypes = [vp]
        L.hc_destroy.argtypes = [vp]
        L.hc_num_subdomains.argtypes = [vp]
        L.hc_sub_ints.argtypes = [vp, i, ip]
        L.hc_sub_arrays.argtypes = [vp, i, vp, vp, vp, vp, vp]
        L.hc_sub_bytes.restype = C.c_longlong
        L.hc_sub_bytes.argtypes = [vp, i]
        L.hc_plan_waves.argtypes = [vp, d]
        L.hc_pool_bytes.restype = C.c_longlong
        L.hc_pool_bytes.argtypes = [vp]
        L.hc_wave_members.argtypes = [vp, i, ip]
        L.hc_build_wave.argtypes = [vp, i, i, i, i]
        L.hc_sub_ptr.restype = vp
        L.hc_sub_ptr.argtypes = [vp, i, i]
        L.hc_build_coarse.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
        L.hc_sched_shape.argtypes = [vp, i, ip]
        L.hc_race_check.restype = C.c_longlong
        L.hc_race_check.argtypes = [vp, i, vp, vp, i, C.c_char_p, i]
        L.hc_run_factor.argtypes = [vp, i, C.c_uint]
        L.hc_run_solve.argtypes = [vp, i, vp, vp, i, i, C.c_uint]
        L.hc_merge_steps.argtypes = [vp, i, i, i]
        L.hc_element_types.argtypes = [vp, vp, vp, ip, vp, vp, vp]
        L.hc_pairs.argtypes = [vp, vp]
        L.hc_build_wave_virtual.argtypes = [vp, i, i, i, i]
        L.hc_factor_task_flops.restype = d
        L.hc_factor_task_flops.argtypes = [vp]
        L.hc_align_check.restype = C.c_longlong
        L.hc_align_check.argtypes = [vp, i, C.c_char_p, i]
        L.hc_set_persistent.argtypes = [vp, i]
        L.hc_tma_check.restype = C.c_longlong
        L.hc_tma_check.argtypes = [vp, i, C.c_char_p, i]
        L.hc_persistent_tasks.restype = C.c_longlong
        L.hc_persistent_tasks.argtypes = [vp]
        L.hc_run_factor_persistent.argtypes = [vp, i, C.c_uint]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


class HostSetup:
    """The library's host-side set-up of one mesh and partition."""

    def __init__(self, cfg, instances=1, mixed=False, xyz=None, boxes=None, load=None):
        L = lib()
        self.L = L
        section = getattr(cfg, "kind", "beam") == "section"
        if section and xyz is None:
            from workloads.section import section_nodes
            xyz = section_nodes(cfg)
        if section and boxes is None:
            boxes = np.array(cfg.boxes)
        self._xyz = None if xyz is None else np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
        self._boxes = None if boxes is None else np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1)
        self._load = None if load is None else np.ascontiguousarray(load, dtype=np.float64).reshape(-1)
        nb = 0 if self._boxes is None else len(self._boxes) // 4
        hx, hy, hz = (0.0, 0.0, 0.0) if section else (cfg.hx, cfg.hy, cfg.t)
        self.h = L.hc_create(cfg.NX, cfg.NY, cfg.NZ, hx, hy, hz, cfg.traction, cfg.sx, cfg.sy, cfg.overlap,
                             cfg.oversampling, nb, _p(self._boxes), _p(self._xyz), instances, int(mixed),
                             _p(self._load))
        self.status = L.hc_status(self.h)
        self.error = L.hc_error(self.h).decode()
        self.N = L.hc_num_subdomains(self.h)
        self.mixed = bool(mixed)
        self.dtype = np.float32 if mixed else np.float64

    def close(self):
        if self.h:
            self.L.hc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def sub(self, j):
        out = (C.c_int * len(SUB_FIELDS))()
        assert self.L.hc_sub_ints(self.h, j, out) == 0
        d = dict(zip(SUB_FIELDS, list(out)))
        d["pins"] = [d.pop(f"pin{i}") for i in range(6)]
        return d

    def arrays(self, j):
        s = self.sub(j)
        cls = np.zeros(s["npl"], dtype=np.int8)
        mu = np.zeros(s["nnode"])
        load = np.zeros(s["nfull"])
        mapK = np.zeros(s["bK"], dtype=np.int32)
        mapA = np.zeros(s["bA"], dtype=np.int32)
        assert self.L.hc_sub_arrays(self.h, j, _p(cls), _p(mu), _p(load), _p(mapK), _p(mapA)) == 0
        return {"cls": cls, "mu": mu, "load": load, "mapK": mapK, "mapA": mapA}

    def sub_bytes(self, j):
        return self.L.hc_sub_bytes(self.h, j)

    def plan_waves(self, budget_bytes):
        return self.L.hc_plan_waves(self.h, float(budget_bytes))

    @property
    def pool_bytes(self):
        return self.L.hc_pool_bytes(self.h)

    def members(self, w):
        out = (C.c_int * self.N)()
        n = self.L.hc_wave_members(self.h, w, out)
        assert n >= 0
        return list(out)[:n]

    def build_wave(self, w, groups_factor=16, groups_solve=16, left=False):
        assert self.L.hc_build_wave(self.h, w, groups_factor, groups_solve, int(left)) == 0

    def blocks(self, j, matrix):
        """Views (D, E, Linv) of subdomain j's layer blocks of K ('K') or A11 ('A')."""
        s = self.sub(j)
        b = s["bK"] if matrix == "K" else s["bA"]
        nz = s["nzn"]
        base = 0 if matrix == "K" else 2
        ct = C.c_float if self.mixed else C.c_double
        pd = self.L.hc_sub_ptr(self.h, j, base)
        pl = self.L.hc_sub_ptr(self.h, j, base + 1)
        de = np.ctypeslib.as_array((ct * (b * b * (2 * nz - 1))).from_address(pd)).reshape(2 * nz - 1, b, b)
        li = np.ctypeslib.as_array((ct * (b * b * nz)).from_address(pl)).reshape(nz, b, b)
        return de[:nz], de[nz:], li

    def build_coarse(self, ncpad, AH, AHinv, bH, rH, yH, cH):
        self._coarse = (AH, AHinv, bH, rH, yH, cH)
        assert self.L.hc_build_coarse(self.h, ncpad, *[_p(a) for a in self._coarse]) == 0

    def shape(self, which):
        out = (C.c_int * 3)()
        assert self.L.hc_sched_shape(self.h, which, out) == 0
        return tuple(out)

    def _mv(self, arrs):
        if arrs is None:
            return None, None
        ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data if a is not None else None for a in arrs])
        return ptrs, arrs

    def race(self, which, src=None, dst=None, scatter_add=False):
        ps, _ = self._mv(src)
        pd, _ = self._mv(dst)
        msg = C.create_string_buffer(200)
        n = self.L.hc_race_check(self.h, which, ps, pd, int(scatter_add), msg, 200)
        return n, msg.value.decode()

    def run_factor(self, seed=0, coarse=False):
        return self.L.hc_run_factor(self.h, int(coarse), seed)

    def tma_check(self, which):
        """Violations of the TMA solve ring's slab preconditions (count, first one)."""
        msg = C.create_string_buffer(200)
        n = self.L.hc_tma_check(self.h, which, msg, 200)
        return n, msg.value.decode()

    def set_persistent(self, on=True):
        """Build the persistent factorisation's ticket order with the next build_wave."""
        self.L.hc_set_persistent(self.h, int(on))

    def persistent_tasks(self):
        return self.L.hc_persistent_tasks(self.h)

    def run_factor_persistent(self, window, seed=0):
        """Run the persistent ticket order as `window` resident CTAs would (see host_shim.cpp)."""
        return self.L.hc_run_factor_persistent(self.h, window, seed)

    def run_solve(self, which, src, dst, gather_neg=False, scatter_add=False, seed=0):
        ps, _ = self._mv(src)
        pd, _ = self._mv(dst)
        assert self.L.hc_run_solve(self.h, which, ps, pd, int(gather_neg), int(scatter_add), seed) == 0

    def element_types(self, angles, frames=None):
        """(layered, types, etype, trep) of an angle field, as the library decides them."""
        ang = np.ascontiguousarray(angles, dtype=np.float64).reshape(-1)
        fr = None if frames is None else np.ascontiguousarray(frames, dtype=np.float64).reshape(-1)
        n = len(ang)
        types = np.zeros(n)
        etype = np.full(n, -1, dtype=np.int32)
        trep = np.full(n, -1, dtype=np.int32)
        lay = C.c_int()
        nt = self.L.hc_element_types(self.h, _p(ang), _p(fr), C.byref(lay), _p(types), _p(etype), _p(trep))
        return bool(lay.value), types[:nt], etype, trep[:nt]

    def pairs(self):
        """Coarse pairs as an (n, 6) array: s, t and the node box x0, x1, y0, y1."""
        n = self.L.hc_pairs(self.h, None)
        out = np.zeros((n, 6), dtype=np.int32)
        self.L.hc_pairs(self.h, _p(out))
        return out

    def align_check(self, which):
        """Violations of the tile kernels' alignment preconditions and of the
        schedule's summary flags (count, first one)."""
        msg = C.create_string_buffer(200)
        n = self.L.hc_align_check(self.h, which, msg, 200)
        return n, msg.value.decode()

    def build_wave_virtual(self, w, groups_factor=16, groups_solve=16, left=False):
        """Schedules of wave w without their memory (task counts and work only)."""
        assert self.L.hc_build_wave_virtual(self.h, w, groups_factor, groups_solve, int(left)) == 0

    def factor_task_flops(self):
        return self.L.hc_factor_task_flops(self.h)

    def merge_steps(self, which, group, step):
        return self.L.hc_merge_steps(self.h, which, group, step)
