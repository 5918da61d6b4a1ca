"""ctypes binding of libmsgfem (include/msgfem.h): argument marshalling only.

Every step of the local stage runs in the library's CUDA kernels; this module
only converts arrays and reports status codes.  It fails loudly when the
library has not been built.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmsgfem.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTSPD", 5: "ENOCONV", 6: "ESTATE"}
EXPORTS = ("msgfem_setup", "msgfem_update_angles", "msgfem_local_spaces", "msgfem_local_spaces_var",
           "msgfem_coarse_assemble",
           "msgfem_solve", "msgfem_get_basis", "msgfem_get_info", "msgfem_num_subdomains",
           "msgfem_get_profile", "msgfem_reset_profile", "msgfem_energy_error_noalloc", "msgfem_last_error",
           "msgfem_autotune", "msgfem_coarse_assemble_threshold", "msgfem_solution_errors", "msgfem_plan",
           "msgfem_export_local", "msgfem_import_local", "msgfem_probe_fma", "msgfem_schwarz_solve",
           "msgfem_get_numbering",
           "msgfem_destroy",
           # include/msgfem_warm.h
           "msgfem_net_create", "msgfem_net_param_count", "msgfem_net_get_params", "msgfem_net_set_params",
           "msgfem_net_forward", "msgfem_net_gradient", "msgfem_net_adam_step", "msgfem_net_destroy",
           "msgfem_warm_features", "msgfem_warm_sizes", "msgfem_warm_targets", "msgfem_set_start_block")


class MsgfemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("hx", C.c_double), ("hy", C.c_double),
                ("hz", C.c_double), ("traction", C.c_double), ("xyz", C.c_void_p), ("load", C.c_void_p),
                ("kind", C.c_int), ("n_nodes", C.c_int), ("n_elems", C.c_int), ("node_xyz", C.c_void_p),
                ("hex8", C.c_void_p), ("dirichlet_node", C.c_void_p)]


class Plies(C.Structure):
    _fields_ = [("E9", C.c_void_p), ("elem_angle_deg", C.c_void_p), ("elem_frame", C.c_void_p)]


class Partition(C.Structure):
    _fields_ = [("sx", C.c_int), ("sy", C.c_int), ("n_boxes", C.c_int), ("boxes", C.c_void_p),
                ("elem_part", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("block", C.c_int), ("max_iter", C.c_int), ("tol", C.c_double),
                ("seed", C.c_ulonglong), ("stream", C.c_void_p), ("profile", C.c_int), ("solver", C.c_int),
                ("streams", C.c_int), ("refine", C.c_int), ("instances", C.c_int), ("solve_kernel", C.c_int),
                ("factor_schedule", C.c_int), ("direct_launch", C.c_int), ("wave_mb", C.c_double),
                ("dev_alloc", C.c_void_p), ("dev_free", C.c_void_p), ("alloc_ctx", C.c_void_p), ("method", C.c_int),
                ("factor_kernel", C.c_int), ("tile_chol", C.c_int), ("factor_persistent", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("n_subdomains", C.c_int), ("waves", C.c_int), ("pool_mb", C.c_double), ("blocks_mb", C.c_double),
                ("largest_mb", C.c_double), ("n_dof", C.c_longlong), ("max_star_dof", C.c_int)]


# msgfem_options.dev_alloc / dev_free
DEV_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class Tuning(C.Structure):
    _fields_ = [("factor_schedule", C.c_int), ("factor_streams", C.c_int), ("factor_ms", (C.c_double * 2) * 2),
                ("streams", C.c_int), ("solve_kernel", C.c_int), ("best_ms", C.c_double),
                ("solve_ms", (C.c_double * 4) * 4), ("factor_kernel", C.c_int),
                ("factor_ms_tc", (C.c_double * 2) * 2), ("tc_factor_diff", C.c_double),
                ("fma_factor_diff", C.c_double), ("factor_persistent", C.c_int),
                ("factor_ms_persistent", C.c_double * 2)]


class Profile(C.Structure):
    _fields_ = [("assemble_ms", C.c_double), ("factor_ms", C.c_double), ("solve_ms", C.c_double),
                ("iterate_ms", C.c_double), ("coarse_ms", C.c_double), ("factor_flops", C.c_double),
                ("solve_flops", C.c_double), ("launches", C.c_longlong), ("solve_calls", C.c_int),
                ("solve_bytes", C.c_double), ("stencil_ms", C.c_double), ("ortho_ms", C.c_double),
                ("stencil_flops", C.c_double), ("waves", C.c_int), ("pool_mb", C.c_double),
                ("factor_flops_inverse", C.c_double), ("factor_flops_executed", C.c_double)]


class PcgInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("residual", C.c_double), ("lambda_min", C.c_double),
                ("lambda_max", C.c_double), ("kappa", C.c_double)]


class SubInfo(C.Structure):
    _fields_ = [("n_star_dof", C.c_int), ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("floating", C.c_int),
                ("iterations", C.c_int), ("basis_size", C.c_int), ("residual", C.c_double),
                ("threshold_reached", C.c_int), ("cold_restart", C.c_int), ("n_loc", C.c_int)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libmsgfem.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2211_13893_gb300.build.build()")
    lib = C.CDLL(path)
    h = C.c_void_p
    sig = {
        "msgfem_setup": (C.c_int, [C.POINTER(Mesh), C.POINTER(Plies), C.POINTER(Partition), C.c_int, C.c_int,
                                   C.POINTER(Options), C.POINTER(h)]),
        "msgfem_update_angles": (C.c_int, [h, C.c_void_p]),
        "msgfem_local_spaces": (C.c_int, [h, C.c_int, C.c_void_p]),
        "msgfem_local_spaces_var": (C.c_int, [h, C.c_void_p, C.c_void_p]),
        "msgfem_coarse_assemble": (C.c_int, [h, C.POINTER(C.c_int)]),
        "msgfem_coarse_assemble_threshold": (C.c_int, [h, C.c_double, C.POINTER(C.c_int)]),
        "msgfem_solve": (C.c_int, [h, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
        "msgfem_get_basis": (C.c_int, [h, C.c_int, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_int)]),
        "msgfem_get_info": (C.c_int, [h, C.c_int, C.POINTER(SubInfo)]),
        "msgfem_get_numbering": (C.c_int, [h, C.c_void_p, C.c_void_p, C.c_void_p]),
        "msgfem_get_profile": (C.c_int, [h, C.POINTER(Profile)]),
        "msgfem_autotune": (C.c_int, [h, C.c_int, C.POINTER(Tuning)]),
        "msgfem_energy_error_noalloc": (C.c_int, [h, C.c_void_p, C.c_void_p, C.c_void_p]),
        "msgfem_solution_errors": (C.c_int, [h, C.c_void_p, C.POINTER(C.c_double)]),
        "msgfem_export_local": (C.c_int, [h, C.c_int, C.c_void_p, C.c_void_p]),
        "msgfem_import_local": (C.c_int, [h, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
        "msgfem_plan": (C.c_int, [C.POINTER(Mesh), C.POINTER(Partition), C.c_int, C.c_int, C.POINTER(Options),
                                  C.POINTER(PlanInfo)]),
        "msgfem_reset_profile": (C.c_int, [h]),
        "msgfem_probe_fma": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "msgfem_schwarz_solve": (C.c_int, [h, h, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                                           C.POINTER(PcgInfo)]),
        "msgfem_num_subdomains": (C.c_int, [h]),
        "msgfem_last_error": (C.c_char_p, [h]),
        "msgfem_destroy": (None, [h]),
        "msgfem_net_create": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(h)]),
        "msgfem_net_param_count": (C.c_longlong, [h]),
        "msgfem_net_get_params": (C.c_int, [h, C.c_void_p]),
        "msgfem_net_set_params": (C.c_int, [h, C.c_void_p]),
        "msgfem_net_forward": (C.c_int, [h, C.c_void_p, C.c_int, C.c_void_p]),
        "msgfem_net_gradient": (C.c_int, [h, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
        "msgfem_net_adam_step": (C.c_int, [h, C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.c_float, C.c_float,
                                           C.c_float, C.c_void_p]),
        "msgfem_net_destroy": (None, [h]),
        "msgfem_warm_features": (C.c_int, [h, C.c_void_p, C.c_float, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
        "msgfem_warm_sizes": (C.c_int, [h, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "msgfem_warm_targets": (C.c_int, [h, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
        "msgfem_set_start_block": (C.c_int, [h, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """Host numpy array (C-contiguous float64) or a torch CUDA tensor -> address."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class MSGFEM:
    """One MS-GFEM problem: a laminated hexahedral mesh, its decomposition and the handle.

    ``xyz`` (node coordinates), ``frames`` (per-element ply frames) and
    ``boxes`` (explicit subdomain boxes) are optional; without them the mesh
    is the box beam of bricks hx * hy * hz with the sx * sy partition."""

    def __init__(self, nx, ny, nz, hx, hy, hz, traction, E9, elem_angles, sx, sy, overlap, oversampling,
                 block=0, max_iter=0, tol=0.0, seed=0, stream=None, precision=0, profile=0, solver=0, streams=0, refine=0,
                 instances=0, xyz=None, frames=None, boxes=None, wave_mb=0.0, solve_kernel=0,
                 factor_schedule=0, direct_launch=0, allocator=None, load=None, method=0, hex8=None,
                 dirichlet=None, elem_part=None, factor_kernel=0, tile_chol=0, factor_persistent=0):
        """``allocator``: optional pair (alloc(nbytes) -> device address, free(address,
        nbytes)) through which the handle takes all its device memory.  ``load``:
        optional nodal forces [n_nodes * 3] replacing the end-face traction.
        ``method``: 0 MS-GFEM, 1 the GenEO comparison (oversampling = overlap).
        ``hex8``: a hexahedron list [n_elems, 8] (standard local order) with
        ``xyz`` [n_nodes, 3] its node coordinates; nx, ny, nz, hx, hy, hz are then
        ignored and the structured numbering is recovered by the library.
        ``dirichlet``: per-node clamp flags; ``elem_part``: per-element part ids.
        ``tile_chol``: mixed precision, tile Cholesky of the FP32 factorisation in
        FP64 (0) or in FP32 with an FP64 retry on a non-positive pivot (1).
        ``factor_persistent``: mixed precision, the FP32 factorisation as one
        persistent launch (1) instead of the captured step schedule (0)."""
        self.lib = load_library()
        self.h = C.c_void_p()
        self._E9 = np.ascontiguousarray(E9, dtype=np.float64)
        ang = elem_angles
        if not hasattr(ang, "data_ptr"):
            ang = np.ascontiguousarray(ang, dtype=np.float64).reshape(-1)
        self._ang = ang
        self._xyz = None if xyz is None else np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
        self._frames = None if frames is None else np.ascontiguousarray(frames, dtype=np.float64).reshape(-1)
        self._boxes = None if boxes is None else np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1)
        self._load = None if load is None else np.ascontiguousarray(load, dtype=np.float64).reshape(-1)
        self._dir = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8).reshape(-1)
        self._epart = None if elem_part is None else np.ascontiguousarray(elem_part, dtype=np.int32).reshape(-1)
        if hex8 is not None:
            self._hex8 = np.ascontiguousarray(hex8, dtype=np.int32).reshape(-1)
            n_nodes = len(self._xyz) // 3
            self.mesh = Mesh(0, 0, 0, 0.0, 0.0, 0.0, traction, None, _ptr(self._load), 1, n_nodes,
                             len(self._hex8) // 8, _ptr(self._xyz), _ptr(self._hex8), _ptr(self._dir))
            self.n_dof = 3 * n_nodes
        else:
            self.mesh = Mesh(nx, ny, nz, hx, hy, hz, traction, _ptr(self._xyz), _ptr(self._load), 0, 0, 0, None,
                             None, _ptr(self._dir))
            self.n_dof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
        plies = Plies(self._E9.ctypes.data, _ptr(ang), _ptr(self._frames))
        nb = 0 if self._boxes is None else len(self._boxes) // 4
        part = Partition(sx, sy, nb, _ptr(self._boxes), _ptr(self._epart))
        opt = Options(precision, block, max_iter, tol, seed, stream, profile, solver, streams, refine, instances,
                      solve_kernel, factor_schedule, direct_launch, wave_mb)
        opt.method = method
        opt.factor_kernel = factor_kernel
        opt.tile_chol = tile_chol
        opt.factor_persistent = factor_persistent
        if allocator is not None:
            alloc, free = allocator
            # the callbacks must outlive the handle: kept on the instance
            self._alloc_cb = DEV_ALLOC(lambda n, ctx: alloc(n) or None)
            self._free_cb = DEV_FREE(lambda p, n, ctx: free(p, n))
            opt.dev_alloc = C.cast(self._alloc_cb, C.c_void_p).value
            opt.dev_free = C.cast(self._free_cb, C.c_void_p).value
        self.instances = max(1, instances)
        st = self.lib.msgfem_setup(C.byref(self.mesh), C.byref(plies), C.byref(part), overlap, oversampling,
                                   C.byref(opt), C.byref(self.h))
        self._check(st)
        self.N = self.lib.msgfem_num_subdomains(self.h)
        self.n_loc = None

    @classmethod
    def from_config(cls, cfg, angles, **kw):
        """A workload description: a box beam, or a curved section with node
        coordinates, ply frames and subdomain boxes (``workloads.section``)."""
        if getattr(cfg, "kind", "beam") == "section":
            from workloads.section import section_frames, section_nodes
            kw.setdefault("xyz", section_nodes(cfg))
            kw.setdefault("frames", section_frames(cfg))
            kw.setdefault("boxes", np.array(cfg.boxes))
            return cls(cfg.NX, cfg.NY, cfg.NZ, 0.0, 0.0, 0.0, cfg.traction, cfg.material, angles,
                       cfg.sx, cfg.sy, cfg.overlap, cfg.oversampling, **kw)
        return cls(cfg.NX, cfg.NY, cfg.NZ, cfg.hx, cfg.hy, cfg.t, cfg.traction, cfg.material, angles,
                   cfg.sx, cfg.sy, cfg.overlap, cfg.oversampling, **kw)

    def _check(self, st, allow=()):
        if st != 0 and st not in allow:
            msg = self.lib.msgfem_last_error(self.h) if self.h else b""
            raise MsgfemError(st, (msg or b"").decode())
        return st

    def update_angles(self, angles):
        if not hasattr(angles, "data_ptr"):
            angles = np.ascontiguousarray(angles, dtype=np.float64).reshape(-1)
        self._ang = angles
        self._check(self.lib.msgfem_update_angles(self.h, _ptr(angles)))

    def local_spaces(self, n_loc, lam_out=None, allow_noconv=False):
        """Returns eigenvalues (N, n_loc) (numpy) or fills lam_out (device tensor).
        n_loc may also be one count per subdomain (msgfem_local_spaces_var): the
        rows are then max(n_loc) long, NaN from a subdomain's own count on."""
        allow = (5,) if allow_noconv else ()
        if np.ndim(n_loc) == 0:
            n_loc = int(n_loc)
            self.n_loc = n_loc
            out = lam_out if lam_out is not None else np.zeros((self.N, n_loc))
            self._check(self.lib.msgfem_local_spaces(self.h, n_loc, _ptr(out)), allow=allow)
            return out
        if hasattr(n_loc, "data_ptr"):       # a device (or host) tensor of int32 counts
            if n_loc.numel() != self.N or str(n_loc.dtype) != "torch.int32" or not n_loc.is_contiguous():
                raise ValueError(f"n_loc needs {self.N} contiguous int32 counts")
            counts, ptr = n_loc.cpu().numpy(), n_loc.data_ptr()
        else:
            counts = np.ascontiguousarray(n_loc, dtype=np.int32).reshape(-1)
            if counts.shape[0] != self.N:
                raise ValueError(f"n_loc needs one count per subdomain ({self.N}), got {counts.shape[0]}")
            ptr = counts.ctypes.data
        self.n_loc = int(counts.max())
        out = lam_out if lam_out is not None else np.zeros((self.N, self.n_loc))
        self._check(self.lib.msgfem_local_spaces_var(self.h, ptr, _ptr(out)), allow=allow)
        return out

    def coarse_assemble(self, threshold=None):
        """Coarse Galerkin assembly; with a threshold t, subdomain j keeps the
        eigenvectors with 1 / lambda > t (msgfem_coarse_assemble_threshold)."""
        nc = C.c_int()
        if threshold is None:
            self._check(self.lib.msgfem_coarse_assemble(self.h, C.byref(nc)))
        else:
            self._check(self.lib.msgfem_coarse_assemble_threshold(self.h, float(threshold), C.byref(nc)))
        return nc.value

    def solve(self, u_ref=None, u_out=None):
        """Returns (u^G, energy error or None); u_out may be a device tensor."""
        u = u_out if u_out is not None else np.zeros(self.n_dof)
        err = C.c_double(-1.0)
        if u_ref is not None and not hasattr(u_ref, "data_ptr"):
            u_ref = np.ascontiguousarray(u_ref, dtype=np.float64)
        self._check(self.lib.msgfem_solve(self.h, _ptr(u), _ptr(u_ref), C.byref(err)))
        return u, (err.value if u_ref is not None else None)

    def solution_errors(self, u_ref):
        """(e_d, e_eps): relative L2 errors of the last coarse solution against
        u_ref (numpy array or device tensor), include/msgfem.h msgfem_solution_errors."""
        if not hasattr(u_ref, "data_ptr"):
            u_ref = np.ascontiguousarray(u_ref, dtype=np.float64)
        out = (C.c_double * 2)()
        self._check(self.lib.msgfem_solution_errors(self.h, _ptr(u_ref), out))
        return float(out[0]), float(out[1])

    def export_local(self, j):
        """Subdomain j's local space (include/msgfem.h msgfem_export_local):
        (phi [n_star_dof, n_loc + 1] = eigenvectors then psi_j, eigenvalues [n_loc])."""
        rows = C.c_int()
        self._check(self.lib.msgfem_get_basis(self.h, j, None, C.byref(rows), None, None))
        n = self.n_loc
        phi = np.zeros((n + 1) * rows.value)
        lam = np.zeros(n)
        self._check(self.lib.msgfem_export_local(self.h, j, phi.ctypes.data, lam.ctypes.data))
        return phi.reshape(n + 1, rows.value).T, lam

    def import_local(self, lam, phis):
        """Resume from exported local spaces (msgfem_import_local): lam [N, n_loc],
        phis[j] as returned by export_local ([n_star_dof_j, n_loc + 1]); the
        shapes are checked against this handle before the library reads them."""
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        if lam.ndim != 2 or lam.shape[0] != self.N or len(phis) != self.N:
            raise ValueError(f"lam must be [{self.N}, n_loc] with one phi per subdomain")
        n_loc = lam.shape[1]
        for j, p in enumerate(phis):
            if np.shape(p) != (self.basis_rows(j), n_loc + 1):
                raise ValueError(f"phi of subdomain {j} has shape {np.shape(p)}, expected "
                                 f"({self.basis_rows(j)}, {n_loc + 1})")
        cols = [np.ascontiguousarray(np.asarray(p, dtype=np.float64).T) for p in phis]
        ptrs = (C.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
        self._check(self.lib.msgfem_import_local(self.h, n_loc, lam.ctypes.data, ptrs))
        self.n_loc = n_loc

    def save_local(self, path):
        """Write the local stage to path (.npz: eigenvalues and every subdomain's
        exported space) with a JSON manifest next to it (path + '.json')."""
        import json
        out = [self.export_local(j) for j in range(self.N)]
        lam = np.stack([o[1] for o in out])
        np.savez(path, lam=lam, **{f"phi_{j}": o[0] for j, o in enumerate(out)})
        with open(str(path) + ".json", "w") as f:
            json.dump({"n_subdomains": self.N, "n_loc": int(self.n_loc), "n_dof": int(self.n_dof),
                       "n_star_dof": [int(o[0].shape[0]) for o in out],
                       "boxes": [list(self.basis_box(j)) for j in range(self.N)]}, f)

    def load_local(self, path):
        """Resume from a file written by save_local (the handle must be set up like
        the one that wrote it)."""
        import json
        with open(str(path) + ".json") as f:
            man = json.load(f)
        if man["n_subdomains"] != self.N or man["n_dof"] != self.n_dof:
            raise ValueError("the checkpoint was written for another problem")
        # the oversampling domains (their DoF counts and node boxes) must be the
        # ones of this handle: another overlap, oversampling or partition with the
        # same mesh would otherwise pass and be read with the wrong sizes
        rows = [self.basis_rows(j) for j in range(self.N)]
        if man.get("n_star_dof") != rows or man.get("boxes") != [list(self.basis_box(j)) for j in range(self.N)]:
            raise ValueError("the checkpoint's oversampling domains differ from this handle's")
        name = str(path) if str(path).endswith(".npz") else str(path) + ".npz"
        data = np.load(name)
        self.import_local(data["lam"], [data[f"phi_{j}"] for j in range(self.N)])

    def basis_rows(self, j):
        """DoFs of Omega*_j (rows of the layouts of basis / export_local)."""
        rows = C.c_int()
        self._check(self.lib.msgfem_get_basis(self.h, j, None, C.byref(rows), None, None))
        return rows.value

    def basis_box(self, j):
        """Node box (i0, i1, j0, j1) of Omega*_j."""
        box = (C.c_int * 4)()
        self._check(self.lib.msgfem_get_basis(self.h, j, None, None, None, box))
        return tuple(box)

    def basis(self, j):
        rows, cols, box = C.c_int(), C.c_int(), (C.c_int * 4)()
        self._check(self.lib.msgfem_get_basis(self.h, j, None, C.byref(rows), C.byref(cols), box))
        out = np.zeros(rows.value * cols.value)
        self._check(self.lib.msgfem_get_basis(self.h, j, out.ctypes.data, C.byref(rows), C.byref(cols), box))
        return out.reshape(cols.value, rows.value).T, tuple(box)

    def autotune(self, reps=0):
        """Time the block-solve launch shapes on this handle and adopt the fastest
        (include/msgfem.h msgfem_autotune); returns the choice and the timings."""
        t = Tuning()
        self._check(self.lib.msgfem_autotune(self.h, reps, C.byref(t)))
        return {"factor_schedule": t.factor_schedule, "factor_streams": t.factor_streams,
                "factor_ms": [[t.factor_ms[f][g] for g in range(2)] for f in range(2)],
                "streams": t.streams, "solve_kernel": t.solve_kernel, "best_ms": t.best_ms,
                "solve_ms": [[t.solve_ms[g][v] for v in range(4)] for g in range(4)],
                "factor_kernel": t.factor_kernel,
                "factor_ms_tc": [[t.factor_ms_tc[f][g] for g in range(2)] for f in range(2)],
                "tc_factor_diff": t.tc_factor_diff, "fma_factor_diff": t.fma_factor_diff,
                "factor_persistent": t.factor_persistent,
                "factor_ms_persistent": [t.factor_ms_persistent[f] for f in range(2)]}

    def schwarz_solve(self, coarse=None, b=None, u0=None, rtol=0.0, max_iter=0, u_out=None, allow_noconv=False):
        """Two-level additive Schwarz PCG for the fine problem (include/msgfem.h
        msgfem_schwarz_solve) with this handle's A11 factors as the local solves
        (oversampling = overlap) and ``coarse``'s coarse space (an MSGFEM after
        coarse_assemble, or None for one level).  Returns (u, info dict)."""
        u = u_out if u_out is not None else np.zeros(self.n_dof)
        if b is not None and not hasattr(b, "data_ptr"):
            b = np.ascontiguousarray(b, dtype=np.float64)
        if u0 is not None and not hasattr(u0, "data_ptr"):
            u0 = np.ascontiguousarray(u0, dtype=np.float64)
        inf = PcgInfo()
        self._check(self.lib.msgfem_schwarz_solve(self.h, coarse.h if coarse is not None else None, _ptr(b), _ptr(u0),
                                                  float(rtol), int(max_iter), _ptr(u), C.byref(inf)),
                    allow=(5,) if allow_noconv else ())
        return u, {k: getattr(inf, k) for k, _ in PcgInfo._fields_}

    def numbering(self):
        """(dims (nx, ny, nz), node_of_user, elem_of_user) of the structured numbering
        (include/msgfem.h msgfem_get_numbering)."""
        dims = (C.c_int * 3)()
        self._check(self.lib.msgfem_get_numbering(self.h, dims, None, None))
        nx, ny, nz = dims[0], dims[1], dims[2]
        nodes = np.zeros((nx + 1) * (ny + 1) * (nz + 1), dtype=np.int32)
        elems = np.zeros(nx * ny * nz, dtype=np.int32)
        self._check(self.lib.msgfem_get_numbering(self.h, None, nodes.ctypes.data, elems.ctypes.data))
        return (nx, ny, nz), nodes, elems

    def info(self, j):
        inf = SubInfo()
        self._check(self.lib.msgfem_get_info(self.h, j, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in SubInfo._fields_}

    def profile(self, reset=False):
        pr = Profile()
        self._check(self.lib.msgfem_get_profile(self.h, C.byref(pr)))
        if reset:
            self._check(self.lib.msgfem_reset_profile(self.h))
        return {k: getattr(pr, k) for k, _ in Profile._fields_}

    # learned warm start (include/msgfem_warm.h)
    def warm_features(self, dtheta, scale, feat, ld):
        """Fill feat (device float32 [N][ld]) from dtheta (device float64, one per element)."""
        nf = C.c_int()
        self._check(self.lib.msgfem_warm_features(self.h, _ptr(dtheta), scale, _ptr(feat), ld, C.byref(nf)))
        return nf.value

    def warm_sizes(self, j, n_loc=0):
        """(n2, nw): interface rows and wanted non-rigid pairs of subdomain j."""
        n2, nw = C.c_int(), C.c_int()
        self._check(self.lib.msgfem_warm_sizes(self.h, j, n_loc, C.byref(n2), C.byref(nw)))
        return n2.value, nw.value

    def warm_targets(self, j, out, ld, ref=None):
        """B2 rows of subdomain j's wanted eigenvectors into out (device float32 [n2][ld])."""
        self._check(self.lib.msgfem_warm_targets(self.h, j, _ptr(ref), _ptr(out), ld))

    def set_start_block(self, j, X0, ld=0, ncols=0):
        """Register X0 (device float32 [n2][ld]) as subdomain j's start block; None clears it."""
        self._check(self.lib.msgfem_set_start_block(self.h, j, _ptr(X0), ld, ncols))

    def close(self):
        if self.h:
            self.lib.msgfem_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """Warm-start network (include/msgfem_warm.h): MLP with tanh hidden layers, FP32."""

    def __init__(self, sizes, max_batch, params=None, stream=None):
        self.lib = load_library()
        self.h = C.c_void_p()
        self.sizes = [int(x) for x in sizes]
        sz = (C.c_int * len(self.sizes))(*self.sizes)
        init = None
        if params is not None:
            init = np.ascontiguousarray(params, dtype=np.float32)
        st = self.lib.msgfem_net_create(len(self.sizes), sz, int(max_batch), _ptr(init), stream, C.byref(self.h))
        if st != 0:
            raise MsgfemError(st, "msgfem_net_create")
        self.n_params = int(self.lib.msgfem_net_param_count(self.h))

    def _check(self, st, what):
        if st != 0:
            raise MsgfemError(st, what)

    def params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        self._check(self.lib.msgfem_net_get_params(self.h, out.ctypes.data), "get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.msgfem_net_set_params(self.h, p.ctypes.data), "set_params")

    def forward(self, X, Y, batch):
        self._check(self.lib.msgfem_net_forward(self.h, _ptr(X), int(batch), _ptr(Y)), "forward")

    def gradient(self, X, T, batch):
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_double()
        self._check(self.lib.msgfem_net_gradient(self.h, _ptr(X), _ptr(T), int(batch), g.ctypes.data,
                                                 C.addressof(loss)), "gradient")
        return loss.value, g

    def adam_step(self, X, T, batch, lr, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=False):
        loss = C.c_double()
        self._check(self.lib.msgfem_net_adam_step(self.h, _ptr(X), _ptr(T), int(batch), lr, beta1, beta2, eps,
                                                  C.addressof(loss) if want_loss else None), "adam_step")
        return loss.value if want_loss else None

    def close(self):
        if self.h:
            self.lib.msgfem_net_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_fma(precision=0):
    """FMA throughput of the current device in TFLOP/s (include/msgfem.h
    msgfem_probe_fma): precision 0 = FP64, 1 = FP32."""
    lib = load_library()
    tf, sms = C.c_double(), C.c_double()
    st = lib.msgfem_probe_fma(precision, C.byref(tf), C.byref(sms))
    if st != 0:
        raise MsgfemError(st, "msgfem_probe_fma")
    return tf.value, int(sms.value)


def plan(cfg, precision=0, wave_mb=0.0, instances=0):
    """Device storage of a workload (include/msgfem.h msgfem_plan), planned on the
    host without a GPU: dict of the msgfem_plan_info fields and the status."""
    lib = load_library()
    section = getattr(cfg, "kind", "beam") == "section"
    xyz = boxes = None
    if section:
        from workloads.section import section_nodes
        xyz = np.ascontiguousarray(section_nodes(cfg), dtype=np.float64).reshape(-1)
        boxes = np.ascontiguousarray(cfg.boxes, dtype=np.int32).reshape(-1)
        mesh = Mesh(cfg.NX, cfg.NY, cfg.NZ, 0.0, 0.0, 0.0, cfg.traction, _ptr(xyz), None)
    else:
        mesh = Mesh(cfg.NX, cfg.NY, cfg.NZ, cfg.hx, cfg.hy, cfg.t, cfg.traction, None, None)
    part = Partition(cfg.sx, cfg.sy, 0 if boxes is None else len(boxes) // 4, _ptr(boxes))
    opt = Options()
    opt.precision, opt.wave_mb, opt.instances = precision, wave_mb, instances
    info = PlanInfo()
    st = lib.msgfem_plan(C.byref(mesh), C.byref(part), cfg.overlap, cfg.oversampling, C.byref(opt), C.byref(info))
    out = {k: getattr(info, k) for k, _ in PlanInfo._fields_}
    out["status"] = STATUS.get(st, st)
    return out
