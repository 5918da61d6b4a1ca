"""Write tests/golden/c2_oracle.json: oracle results for the full c2 workload.

Calls only oracle/ (and the seeded generators of workloads/): the dense-reduced
local eigensolver (Eq. algebraicAharmonic in reduced form) for every one of
the 32 subdomains, the Gram-Schmidt'd PoU basis with the particular functions
appended (Sec. 4.4, variant ii), the coarse Galerkin solve (Eq.
GFEM_coarse_approximation), the fine solution u_h (Eq. fe_matrix_system) by a
banded Cholesky, and the relative energy error of u^G (Thm. error_bound).
The coarse solution u^G itself goes to c2_oracle_uG.npy.

    python tests/golden/make_c2_golden.py [--workers 8]

Takes about ten minutes on 8 cores (one subdomain per worker, spawn pool).
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle.json")
# the oracle's coarse solution u^G on all 301,080 DoFs (float64, .npy)
OUT_UG = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle_uG.npy")


def _local(j):
    from oracle.assemble import ElementCache
    from oracle.coarse import gram_schmidt
    from oracle.local import local_eigs_dense, local_problem, particular
    from oracle.mesh import BeamMesh
    from oracle.partition import partition_of_unity, subdomains
    from workloads import element_angles, get_config
    cfg = get_config("c2")
    mesh = BeamMesh.from_config(cfg)
    ang = element_angles(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(mesh, subs, cfg.overlap)
    b = mesh.compression_load(cfg.traction)
    lp = local_problem(mesh, ang, cfg.material, subs[j], mus[j], b, cache=ElementCache(mesh, cfg.material))
    lam, phi = local_eigs_dense(lp, cfg.n_loc)
    psi = particular(lp)
    vecs = [lp.mu * phi[:, k] for k in range(phi.shape[1])]
    psi_w = lp.mu * psi
    if np.any(psi_w != 0.0):
        vecs.append(psi_w)
    Q = gram_schmidt(lp.A, vecs)
    gd = (3 * lp.nodes[:, None] + np.arange(3)).ravel()
    return j, np.asarray(lam), np.asarray(Q), gd


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import scipy.sparse as sp
    from oracle.assemble import ElementCache, assemble_global
    from oracle.coarse import coarse_solve
    from oracle.fine import energy_norm, solve_fine
    from oracle.mesh import BeamMesh
    from workloads import element_angles, get_config
    cfg = get_config("c2")
    t0 = time.time()
    # one BLAS thread per worker process (set before the workers start and import numpy)
    blas = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    with mp.get_context("spawn").Pool(args.workers) as pool:
        res = sorted(pool.map(_local, range(cfg.n_sub)), key=lambda r: r[0])
    t_local = time.time() - t0
    if blas is None:
        os.environ.pop("OMP_NUM_THREADS")
    else:
        os.environ["OMP_NUM_THREADS"] = blas
    mesh = BeamMesh.from_config(cfg)
    ang = element_angles(cfg)
    A = assemble_global(mesh, ang, cfg.material, cache=ElementCache(mesh, cfg.material))
    b = mesh.compression_load(cfg.traction)
    cols = []
    counts = []
    for _, _, Q, gd in res:
        counts.append(len(Q))
        for q in Q:
            col = np.zeros(mesh.n_dof)
            col[gd] = q
            cols.append(col)
    V = sp.csc_matrix(np.stack(cols, axis=1))
    AH = (V.T @ (A @ V)).toarray()
    AH = 0.5 * (AH + AH.T)
    c = coarse_solve(AH, V.T @ b)
    uG = V @ c
    uh = solve_fine(mesh, A, b)
    err = energy_norm(A, uh - uG) / energy_norm(A, uh)
    out = {
        "source": "oracle/ (dense-reduced local eigensolver, Gram-Schmidt basis with psi appended, "
                  "coarse Galerkin solve, banded-Cholesky fine solution); written by tests/golden/make_c2_golden.py",
        "config": "c2", "n_loc": cfg.n_loc,
        "lam": [[float(x) for x in r[1][:cfg.n_loc]] for r in res],
        "basis_counts": counts,
        "energy_error": float(err),
        "uh_energy": float(energy_norm(A, uh)),
        "seconds_local": t_local, "seconds_total": time.time() - t0,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    np.save(OUT_UG, np.asarray(uG, dtype=np.float64))
    print(f"wrote {OUT}: energy error {err:.6e}, {t_local:.0f} s local, {time.time() - t0:.0f} s total")


if __name__ == "__main__":
    main()
