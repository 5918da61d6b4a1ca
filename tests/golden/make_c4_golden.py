"""Write tests/golden/c4_sample_eigs.json: oracle eigenvalues of sampled
subdomains of the full c4 C-section spar (250 x 110 x 32 curved hexahedra,
2,758,239 DoF, 256 subdomains).

Calls only oracle/ (and the seeded generators of workloads/): the curved mesh
and ply frames, the partition of unity of all 256 subdomains (Sec. 4.2), and
for each sampled subdomain the A-harmonic local eigenproblem (Eq.
AHarmonicGeneralizeEigenProblem) in the dense-reduced form for every sample,
with the sample's own eigenpair count (16 to 31, growing with the size of
its oversampling domain, workloads.section.n_loc_per_subdomain).
(ARPACK shift-invert on the saddle pencil, the paper's own design, missed one
copy of the six-fold zero eigenvalue of the floating corner domain 83: a
single-vector Lanczos need not resolve every copy of a multiple eigenvalue,
so it is not used for stored values.)  The samples cover the smallest domain
(clamped end, flange tip), a clamped corner domain, a floating domain over a
curved corner and a floating domain on the loaded end.

    python tests/golden/make_c4_golden.py

Takes about six minutes on 8 cores.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_sample_eigs.json")
SAMPLES = {0: "dense", 18: "dense", 83: "dense", 248: "dense"}


def main():
    from oracle.arpack import local_eigs_arpack
    from oracle.assemble import make_cache
    from oracle.local import local_eigs_dense, local_problem
    from oracle.mesh import make_mesh
    from oracle.partition import partition_of_unity, subdomains
    from workloads import element_angles, get_config
    from workloads.section import n_loc_per_subdomain
    cfg = get_config("c4")
    counts = n_loc_per_subdomain(cfg)
    t0 = time.time()
    m = make_mesh(cfg)
    ang = element_angles(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(m, subs, cfg.overlap)
    b = m.compression_load(cfg.traction)
    cache = make_cache(m, cfg.material)
    print(f"mesh, partition of unity and load: {time.time() - t0:.1f} s", flush=True)
    out = {"config": "c4", "n_loc": [cfg.n_loc, cfg.n_loc_max], "samples": {}}
    for j, how in SAMPLES.items():
        t1 = time.time()
        lp = local_problem(m, ang, cfg.material, subs[j], mus[j], b, cache)
        lam, _ = (local_eigs_dense if how == "dense" else local_eigs_arpack)(lp, int(counts[j]))
        out["samples"][str(j)] = {"solver": how, "n_loc": int(counts[j]), "n_star_dof": int(lp.n_star),
                                  "n1": int(len(lp.I1)),
                                  "n2": int(len(lp.I2)), "n3": int(len(lp.I3)), "star": list(subs[j].star),
                                  "lambda": [float(x) for x in lam]}
        print(f"subdomain {j}: {lp.n_star} DoF, n2 {len(lp.I2)}, {how}, {time.time() - t1:.1f} s, "
              f"lambda[:4] {np.array(lam[:4])}", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
