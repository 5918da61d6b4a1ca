"""Write tests/golden/c3_sample_eigs.json: oracle eigenvalues of sampled
subdomains of the c3 beam (384 x 24 x 48 hexahedra, 1,414,875 DoF, 64
subdomains of up to 52k DoF, n_loc = 24).

Calls only oracle/ (and the seeded generators of workloads/): the beam, the
partition of unity of all 64 subdomains (Sec. 4.2), and for each sample the
A-harmonic local eigenproblem (Eq. AHarmonicGeneralizeEigenProblem) in the
dense-reduced form (exact up to rounding).  The samples are the clamped
subdomain at x = 0, a floating interior one and the loaded one at x = L.

    python tests/golden/make_c3_golden.py

Takes about half an hour on 8 cores.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_sample_eigs.json")
SAMPLES = (0, 31, 63)


def main():
    from oracle.assemble import make_cache
    from oracle.local import local_eigs_dense, local_problem
    from oracle.mesh import make_mesh
    from oracle.partition import partition_of_unity, subdomains
    from workloads import element_angles, get_config
    cfg = get_config("c3")
    t0 = time.time()
    m = make_mesh(cfg)
    ang = element_angles(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(m, subs, cfg.overlap)
    b = m.compression_load(cfg.traction)
    cache = make_cache(m, cfg.material)
    print(f"mesh, partition of unity and load: {time.time() - t0:.1f} s", flush=True)
    out = {"config": "c3", "n_loc": cfg.n_loc, "samples": {}}
    for j in SAMPLES:
        t1 = time.time()
        lp = local_problem(m, ang, cfg.material, subs[j], mus[j], b, cache)
        lam, _ = local_eigs_dense(lp, cfg.n_loc + 1)
        out["samples"][str(j)] = {"solver": "dense", "n_star_dof": int(lp.n_star), "n1": int(len(lp.I1)),
                                  "n2": int(len(lp.I2)), "n3": int(len(lp.I3)), "star": list(subs[j].star),
                                  "lambda": [float(x) for x in lam]}
        print(f"subdomain {j}: {lp.n_star} DoF, n2 {len(lp.I2)}, {time.time() - t1:.1f} s, "
              f"lambda[:4] {np.array(lam[:4])}", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
