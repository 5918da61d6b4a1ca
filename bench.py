"""Benchmark of the MS-GFEM local stage on GB300: local eigensolves per second.

One step = the whole hot path over one batch of subdomains: element stiffness
and subdomain matrices, layer-block factorisations, the A-harmonic local
eigenproblems to convergence with the particular functions, the PoU-weighted
coarse basis and Galerkin assembly, and the coarse solve with prolongation
(msgfem_local_spaces + msgfem_coarse_assemble + msgfem_solve).  value = the
subdomains processed per second (all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c2] [--impl ours|reference]
                  [--no-mixed] [--no-warm] [--no-cpu-baseline] [--streams S]

The JSON line's value is the plain FP64 form on the chosen beam (c2 by
default); it also carries
  roofline     the FP64 factorisation against the FP64 peak, with the phase
               times of solves, stencils and orthogonalisation;
  mixed        the same workload with FP32 factors and solves plus adaptive
               FP64 refinement: subdomains/s, the eigenvalue and energy-norm
               differences to the FP64 run, an HBM roofline entry for the
               FP32 solves, and (warm) a second input of the workload solved
               from the cold start and warm-started from the first input's
               eigenvectors;
  c4           the batched uneven C-section spar (250 x 110 x 32 curved hexes,
               256 subdomains of 4k-42k DoF, 16 to 31 eigenpairs each, growing
               with the subdomain's size) in mixed precision, all in one
               handle (memory-bounded waves when the factors do not fit):
               subdomains/s, phase times, the FP32-solve HBM roofline entry and
               the eigenvalues of sampled subdomains against stored oracle
               values;
  warm_c5      the learned warm start on the wrinkled c1 beam (512 samples,
               384 for training), 128 beams batched per local stage: cold
               start vs nominal-basis reuse vs trained network;
  aspect       the element aspect-ratio study (in-plane edge 1, 4, 8, 15 ply
               thicknesses): 1/lambda decay, mixed vs FP64, iterations;
  cpu_baseline the oracle on a sample of the workload's subdomains, one per
               host core.
Under torchrun (N > 1) every rank runs an independent replica of the workload
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk x 2 flop x max SM clock (derived, 1.26)


def _hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s), else the fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback (6.8 TB/s)"
METRIC = "local eigensolves/s on 1 GB300 at fixed energy-norm error: plain FP64 vs mixed+warm"
L2_BYTES = 129 * 2 ** 20

# DRAM traffic (bytes) of one FP64 layer-block factorisation (one replay of its graph):
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one factorisation graph launch on
# p2 (six c2-sized subdomains, 6.184 GB); c2 scaled by 32 / 6 subdomains.
NCU_TRAFFIC = {"p2": 6.184e9, "c2": 6.184e9 * 32 / 6}


class _Range:
    """NVTX range around a timed region (lets ncu --nvtx-include select it); no-op without NVTX."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        try:
            import torch
            torch.cuda.nvtx.range_push(self.name)
            self.on = True
        except Exception:
            self.on = False
        return self

    def __exit__(self, *exc):
        if self.on:
            import torch
            torch.cuda.nvtx.range_pop()
        return False


def max_over_ranks(x, world, device):
    """The largest value of x over all ranks (every rank gets it); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, steps, total_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank * steps / (total_ms / 1000.0)


def _solve_kernel_name(tuning):
    """Kernel of the FP32 8-column block solves for the autotuner's choice (default: the cp.async ring)."""
    k = (tuning or {}).get("solve_kernel", 1)
    return {1: "k_solve_async (FP32 block solves, 8 right-hand sides, cp.async ring)",
            2: "k_solve_stream<float, 1> (FP32 block solves, 8 right-hand sides, register streaming)",
            3: "k_solve_stream<float, 2> (FP32 block solves, 8 right-hand sides, two-CTA cluster)",
            4: "k_solve_tma (FP32 block solves, 8 right-hand sides, TMA-filled ring)"}.get(k, str(k))


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def workload_desc(cfg):
    if getattr(cfg, "kind", "beam") == "section":
        return (f"C-section spar {cfg.NX}x{cfg.NY}x{cfg.NZ} curved hex ({cfg.n_dof} DoF, {cfg.NZ} plies), "
                f"{cfg.n_sub} subdomains ({cfg.sx} x {cfg.sy} graded boxes), overlap {cfg.overlap}, "
                f"oversampling {cfg.oversampling}, n_loc={cfg.n_loc}")
    return (f"laminated beam {cfg.NX}x{cfg.NY}x{cfg.NZ} hex ({cfg.n_dof} DoF, {cfg.NZ} plies), "
            f"{cfg.sx}x{cfg.sy} subdomains, overlap {cfg.overlap}, oversampling {cfg.oversampling}, "
            f"n_loc={cfg.n_loc}, FP64")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle arm
def _oracle_sub(args):
    name, j, solver = args
    os.environ["OMP_NUM_THREADS"] = "1"
    import numpy as np  # noqa: F401
    from oracle.arpack import local_eigs_arpack
    from oracle.assemble import make_cache
    from oracle.local import local_eigs_dense, local_problem, particular
    from oracle.mesh import make_mesh
    from oracle.partition import partition_of_unity, subdomains
    from workloads import element_angles, get_config
    cfg = get_config(name)
    m = make_mesh(cfg)
    ang = element_angles(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(m, subs, cfg.overlap)
    t0 = time.perf_counter()
    lp = local_problem(m, ang, cfg.material, subs[j], mus[j], m.compression_load(cfg.traction),
                       make_cache(m, cfg.material))
    (local_eigs_arpack if solver == "arpack" else local_eigs_dense)(lp, cfg.n_loc)
    particular(lp)
    return time.perf_counter() - t0


def oracle_rate(name, n_sub_sample, cores, solver="arpack"):
    """Subdomains/s of the oracle on `n_sub_sample` subdomains run in parallel,
    one subdomain per core (a spawn pool: no fork after CUDA initialisation)."""
    from workloads import get_config
    cfg = get_config(name)
    ids = [(name, (5 + 7 * i) % cfg.n_sub, solver) for i in range(n_sub_sample)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(min(cores, n_sub_sample)) as pool:
        per = pool.map(_oracle_sub, ids)
    wall = time.perf_counter() - t0
    return n_sub_sample / wall, wall, per


def run_reference(args):
    """The oracle as the reference arm (the reference is paper text only).  One
    step = the local stage of one subdomain of the workload (its matrices,
    ARPACK shift-invert on the saddle pencil with SuperLU, the paper's solver
    design, and the particular function) on one host core.  The W warm-up steps
    and then the K timed steps run concurrently in a spawn pool, one subdomain
    per core as the paper runs one subdomain per rank, with as many workers as
    the rounds of the timed batch need (K = 20 on 16 cores: two rounds of 10);
    value = K / wall time of the timed batch."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from workloads import get_config
    cfg = get_config(args.config)
    cores = os.cpu_count() or 1
    steps = max(1, args.steps)
    rounds = -(-steps // cores)
    workers = -(-steps // rounds)
    ids = [(args.config, (5 + 7 * i) % cfg.n_sub, "arpack") for i in range(args.warmup + steps)]
    t_all = time.perf_counter()
    with mp.get_context("spawn").Pool(workers) as pool:
        if args.warmup:
            pool.map(_oracle_sub, ids[:args.warmup], chunksize=1)          # untimed warm-up steps
        t0 = time.perf_counter()
        per = pool.map(_oracle_sub, ids[args.warmup:], chunksize=1)
        wall = time.perf_counter() - t0
    value = steps / wall
    sample = (f"{steps} timed steps, each one subdomain of {args.config} (ARPACK shift-invert on the saddle pencil "
              f"with SuperLU, the paper's solver design), run concurrently on {workers} host cores in {rounds} "
              f"round(s); per-subdomain time {min(per):.1f}-{max(per):.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "subdomains/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(cfg), "name": args.config},
            "cpu_baseline": {"kind": "oracle", "cores": workers, "sample": sample, "value": value,
                             "unit": "subdomains/s"},
            "e2e": {"value": value, "unit": "subdomains/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import numpy as np
    import torch
    world, rank, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_2211_13893_gb300 import MSGFEM
    from workloads import element_angles, get_config
    cfg = get_config(args.config)
    ang = element_angles(cfg).reshape(-1)
    ang_dev = torch.tensor(ang, dtype=torch.float64, device=dev)
    probe = None
    if rank == 0:
        from paper_2211_13893_gb300.msgfem import probe_fma
        f64, sms = probe_fma(0)
        f32, _ = probe_fma(1)
        probe = {"fp64_tflops": f64, "fp32_tflops": f32, "sms": sms,
                 "note": "dependent-chain FMA loops on every SM (msgfem_probe_fma), CUDA events, before the timed steps"}
    stream = torch.cuda.current_stream(dev)
    m = MSGFEM.from_config(cfg, ang_dev, seed=1234 + rank, stream=stream.cuda_stream, profile=1,
                           streams=args.streams, direct_launch=int(args.direct_launch))
    lam_dev = torch.empty((m.N, cfg.n_loc), dtype=torch.float64, device=dev)
    u_dev = torch.empty(m.n_dof, dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        m.local_spaces(cfg.n_loc, lam_out=lam_dev)
        m.coarse_assemble()
        m.solve(u_out=u_dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    step()
    tuning = None
    if not args.no_autotune:
        t1 = time.perf_counter()
        tuning = m.autotune()                # factor schedule and block-solve launch shapes
        tuning["seconds"] = time.perf_counter() - t1
    for _ in range(max(1, args.warmup - 1)):
        step()
    barrier()
    m.profile(reset=True)
    launches0 = m.profile()["launches"]
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms = []
    for _ in range(args.steps):
        flush.zero_()                     # L2 flush between timed steps (not timed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with _Range("msgfem_timed"):
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    barrier()
    clocks = sampler.stop()
    prof = m.profile()
    launches = prof["launches"] - launches0
    total_ms = sum(ms)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = job_rate(world, m.N, args.steps, total_ms)
    # roofline of the dominant kernel class (FP64 ALU bound)
    fact_tf = prof["factor_flops"] * args.steps / (prof["factor_ms"] / 1000.0) / 1e12 if prof["factor_ms"] else 0.0
    fact_inv_tf = fact_tf * prof["factor_flops_inverse"] / prof["factor_flops"] if prof["factor_flops"] else 0.0
    fact_x_tf = fact_tf * prof["factor_flops_executed"] / prof["factor_flops"] if prof["factor_flops"] else 0.0
    solve_tf = prof["solve_flops"] * args.steps / (prof["solve_ms"] / 1000.0) / 1e12 if prof["solve_ms"] else 0.0
    if prof["solve_ms"] >= prof["factor_ms"]:
        dom, achieved, share = "k_solve_stream<double> (block triangular solves)", solve_tf, prof["solve_ms"] / total_ms
    else:
        dom, achieved, share = "k_tile_task<double> (layer-block Cholesky tile tasks)", fact_tf, prof["factor_ms"] / total_ms
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": NCU_TRAFFIC.get(args.config), "kernel": dom,
            "traffic_note": "bytes per factorisation graph replay (one per step), from an ncu capture on p2 scaled "
                            "to the workload's subdomains",
            "peak_note": "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (derived); measured by the FMA probe "
                         "in this run: see probe",
            "achieved_note": "algorithmic flops of the block-tridiagonal Cholesky of K and A11 (per matrix sum_l "
                             "n^3/3 + (nL-1) 2 n^3, unpadded layer sizes) over the factorisation phase's CUDA-event "
                             "time on the launching stream",
            "probe": probe,
            "time_share": share,
            "factor": {"tflops": fact_tf, "ms_per_step": prof["factor_ms"] / args.steps,
                       "tflops_with_inverse": fact_inv_tf, "tflops_executed": fact_x_tf,
                       "executed_over_algorithmic": prof["factor_flops_executed"] / prof["factor_flops"]
                       if prof["factor_flops"] else None},
            "solve": {"tflops": solve_tf, "ms_per_step": prof["solve_ms"] / args.steps,
                      "calls_per_step": prof["solve_calls"],
                      "gbs": prof["solve_bytes"] * args.steps / (prof["solve_ms"] / 1000.0) / 1e9
                      if prof["solve_ms"] else None},
            "stencil": {"ms_per_step": prof["stencil_ms"] / args.steps,
                        "tflops": prof["stencil_flops"] * args.steps / (prof["stencil_ms"] / 1000.0) / 1e12
                        if prof["stencil_ms"] else None},
            "ortho_ms_per_step": prof["ortho_ms"] / args.steps,
            "iterate_ms_per_step": prof["iterate_ms"] / args.steps,
            "assemble_ms_per_step": prof["assemble_ms"] / args.steps,
            "coarse_ms_per_step": prof["coarse_ms"] / args.steps}
    # end to end through the C ABI with host buffers
    ang_host = torch.tensor(ang, dtype=torch.float64).pin_memory()
    lam_host = torch.empty((m.N, cfg.n_loc), dtype=torch.float64).pin_memory()
    u_host = torch.empty(m.n_dof, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.update_angles(ang_host.numpy())
        m.local_spaces(cfg.n_loc, lam_out=lam_host.numpy())
        m.coarse_assemble()
        m.solve(u_out=u_host.numpy())
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_total = sum(e2e_ms)
    e2e_total = max_over_ranks(e2e_total, world, dev)
    e2e = {"value": world * m.N * args.steps / (e2e_total / 1000.0), "unit": "subdomains/s",
           "h2d_bytes_per_step": int(ang.nbytes), "d2h_bytes_per_step": int(lam_host.numel() * 8 + u_host.numel() * 8)}
    infos = [m.info(j) for j in range(m.N)]
    extra = {"iterations_max": max(i["iterations"] for i in infos),
             "residual_max": max(i["residual"] for i in infos),
             "lambda_sub5_head": [float(x) for x in lam_dev[5 % m.N, :8].cpu().numpy()]}
    tuning_fp64 = tuning
    lam_fp64 = lam_dev.clone()
    u_fp64 = u_dev.clone()
    m.close()
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed(args, cfg, ang_dev, stream, dev, rank, lam_fp64, u_fp64, flush, world)
    c4 = None
    if not args.no_c4:
        c4 = run_c4(args, dev, stream, flush, rank, world)
    warm = None
    if not args.no_warm and rank == 0:
        warm = run_warm_c5(args, dev)
    aspect = None
    if not args.no_aspect and rank == 0:
        aspect = run_aspect(args, dev, stream)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        n = max(1, min(cores, args.ref_sample))
        r, wall, per = oracle_rate(args.config, n, cores)
        cpu = {"value": r, "unit": "subdomains/s", "cores": min(cores, n), "kind": "oracle",
               "sample": f"{n} subdomains of {args.config}, ARPACK shift-invert + SuperLU (paper design), "
                         f"one per core, wall {wall:.1f} s"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "subdomains/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_desc(cfg), "name": args.config, "precision": "plain FP64",
                           "l2": "flushed between timed steps (256 MiB write); working set ~25 GB >> L2",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "solver": extra, "autotune": tuning_fp64, "mixed": mixed, "c4": c4,
                "warm_c5": warm, "aspect": aspect}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_c4(args, dev, stream, flush, rank, world):
    """The batched uneven C-section spar in mixed precision: one handle holding
    all 256 subdomains (oversampling domains of 4k-42k DoF), one step = local
    stage + coarse assembly + coarse solve, as for the main workload."""
    import numpy as np
    import torch
    from paper_2211_13893_gb300 import MSGFEM
    from workloads import element_angles, get_config
    from workloads.section import n_loc_per_subdomain, omega_star_sizes
    cfg = get_config("c4")
    counts = n_loc_per_subdomain(cfg)        # 16 .. 31 eigenpairs, growing with the subdomain's size
    t0 = time.perf_counter()
    ang = torch.tensor(element_angles(cfg).reshape(-1), dtype=torch.float64, device=dev)
    m = MSGFEM.from_config(cfg, ang, seed=11, stream=stream.cuda_stream, profile=1, precision=1,
                           streams=args.streams, factor_kernel=max(args.factor_kernel, 0),
                           solve_kernel=args.solve_kernel, tile_chol=args.tile_chol,
                           factor_persistent=args.factor_persistent)
    setup_s = time.perf_counter() - t0
    lam = torch.empty((m.N, int(counts.max())), dtype=torch.float64, device=dev)
    u = torch.empty(m.n_dof, dtype=torch.float64, device=dev)

    def step():
        m.local_spaces(counts, lam_out=lam, allow_noconv=True)   # unconverged pairs are reported below
        m.coarse_assemble()
        m.solve(u_out=u)

    step()                                   # warm-up: graph capture, first launches
    tuning = None
    if not args.no_autotune:
        t1 = time.perf_counter()
        tuning = m.autotune()                # launch shapes of the block solves on this batch
        tuning["seconds"] = time.perf_counter() - t1
        step()                               # re-capture the solve graphs with the chosen shapes
    torch.cuda.synchronize()
    m.profile(reset=True)
    ms = []
    for _ in range(args.c4_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with _Range("msgfem_timed_c4"):
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = m.profile()
    total = sum(ms)
    total = max_over_ranks(total, world, dev)
    k = args.c4_steps
    infos = [m.info(j) for j in range(m.N)]
    sizes = omega_star_sizes(cfg)
    hbm, hbm_note = _hbm_peak()
    solve_gbs = prof["solve_bytes"] * k / (prof["solve_ms"] / 1000.0) / 1e9 if prof["solve_ms"] else 0.0
    sample = None
    gold_path = os.path.join(ROOT, "tests", "golden", "c4_sample_eigs.json")
    if os.path.exists(gold_path):
        gold = json.load(open(gold_path))
        lh = lam.cpu().numpy()
        d = 0.0
        for key, rec in gold["samples"].items():
            ref = np.array(rec["lambda"])
            if len(ref) != counts[int(key)]:
                continue                     # a golden file written for other counts
            got = lh[int(key), :len(ref)]
            big = max(float(np.abs(ref).max()), 1.0)
            scale = np.where(np.abs(ref) > 1e-8 * big, np.abs(ref), big)
            d = max(d, float((np.abs(got - ref) / scale).max()))
        sample = {"subdomains": [int(x) for x in gold["samples"]], "eig_rel_diff_vs_oracle_max": d}
    out = {"workload": (f"C-section spar 250x110x32 curved hex ({cfg.n_dof} DoF, 32 plies), 256 subdomains "
                        f"(16 x 16 graded boxes), overlap 1, oversampling 3, n_loc {int(counts.min())}-"
                        f"{int(counts.max())} per subdomain (mean {counts.mean():.1f}, growing with its size), "
                        f"oversampling domains {int(sizes.min())}-{int(sizes.max())} DoF "
                        f"(mean {int(sizes.mean())}); mixed precision"),
           "value": world * m.N * k / (total / 1000.0), "unit": "subdomains/s", "ms_per_step": total / k,
           "setup_s": setup_s, "waves": prof["waves"], "pool_gb": prof["pool_mb"] / 1024.0,
           "assemble_ms_per_step": prof["assemble_ms"] / k, "factor_ms_per_step": prof["factor_ms"] / k,
           "factor_tflops": prof["factor_flops"] * k / (prof["factor_ms"] / 1000.0) / 1e12
           if prof["factor_ms"] else None,
           "solve_ms_per_step": prof["solve_ms"] / k, "iterate_ms_per_step": prof["iterate_ms"] / k,
           "stencil_ms_per_step": prof["stencil_ms"] / k, "ortho_ms_per_step": prof["ortho_ms"] / k,
           "coarse_ms_per_step": prof["coarse_ms"] / k,
           "iterations_max": max(i["iterations"] for i in infos),
           "residual_max": max(i["residual"] for i in infos),
           "unconverged_subdomains": [j for j, i in enumerate(infos) if i["residual"] > 1e-5],
           "roofline": {"bound": "hbm", "achieved": solve_gbs, "peak": hbm, "unit": "GB/s",
                        "frac": solve_gbs / hbm, "peak_note": hbm_note,
                        "kernel": _solve_kernel_name(tuning),
                        "time_share": prof["solve_ms"] / total if total else None},
           "sampled_parity": sample, "autotune": tuning}
    m.close()
    return out


def run_mixed(args, cfg, ang_dev, stream, dev, rank, lam_fp64, u_fp64, flush, world):
    """The same workload in mixed precision (FP32 factors and solves with FP64
    refinement); its solution is compared with the FP64 one in the energy norm."""
    import ctypes as C
    import torch
    from paper_2211_13893_gb300 import MSGFEM
    m = MSGFEM.from_config(cfg, ang_dev, seed=1234 + rank, stream=stream.cuda_stream, profile=1,
                           streams=args.streams, precision=1, direct_launch=int(args.direct_launch),
                           factor_kernel=max(args.factor_kernel, 0), solve_kernel=args.solve_kernel,
                           tile_chol=args.tile_chol, factor_persistent=args.factor_persistent)
    lam = torch.empty_like(lam_fp64)
    u = torch.empty_like(u_fp64)

    def step():
        m.local_spaces(cfg.n_loc, lam_out=lam)
        m.coarse_assemble()
        m.solve(u_out=u)

    step()
    tuning = None
    if not args.no_autotune:
        t1 = time.perf_counter()
        tuning = m.autotune()
        tuning["seconds"] = time.perf_counter() - t1
    for _ in range(max(2, args.warmup - 1)):
        step()
    torch.cuda.synchronize()
    m.profile(reset=True)
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with _Range("msgfem_timed_mixed"):
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = m.profile()
    total = sum(ms)
    total = max_over_ranks(total, world, dev)
    e = C.c_double(-1.0)
    m.lib.msgfem_energy_error_noalloc(m.h, u.data_ptr(), u_fp64.data_ptr(), C.addressof(e))
    hbm, hbm_note = _hbm_peak()
    solve_gbs = prof["solve_bytes"] * args.steps / (prof["solve_ms"] / 1000.0) / 1e9 if prof["solve_ms"] else 0.0
    rel = _eig_rel(lam, lam_fp64)
    warm = _c2_mixed_warm(cfg, m, stream, dev) if (not args.no_warm and rank == 0) else None
    out = {"value": world * m.N * args.steps / (total / 1000.0), "unit": "subdomains/s",
           "ms_per_step": total / args.steps, "dtype": "f32 factors/solves + f64 refinement/RR/coarse",
           "factor_ms_per_step": prof["factor_ms"] / args.steps, "solve_ms_per_step": prof["solve_ms"] / args.steps,
           "factor_tflops": prof["factor_flops"] * args.steps / (prof["factor_ms"] / 1000.0) / 1e12
           if prof["factor_ms"] else None,
           "eig_rel_diff_vs_fp64": rel, "energy_norm_diff_vs_fp64": e.value,
           "iterate_ms_per_step": prof["iterate_ms"] / args.steps,
           "stencil": {"ms_per_step": prof["stencil_ms"] / args.steps,
                       "tflops": prof["stencil_flops"] * args.steps / (prof["stencil_ms"] / 1000.0) / 1e12
                       if prof["stencil_ms"] else None},
           "ortho_ms_per_step": prof["ortho_ms"] / args.steps, "autotune": tuning,
           "roofline": {"bound": "hbm", "achieved": solve_gbs, "peak": hbm, "unit": "GB/s",
                        "frac": solve_gbs / hbm, "peak_note": hbm_note,
                        "kernel": _solve_kernel_name(tuning),
                        "time_share": prof["solve_ms"] / total if total else None,
                        "calls_per_step": prof["solve_calls"]},
           "warm": warm}
    m.close()
    return out


def _eig_rel(lam, ref):
    """Largest per-eigenvalue relative difference; rigid zeros (below 1e-8 of the
    subdomain's largest, floored at 1) compared at the scale 1."""
    import torch
    big = torch.clamp(ref.abs().amax(dim=1, keepdim=True), min=1.0)
    scale = torch.where(ref.abs() > 1e-8 * big, ref.abs(), torch.ones_like(ref))
    return ((lam - ref).abs() / scale).max().item()


def _c2_mixed_warm(cfg, m, stream, dev):
    """Mixed + warm on the metric's own workload, local stage only: a second
    input of the same beam (the next seed of the 1-degree ply-angle noise) is
    solved from the cold start and from the first input's eigenvectors
    (nominal-basis reuse through msgfem_set_start_block).  The block Krylov start
    block has 8 columns, so it carries the 8 lowest of the 20 (clamped) or 14
    (floating) wanted eigenvectors; the eigensolver iterates to the same
    tolerance either way."""
    from dataclasses import replace
    import torch
    from paper_2211_13893_gb300.warm import WarmStart
    from workloads import element_angles
    ws = WarmStart(m, cfg.n_loc, stream=stream.cuda_stream)
    m.local_spaces(cfg.n_loc)
    ws.set_nominal()
    nominal = ws.nominal_blocks()
    ang2 = element_angles(replace(cfg, noise_seed=cfg.noise_seed + 1)).reshape(-1)
    m.update_angles(torch.tensor(ang2, dtype=torch.float64, device=dev))
    out, lam = {}, {}
    for kind in ("cold", "warm"):
        ws.apply(None if kind == "cold" else nominal)
        ms = []
        for _ in range(2):                         # the second repetition is the timed one
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lam[kind] = m.local_spaces(cfg.n_loc).copy()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        its = [m.info(j)["iterations"] for j in range(m.N)]
        out[kind] = {"subdomains_per_s": m.N / (ms[-1] / 1000.0), "local_stage_ms": ms[-1],
                     "iterations_mean": float(sum(its) / len(its)), "iterations_max": int(max(its))}
    ws.apply(None)
    out["eig_rel_diff_warm_vs_cold"] = _eig_rel(torch.tensor(lam["warm"]), torch.tensor(lam["cold"]))
    out["workload"] = (f"{cfg.name} with the ply-angle noise of seed {cfg.noise_seed + 1}, mixed precision, local "
                       f"stage only; warm start: the 8 lowest eigenvectors per subdomain of the seed-"
                       f"{cfg.noise_seed} input")
    return out


def run_aspect(args, dev, stream):
    """The element aspect-ratio study (Sec. 5.3) on the GPU: the c1 topology with
    in-plane element edges of 1, 4, 8 and 15 ply thicknesses, oversampling 4,
    n_loc = 12, FP64 and mixed: 1/lambda of the wanted pairs of subdomain 0 (the
    decay that drives the error bound), the largest relative eigenvalue
    difference of the mixed run to the FP64 one, block iterations, residuals
    and the local-stage time.  Oracle parity at every aspect ratio is in
    tests/test_gpu_aspect.py."""
    import numpy as np
    import torch
    from paper_2211_13893_gb300 import MSGFEM
    from workloads import element_angles, get_config
    from workloads.configs import ASPECT_RATIOS
    out = {}
    for ar in ASPECT_RATIOS:
        cfg = get_config(f"a{ar}")
        ang = element_angles(cfg)
        rec = {}
        lam = {}
        for prec in (0, 1):
            m = MSGFEM.from_config(cfg, ang, seed=5, precision=prec, stream=stream.cuda_stream)
            m.local_spaces(cfg.n_loc)                       # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lam[prec] = m.local_spaces(cfg.n_loc)
            torch.cuda.synchronize()
            ms = 1000.0 * (time.perf_counter() - t0)
            infos = [m.info(j) for j in range(m.N)]
            rec["fp64" if prec == 0 else "mixed"] = {
                "local_stage_ms": ms, "iterations_max": max(i["iterations"] for i in infos),
                "residual_max": max(i["residual"] for i in infos)}
            m.close()
        l0 = lam[0][0]
        rec["inv_lambda_sub0"] = [float(1.0 / x) if x > 0 else None for x in l0]
        # non-rigid eigenvalues relative to themselves, rigid zeros at the scale 1
        scale = np.where(np.abs(lam[0]) > 1e-8 * np.maximum(np.abs(lam[0]).max(axis=1, keepdims=True), 1.0),
                         np.abs(lam[0]), 1.0)
        rec["mixed_eig_rel_diff_vs_fp64"] = float((np.abs(lam[1] - lam[0]) / scale).max())
        out[f"aspect_{ar}"] = rec
    cfg = get_config(f"a{ASPECT_RATIOS[0]}")
    out["workload"] = ("c1 topology 24x4x12, ply 0.25 mm, in-plane element edge = aspect ratio x ply thickness, "
                       f"2x1 subdomains, overlap {cfg.overlap}, oversampling {cfg.oversampling}, n_loc {cfg.n_loc}")
    return out


def run_warm_c5(args, dev, n_train=384, n_test=128, batch=128):
    """Learned warm start on the wrinkled c1 beam (c5): 512 seeded wrinkle
    fields, the network trained on the eigenbases of samples 0..383 (computed
    by the eigensolver itself, cold), tested on 384..511.  The samples run as
    batched instances of one handle (`batch` beams, 2 subdomains each, per
    local stage).  Reports block iterations to the 1e-6 energy-norm
    tolerance, the largest principal angle between the start block and the
    converged wanted space, and local-stage solves/s of the whole test batch
    for the cold start, nominal-basis reuse and the trained network (feature
    extraction and inference included in the warm timing)."""
    import numpy as np
    import torch
    from paper_2211_13893_gb300 import MSGFEM
    from paper_2211_13893_gb300.warm import WarmStart
    from workloads import element_angles, get_config, wrinkle_field
    cfg = get_config("c5")
    base = element_angles(cfg)
    nel = base.size
    stream = torch.cuda.current_stream(dev)
    S = batch
    t0 = time.perf_counter()
    fields = np.stack([wrinkle_field(cfg, s) for s in range(n_train + n_test)])
    m = MSGFEM.from_config(cfg, np.tile(base.reshape(-1), S), seed=5, tol=1e-6, stream=stream.cuda_stream,
                           instances=S)
    ws = WarmStart(m, cfg.n_loc, hidden=(32,), seed=3, stream=stream.cuda_stream)
    m.local_spaces(cfg.n_loc)
    ws.set_nominal()
    P = ws.P

    def load(first):
        f = fields[first:first + S]
        m.update_angles(torch.tensor((base[None] + f).reshape(-1), dtype=torch.float64, device=dev))
        return torch.tensor(f.reshape(-1), dtype=torch.float64, device=dev)

    X, T = [], [[] for _ in range(P)]
    for first in range(0, n_train, S):
        dth = load(first)
        m.local_spaces(cfg.n_loc)
        X.append(ws.features(dth).view(S, P, -1))
        tg = ws.targets()
        for j, t in enumerate(tg):
            T[j % P].append(t.reshape(-1))
    X = torch.cat(X)
    T = [torch.stack(t) for t in T]
    t_data = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = ws.fit(X, T, steps=4000, lr=3e-4, batch=64)
    e1.record(stream)
    e1.synchronize()
    train_ms = e0.elapsed_time(e1)

    def angle(A, B):
        qa, _ = np.linalg.qr(A)
        qb, _ = np.linalg.qr(B)
        sv = np.linalg.svd(qa.T @ qb, compute_uv=False)
        return float(np.arccos(np.clip(sv.min(), -1.0, 1.0)))

    dth = load(n_train)
    res = {}
    conv = None
    for kind in ("cold", "nominal", "learned"):
        ms = []
        for rep in range(2):                       # second repetition is the timed one
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if kind == "cold":
                blocks = None
            elif kind == "nominal":
                blocks = ws.nominal_blocks()
            else:
                blocks = ws.predict(ws.features(dth))
            ws.apply(blocks)
            m.local_spaces(cfg.n_loc)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        iters = [m.info(j)["iterations"] for j in range(m.N)]
        if conv is None:
            conv = [t.cpu().numpy() for t in ws.targets(ref=False)]
        angs = []
        rng = np.random.default_rng(7)
        for j in range(m.N):
            n2, nw = ws.size(j)
            start = blocks[j].cpu().numpy()[:, :nw] if blocks is not None else rng.standard_normal((n2, nw))
            angs.append(angle(start, conv[j][:, :nw]))
        res[kind] = {"iterations_mean": float(np.mean(iters)), "iterations_max": int(np.max(iters)),
                     "start_angle_rad_mean": float(np.mean(angs)),
                     "solves_per_s": m.N / (ms[-1] / 1000.0), "ms_per_batch": ms[-1]}
    ws.apply(None)
    # the same test batch in mixed precision (FP32 factors and solves, FP64
    # refinement): cold start vs the trained network's start blocks, and the
    # eigenvalue difference to the FP64 run
    lam64 = m.local_spaces(cfg.n_loc)
    dth_dev = torch.tensor((base[None] + fields[n_train:n_train + S]).reshape(-1), dtype=torch.float64, device=dev)
    mm = MSGFEM.from_config(cfg, dth_dev, seed=5, tol=1e-6, stream=stream.cuda_stream, instances=S, precision=1)
    learned = ws.predict(ws.features(dth))
    mixed = {}
    lam32 = None
    for kind in ("cold", "learned"):
        ms = []
        for rep in range(2):
            for j in range(mm.N):
                _, nw = ws.size(j)
                mm.set_start_block(j, learned[j] if kind == "learned" else None, 8, nw)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lam32 = mm.local_spaces(cfg.n_loc)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        iters = [mm.info(j)["iterations"] for j in range(mm.N)]
        mixed[kind] = {"iterations_mean": float(np.mean(iters)), "iterations_max": int(np.max(iters)),
                       "solves_per_s": mm.N / (ms[-1] / 1000.0), "ms_per_batch": ms[-1]}
    mm.close()
    m.close()
    top = np.abs(lam64).max(axis=1, keepdims=True)
    mixed["eig_rel_diff_vs_fp64"] = float((np.abs(lam32 - lam64) / top).max())
    mixed["speedup_learned_mixed_vs_cold_fp64"] = mixed["learned"]["solves_per_s"] / res["cold"]["solves_per_s"]
    out = {"workload": f"c1 beam 24x4x12 + seeded 3-D wrinkle field (sd 3 deg, l = 10 mm), 2x1 subdomains, "
                       f"n_loc=8, FP64, tol 1e-6; {S} beams batched per local stage",
           "train_samples": n_train, "test_samples": n_test, "data_gen_s": t_data, "train_ms": train_ms,
           "final_losses": losses}
    out.update(res)
    out["mixed"] = mixed
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="c2")
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--ref-sample", type=int, default=16, help="oracle subdomains of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison run")
    ap.add_argument("--no-warm", action="store_true",
                    help="skip the warm-start runs (learned start on c5, nominal-basis reuse on the mixed leg)")
    ap.add_argument("--no-c4", action="store_true", help="skip the batched C-section (c4) run")
    ap.add_argument("--no-aspect", action="store_true", help="skip the element aspect-ratio sweep")
    ap.add_argument("--c4-steps", type=int, default=1, help="timed steps of the c4 run")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default factor schedule and solve launches")
    ap.add_argument("--direct-launch", action="store_true",
                    help="launch the factorisation and solve kernels one by one instead of replaying graphs "
                         "(the same work; for kernel profilers)")
    ap.add_argument("--streams", type=int, default=0, help="stream groups of the library (0 = its default)")
    ap.add_argument("--factor-kernel", type=int, default=-1, choices=(-1, 0, 1),
                    help="FP32 factorisation tile kernel of the mixed legs: 0 FMA, 1 tensor cores; "
                         "-1 = start from 0 and let the autotuner choose")
    ap.add_argument("--solve-kernel", type=int, default=0, choices=(0, 1, 2, 3, 4),
                    help="8-column block-solve kernel of the mixed legs (msgfem_options.solve_kernel); "
                         "0 = the library default, then the autotuner's choice")
    ap.add_argument("--factor-persistent", type=int, default=0, choices=(0, 1),
                    help="mixed legs: the FP32 factorisation as one persistent launch (1) instead of the "
                         "captured step schedule (0); the autotuner may change it")
    ap.add_argument("--tile-chol", type=int, default=0, choices=(0, 1),
                    help="mixed legs: tile Cholesky of the FP32 factorisation in FP64 (0, the library default) "
                         "or FP32 (1)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
