#!/usr/bin/env python
"""Benchmark: Davidson sigma-vectors/s of the MLCC excitation solve on one GB300 per rank.

One step is one pass of the whole hot path over one synthetic system: system set-up with
the recovery of h (Eq. eff_fock), the DIIS / quasi-Newton ground state (T1-dressing,
X1-basis Fock matrix, CC2 doubles, MLCCSD doubles residual, singles residual, energy),
the Jacobian intermediates, and the Davidson solve for the lowest roots with sigma = A c
(and, on the mixed path, the binary64 refinement). value = sigma-vectors evaluated in the
Davidson solves of all ranks / max over ranks of the timed wall time (CUDA events).

Workload (default): the three-level system, 560 orbitals (60 occupied, 500 virtual), 2500
Cholesky vectors, CCSD-active 20 occupied / 140 virtual inside CC2-active 40 / 300, CCS the
rest, 4 roots: the largest of the paper-shaped workloads that one GPU holds (the 1350-orbital
MLCC2 workload needs more device memory than a GB300 has, by mlcc_solve_footprint; the line
states both figures). Synthetic seeded inputs (synth/), larger than L2 (L is 6.3 GB).
--workload mid runs the 340-orbital, 1500-vector two-level system (CCSD 10/60, CC2 the rest).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|bf16|bf16x3|bf16x6|fp64e]
                  [--refine fp64|fp64e] [--impl ours|reference]

--workload serving replays the serving mix instead (synth.serving_request_spec: occupied
20-80, virtual 150-600, N_J = 5 (occ + vir), active fraction 0.1-0.3, CCS/CCSD or MLCC2,
4 roots) with exponential arrival gaps at --rate requests/s through the serving loop
(mlcc_server_*, --slots slots), and reports solves/s with p50 / p99 latency, next to the
same requests solved one at a time (mixed path) and a sample of them in plain binary64:

  python bench.py --workload serving [--requests R] [--slots S] [--rate 20] [--fp64-sample K]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Davidson sigma-vectors/s"
UNIT = "sigma-vectors/s"
WORKLOAD = "three_level"
# FP64 DFMA peak of the GB300 SM: 152 SMs x 2 FP64 FMA/clock x 2 flop x 2.070 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM bytes per algorithmic flop of the emulated binary64 GEMM (k_tc_gemm_emu + k_emu_reduce),
# measured by ncu on a 1500 x 6000 x 6000 product: (5.000 + 2.041 + 2.016 + 0.071) GB / 1.08e11
EMU_DRAM_BYTES_PER_FLOP = (4.999596e9 + 2.041011e9 + 2.016203e9 + 0.071012e9) / (2.0 * 1500 * 6000 * 6000)


def emu_traffic(flop_per_launch, avg_launch_ms):
    """(DRAM bytes per launch, GB/s) of the emulated binary64 GEMM family."""
    b = EMU_DRAM_BYTES_PER_FLOP * flop_per_launch
    return b, b / (avg_launch_ms / 1e3) / 1e9


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return dict(FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        for line in open(self.file.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op):
    """All-reduce of one float over the ranks (CUDA tensor under NCCL, host tensor under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allreduce_max(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX) if world > 1 else x


def allreduce_sum(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM) if world > 1 else x


def aggregate(n_sigma_local, seconds_local, world):
    """Whole-job throughput: sigma-vectors of all ranks / the slowest rank's time."""
    t_max = allreduce_max(seconds_local, world)
    total = allreduce_sum(float(n_sigma_local), world)
    return total / t_max, t_max, total


def rank_spec(rank):
    """The workload of one replica: the same shapes, the seed offset by the rank."""
    from dataclasses import replace
    from synth import CONFIGS
    return replace(CONFIGS[WORKLOAD], seed=CONFIGS[WORKLOAD].seed + rank)


def cpu_sample_oracle(system, n_chol=None):
    """The oracle, as it stands, on the host cores: one Jacobian transformation of the same
    system by its explicit real-arithmetic MLCC2 formula (Appendix A; the CCSD-block terms
    are not in it), at seeded random amplitudes, with the first n_chol Cholesky vectors
    (all by default). Returns (sigma-vectors/s, cores, description, seconds)."""
    import numpy as np
    from oracle.mlcc import MLCCSystem, sigma_mlcc2_paper
    cores = len(os.sched_getaffinity(0))
    nj = system.L.shape[0] if n_chol is None else int(n_chol)
    o = MLCCSystem(system.L[:nj], system.fock, system.spec.n_occ, system.level)
    rng = np.random.default_rng(0)
    t1 = 0.01 * rng.standard_normal((o.nv, o.no))
    x2 = 0.01 * rng.standard_normal(o.doubles_shape())
    x2 = x2 + x2.transpose(2, 3, 0, 1)
    c1 = rng.standard_normal((o.nv, o.no))
    c2 = rng.standard_normal(o.doubles_shape())
    c2 = c2 + c2.transpose(2, 3, 0, 1)
    t0 = time.perf_counter()
    sigma_mlcc2_paper(o, t1, x2, c1, c2)
    dt = time.perf_counter() - t0
    desc = (f"one sigma-vector of the same {system.spec.n_mo}-orbital system ({nj} of its {system.L.shape[0]} "
            "Cholesky vectors) by the oracle's explicit MLCC2 Jacobian formula (Appendix A; CCSD-block terms not "
            "included), FP64 numpy")
    return 1.0 / dt, cores, desc, dt


def set_blas_threads():
    n = str(len(os.sched_getaffinity(0)))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, n)


def run_reference(args):
    """--impl reference: the oracle's Jacobian transformation on the host cores, on this
    workload. A whole sigma takes tens of seconds here, so each step times one sigma of the
    same system with its first quarter of the Cholesky vectors, and the time is scaled to a
    whole sigma by the ratio of one whole sigma to one such sigma, both measured in the
    warm-up (the sigma cost is not proportional to the vector count, hence the measured
    ratio). Rank 0 alone runs it."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    set_blas_threads()
    from synth import CONFIGS, make_system
    system = make_system(CONFIGS[WORKLOAD])
    nj = system.L.shape[0]
    sub = max(1, nj // 4)
    _, cores, desc_full, t_full = cpu_sample_oracle(system)
    _, _, _, t_sub = cpu_sample_oracle(system, sub)
    ratio = t_full / t_sub
    for _ in range(max(0, args.warmup - 1)):
        cpu_sample_oracle(system, sub)
    times = []
    for _ in range(args.steps):
        _, cores, _, dt = cpu_sample_oracle(system, sub)
        times.append(dt * ratio)
    value = args.steps / sum(times)
    sample = (f"per step one sigma-vector of the same {system.spec.n_mo}-orbital system with its first {sub} of {nj} "
              f"Cholesky vectors by the oracle's explicit MLCC2 Jacobian formula (Appendix A; CCSD-block terms not "
              f"included), FP64 numpy, its time scaled by {ratio:.3f} = (one whole sigma, {t_full:.2f} s) / "
              f"(one such sigma, {t_sub:.2f} s), both measured in the warm-up")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, "fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_label(s):
    """What the workload is, with its sizes and levels."""
    cc2_all = s.s_occ == s.n_occ and s.s_vir == s.n_vir
    if s.t_occ and s.t_vir and not cc2_all:
        kind = (f"three-level MLCCSD: CCSD-active {s.t_occ}/{s.t_vir} inside CC2-active {s.s_occ}/{s.s_vir}, "
                f"CCS the rest")
    elif s.t_occ and s.t_vir:
        kind = f"MLCCSD, two levels: CCSD-active {s.t_occ}/{s.t_vir}, CC2 the rest"
    elif cc2_all:
        kind = "CC2 (every orbital CC2-active)"
    else:
        kind = f"MLCC2: CC2-active {s.s_occ}/{s.s_vir}, CCS the rest"
    return (f"{kind}; {s.n_mo} orbitals ({s.n_occ} occ / {s.n_vir} vir), {s.n_chol} Cholesky vectors, "
            f"{s.n_roots} roots")


def larger_workload_excluded(opts_mixed):
    """The larger paper-shaped workload and why it is not the bench's: its device footprint."""
    from paper_2006_05226_gb300 import mlcc
    from synth import CONFIGS
    from synth.generator import level_map
    s = CONFIGS["mlcc2_large"]
    lev = level_map(s.n_occ, s.n_vir, s.s_occ, s.s_vir, s.t_occ, s.t_vir)
    fp = mlcc.solve_footprint(s.n_mo, s.n_occ, s.n_chol, lev, opts_mixed)
    try:
        import torch
        total = int(torch.cuda.get_device_properties(0).total_memory)
    except Exception:
        total = None
    return {"workload": workload_label(s), "footprint_bytes": fp, "device_bytes": total,
            "fits": bool(total is not None and fp <= total)}


def config_dict(args, prec):
    from synth import CONFIGS
    s = CONFIGS[WORKLOAD]
    return {"workload": workload_label(s),
            "n_mo": s.n_mo, "n_occ": s.n_occ, "n_chol": s.n_chol, "ccsd_active": [s.t_occ, s.t_vir],
            "cc2_active": [s.s_occ, s.s_vir], "n_roots": s.n_roots, "precision": prec,
            "l2": f"inputs larger than L2 (L^J_pq is {s.n_chol * s.n_mo ** 2 * 8 / 1e9:.2f} GB)",
            "parallelism": f"replicas{args.gpus}",
            "excited_state_solver": getattr(args, "solver", "davidson")}


def _make_system(spec):
    from synth import make_system
    return make_system(spec)


def run_serving(args):
    """The serving mix through mlcc_server_*: arrivals replayed in real time."""
    rank, world, local = dist_env()
    import multiprocessing as mp
    import numpy as np
    from synth import serving_arrivals, serving_request_spec
    specs = [serving_request_spec(r)[0] for r in range(args.requests)]
    # inputs drawn on the host cores before the first CUDA call (spawned workers)
    t_start = time.perf_counter()

    def progress(what):
        print(f"[serving] {time.perf_counter() - t_start:8.1f} s  {what}", file=sys.stderr, flush=True)

    # each worker's BLAS gets its share of the cores (oversubscribed BLAS threads spin)
    cores = len(os.sched_getaffinity(0))
    workers = max(1, min(len(specs), cores // 4))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = str(max(1, cores // workers))
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            systems = pool.map(_make_system, specs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    progress(f"{len(systems)} synthetic systems drawn")
    arrivals = serving_arrivals(len(specs), rate=args.rate)
    import torch
    torch.cuda.set_device(local)
    from paper_2006_05226_gb300 import mlcc
    precs = {"fp64": mlcc.MLCC_FP64, "bf16": mlcc.MLCC_BF16, "bf16x3": mlcc.MLCC_BF16X3,
             "bf16x6": mlcc.MLCC_BF16X6, "fp64e": mlcc.MLCC_FP64E}
    prec, refine = precs[args.precision], precs[args.refine]
    split = prec in (mlcc.MLCC_BF16, mlcc.MLCC_BF16X3, mlcc.MLCC_BF16X6)

    def opts_for(spec, p, graph=1):
        sp = p in (mlcc.MLCC_BF16, mlcc.MLCC_BF16X3, mlcc.MLCC_BF16X6)
        return mlcc.default_options(n_roots=spec.n_roots, precision=p, gs_precision=p, refine_fp64=1,
                                    lowp_res_tol=1e-5, refine_precision=refine,
                                    gs_tol=1e-9 if sp else 1e-11, gs_energy_tol=1e-10 if sp else 1e-12,
                                    sigma_graph=graph if args.sigma_graph else 0)

    # pinned host copies: the server borrows them until each result is polled
    host = []
    for sy in systems:
        Lp = torch.empty(sy.L.shape, dtype=torch.float64, pin_memory=True)
        Fp = torch.empty(sy.fock.shape, dtype=torch.float64, pin_memory=True)
        Lp.numpy()[...] = sy.L
        Fp.numpy()[...] = sy.fock
        host.append((Lp, Fp))
    # one at a time, same options (warms the kernels up as well)
    ctx = mlcc.Context(local)
    seq_w = []
    t0 = time.perf_counter()
    for sy, (Lp, Fp) in zip(systems, host):
        t1 = time.perf_counter()
        w = mlcc.solve(ctx, Lp.numpy(), Fp.numpy(), sy.spec.n_occ, sy.level, opts_for(sy.spec, prec)).omega
        seq_w.append(w)
        progress(f"{sy.spec.name} ({sy.spec.n_occ} occ / {sy.spec.n_vir} vir, {sy.spec.n_chol} vectors): "
                 f"{time.perf_counter() - t1:.1f} s")
    seq_s = time.perf_counter() - t0
    progress(f"one at a time: {seq_s:.1f} s")
    # the same, with the Jacobian transformations evaluated eagerly (no CUDA graphs)
    seq_nog_s = None
    if args.sigma_graph:
        t0 = time.perf_counter()
        for sy, (Lp, Fp) in zip(systems, host):
            mlcc.solve(ctx, Lp.numpy(), Fp.numpy(), sy.spec.n_occ, sy.level, opts_for(sy.spec, prec, graph=0))
        seq_nog_s = time.perf_counter() - t0
        progress(f"one at a time without sigma graphs: {seq_nog_s:.1f} s")
    # plain binary64, one at a time, on the first fp64_sample requests (accuracy and speed)
    fp64_s, errs = [], []
    for k in range(min(args.fp64_sample, len(systems))):
        sy, (Lp, Fp) = systems[k], host[k]
        t1 = time.perf_counter()
        w64 = mlcc.solve(ctx, Lp.numpy(), Fp.numpy(), sy.spec.n_occ, sy.level,
                         opts_for(sy.spec, mlcc.MLCC_FP64, graph=0)).omega
        fp64_s.append(time.perf_counter() - t1)
        progress(f"binary64 solve of request {k}: {fp64_s[-1]:.1f} s")
        errs.append(float(np.max(np.abs(np.asarray(seq_w[k]) - w64))))
    ctx.close()
    # the mix: submissions at the arrival times, results polled as they finish
    srv = mlcc.Server(local, n_slots=args.slots)
    tickets = [None] * len(specs)
    launches0 = mlcc.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    start = time.perf_counter()

    def submit_all():
        for k, (sy, (Lp, Fp)) in enumerate(zip(systems, host)):
            delay = arrivals[k] - (time.perf_counter() - start)
            if delay > 0:
                time.sleep(delay)
            tickets[k] = srv.submit(Lp.numpy(), Fp.numpy(), sy.spec.n_occ, sy.level, opts_for(sy.spec, prec))

    th = threading.Thread(target=submit_all)
    th.start()
    th.join()
    results = [srv.poll(t) for t in tickets]
    wall = time.perf_counter() - start
    clk = clocks.stop()
    launches = mlcc.launch_count() - launches0
    info = srv.stats()
    srv.close()
    lat = np.array([r.t_finish - r.t_submit for r, _ in results])
    status = [int(r.status) for r, _ in results]
    mix_vs_alone = max(float(np.max(np.abs(w - seq_w[k]))) for k, (_, w) in enumerate(results))
    if rank != 0:
        return 0
    n = len(specs)
    line = {"metric": "solves/s (serving mix)", "value": n / wall, "unit": "solves/s", "n_gpus": world,
            "steps": 1, "warmup": 0, "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision if not split else f"{args.precision}+{args.refine}",
            "data": "synthetic",
            "config": {"workload": f"serving mix: {n} requests (occ 20-80, vir 150-600, N_J = 5 (occ+vir), "
                                   f"active fraction 0.1-0.3, CCS/CCSD or MLCC2, 4 roots), Poisson arrivals "
                                   f"at {args.rate} req/s", "requests": n, "slots": args.slots,
                       "rate_per_s": args.rate, "budget_bytes": int(info.budget_bytes),
                       "sigma_graph": bool(args.sigma_graph),
                       "parallelism": f"replicas{world}"},
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "status": status, "peak_running": int(info.peak_running), "peak_admitted_bytes": int(info.peak_bytes),
            "one_at_a_time_mixed_solves_per_s": n / seq_s,
            "one_at_a_time_mixed_solves_per_s_without_sigma_graphs": (n / seq_nog_s) if seq_nog_s else None,
            "fp64_one_at_a_time": {"requests": len(fp64_s), "mean_seconds": float(np.mean(fp64_s)) if fp64_s else None,
                                   "solves_per_s": len(fp64_s) / sum(fp64_s) if fp64_s else None,
                                   "max_abs_omega_err_Ha": max(errs) if errs else None},
            "max_abs_omega_diff_mix_vs_alone_Ha": mix_vs_alone,
            "clocks": clk, "gpu_launches": int(launches),
            "sizes": [[s.n_occ, s.n_vir, s.n_chol, s.s_occ, s.s_vir, s.t_occ, s.t_vir] for s in specs]}
    print(json.dumps(line), flush=True)
    return 0


def run_probe(args):
    """--probe: the Jacobian transformation of one synthetic system, for kernel profiling.

    The system has the Cholesky-rank GEMM shapes of the benchmark workload scaled down so
    that the device holds a few GB (--occ, --vir, --chol, --ccsd-occ, --ccsd-vir). The
    Jacobian is prepared at seeded small amplitudes (no ground-state solve) and --nsigma
    sigma-vectors in --precision run inside a cudaProfilerStart/Stop range (capture with
    ncu --profile-from-start off). Prints one line; no JSON, not a bench value."""
    import numpy as np
    import torch
    from paper_2006_05226_gb300 import mlcc
    from synth.generator import SystemSpec, default_scale, make_system
    precs = {"fp64": mlcc.MLCC_FP64, "bf16": mlcc.MLCC_BF16, "bf16x3": mlcc.MLCC_BF16X3,
             "bf16x6": mlcc.MLCC_BF16X6, "fp64e": mlcc.MLCC_FP64E}
    prec = precs[args.precision]
    tau = args.chol / 5.0
    spec = SystemSpec("probe", args.occ, args.vir, args.chol, tau, args.occ, args.vir, args.ccsd_occ,
                      args.ccsd_vir, 4, 0, default_scale(tau))
    s = make_system(spec, rhf_tol=1e-8)
    ctx = mlcc.Context(0)
    g = mlcc.System(ctx, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"),
                    args.occ, s.level)
    d = g.dims
    rng = np.random.default_rng(0)
    t1 = torch.as_tensor(0.01 * rng.standard_normal(d.n_singles), device="cuda")
    m = d.s_vir * d.s_occ
    x2 = 0.01 * rng.standard_normal((m, m))
    x2 = torch.as_tensor((x2 + x2.T).ravel(), device="cuda")
    g.jacobian_prepare(t1, x2)
    c = rng.standard_normal(d.vector_len)
    c2 = c[d.n_singles:].reshape(m, m)
    c[d.n_singles:] = (c2 + c2.T).ravel()
    c = torch.as_tensor(c, device="cuda").reshape(1, -1)
    g.sigma(c, precision=prec)      # warm: operand caches, kernel attributes
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    for _ in range(args.nsigma):
        g.sigma(c, precision=prec)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    g.close()
    ctx.close()
    print(f"probe ok: vector_len {d.vector_len}, precision {args.precision}, {args.nsigma} sigma")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="three_level", choices=["mid", "three_level", "es_parity", "serving"],
                    help="three_level (default): 560 orbitals, CCSD 20/140 inside CC2 40/300, CCS rest; "
                         "mid: 340 orbitals, CCSD 10/60, CC2 the rest; es_parity: 170 orbitals, CCSD 6/36 "
                         "inside CC2 16/110, CCS rest (a small case for kernel captures); serving: the request mix")
    ap.add_argument("--requests", type=int, default=8, help="serving: number of requests")
    ap.add_argument("--slots", type=int, default=4, help="serving: concurrent slots")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: arrivals per second")
    ap.add_argument("--fp64-sample", type=int, default=1, help="serving: requests also solved in binary64")
    ap.add_argument("--sigma-graph", type=int, default=1,
                    help="serving: replay each request's Jacobian transformation from a CUDA graph (1) or not (0)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "bf16", "bf16x3", "bf16x6", "fp64e"])
    ap.add_argument("--refine", default="fp64e", choices=["fp64", "fp64e"],
                    help="precision of the ground-state polish and the Davidson refinement sweep")
    ap.add_argument("--no-fp64-check", action="store_true",
                    help="skip the plain binary64 reference solve used to report the error")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--solver", default="davidson", choices=["davidson", "folded"],
                    help="excited states: Davidson on the full Jacobian, or the folded CC2 Jacobian "
                         "(sigma in the --refine precision)")
    ap.add_argument("--probe", action="store_true",
                    help="profiling probe: sigma-vectors of one scaled-down system (see run_probe)")
    ap.add_argument("--occ", type=int, default=40, help="probe: occupied orbitals")
    ap.add_argument("--vir", type=int, default=150, help="probe: virtual orbitals")
    ap.add_argument("--chol", type=int, default=1500, help="probe: Cholesky vectors")
    ap.add_argument("--ccsd-occ", type=int, default=10, help="probe: CCSD-active occupied")
    ap.add_argument("--ccsd-vir", type=int, default=60, help="probe: CCSD-active virtual")
    ap.add_argument("--nsigma", type=int, default=1, help="probe: sigma-vectors in the profiled range")
    args = ap.parse_args()
    if args.probe:
        return run_probe(args)
    global WORKLOAD
    if args.workload != "serving":
        WORKLOAD = args.workload
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)

    rank, world, local = dist_env()
    import numpy as np
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2006_05226_gb300 import mlcc
    from synth import CONFIGS, make_system
    from dataclasses import replace

    spec = rank_spec(rank)
    system = make_system(spec)
    precs = {"fp64": mlcc.MLCC_FP64, "bf16": mlcc.MLCC_BF16, "bf16x3": mlcc.MLCC_BF16X3,
             "bf16x6": mlcc.MLCC_BF16X6, "fp64e": mlcc.MLCC_FP64E}
    prec, refine = precs[args.precision], precs[args.refine]
    split = prec in (mlcc.MLCC_BF16, mlcc.MLCC_BF16X3, mlcc.MLCC_BF16X6)
    # mixed path: split-bf16 ground state polished in binary64 (refine precision) to 1e-9,
    # split-bf16 Davidson to a 1e-5 residual, then one refinement Rayleigh-Ritz sweep
    opts = mlcc.default_options(n_roots=spec.n_roots, precision=prec, gs_precision=prec,
                                refine_fp64=1, lowp_res_tol=1e-5, refine_precision=refine,
                                gs_tol=1e-9 if split else 1e-11,
                                gs_energy_tol=1e-10 if split else 1e-12)
    ctx = mlcc.Context(local)
    L_dev = torch.as_tensor(system.L, device=f"cuda:{local}")
    F_dev = torch.as_tensor(system.fock, device=f"cuda:{local}")

    fold_opts = mlcc.default_options(n_roots=spec.n_roots, precision=refine, es_res_tol=1e-8)

    def step():
        g = mlcc.System(ctx, L_dev, F_dev, spec.n_occ, system.level)
        t1, x2, gi = g.ground_state(opts)
        if args.solver == "folded":
            w, _, ei = g.excited_states_folded(fold_opts, want_vectors=False)
        else:
            w, _, ei = g.excited_states(opts, want_vectors=False)
        g.close()
        return ei.n_sigma, ei.n_sigma_lowp, w, gi

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    profile_range = os.environ.get("MLCC_PROFILE_TIMED", "0") not in ("", "0")
    clocks = ClockSampler(local)
    if not profile_range:   # nvidia-smi polling next to an ncu capture made ncu fail
        clocks.start()
    ctx.kernel_timing(True)
    launches0 = mlcc.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if profile_range:   # ncu --profile-from-start off captures exactly the timed steps
        torch.cuda.cudart().cudaProfilerStart()
    ev0.record(ctx.stream)
    n_sigma = n_lowp = 0
    omegas, gs = None, None
    step_ev = [ev0]
    for k in range(args.steps):
        ns, nl, omegas, gs = step()
        n_sigma += ns
        n_lowp += nl
        if k + 1 < args.steps:   # per-solve latency: events between consecutive steps
            e = torch.cuda.Event(enable_timing=True)
            e.record(ctx.stream)
            step_ev.append(e)
    ev1.record(ctx.stream)
    step_ev.append(ev1)
    torch.cuda.synchronize()
    if profile_range:
        torch.cuda.cudart().cudaProfilerStop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    step_s = [a.elapsed_time(b) / 1e3 for a, b in zip(step_ev[:-1], step_ev[1:])]
    launches = mlcc.launch_count() - launches0
    fams = {f: ctx.kernel_time(f) for f in ("rank_gemm_tc", "rank_gemm_f64e", "rank_gemm_f64",
                                            "ladder_tc", "ladder_f64e", "ladder_f64")}
    phases = {f: ctx.kernel_time(f) for f in ("gs_omega", "jacobian_prepare", "sigma", "sigma_singles",
                                              "sigma_doubles_to_singles", "sigma_cc2_doubles",
                                              "sigma_ccsd_rows", "dav_update_G", "dav_ritz",
                                              "dav_orthonormalise")}
    breakdown = {f: {"calls": n, "total_ms": ms} for f, (n, ms, _) in phases.items() if n}
    ctx.kernel_timing(False)
    clk = clocks.stop()
    barrier(world)
    value, t_max, total_sigma = aggregate(n_sigma, elapsed, world)

    # error against the plain binary64 GPU path (outside the timed region)
    # (also the plain binary64 solve's own time: the baseline the mixed path must beat in
    # solves/s at the stated accuracy)
    err_fp64 = None
    fp64_solve = None
    if prec != mlcc.MLCC_FP64 and not args.no_fp64_check:
        ref_opts = mlcc.default_options(n_roots=spec.n_roots)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        g = mlcc.System(ctx, L_dev, F_dev, spec.n_occ, system.level)
        g.ground_state(ref_opts)
        w_ref, _, ei_ref = g.excited_states(ref_opts, want_vectors=False)
        g.close()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ref_s = e0.elapsed_time(e1) / 1e3
        err_fp64 = float(np.max(np.abs(np.asarray(omegas) - w_ref)))
        fp64_solve = {"seconds": ref_s, "solves_per_s": 1.0 / ref_s, "sigma_vectors": int(ei_ref.n_sigma),
                      "sigma_per_s": ei_ref.n_sigma / ref_s,
                      "mixed_over_fp64_solves_per_s": (args.steps / t_max) * ref_s}

    # end to end through the public host-memory entry point (H2D of L and F inside)
    e2e = None
    if not args.no_e2e:
        # the inputs of the step staged in pinned host memory (outside the timed region)
        host_mem = "pinned"
        try:
            Lp = torch.empty(system.L.shape, dtype=torch.float64, pin_memory=True)
            Fp = torch.empty(system.fock.shape, dtype=torch.float64, pin_memory=True)
            Lh, Fh = Lp.numpy(), Fp.numpy()
            Lh[...] = system.L
            Fh[...] = system.fock
        except Exception:
            Lh = np.ascontiguousarray(system.L)
            Fh = np.ascontiguousarray(system.fock)
            host_mem = "pageable"
        barrier(world)
        t0 = time.perf_counter()
        sol = mlcc.solve(ctx, Lh, Fh, spec.n_occ, system.level, opts, t1=True)
        ei, w2, t1h = sol.es, sol.omega, sol.t1
        dt = time.perf_counter() - t0
        dt = allreduce_max(dt, world)
        e_val = allreduce_sum(float(ei.n_sigma), world) / dt
        e2e = {"value": e_val, "unit": UNIT, "h2d_bytes_per_step": int(Lh.nbytes + Fh.nbytes),
               "d2h_bytes_per_step": int(8 * (len(w2) + t1h.size)), "host_memory": host_mem}

    if rank != 0:
        return 0
    pk, src = peaks()
    bf16_peak = pk.get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"])
    pieces = {mlcc.MLCC_BF16: 1, mlcc.MLCC_BF16X3: 3, mlcc.MLCC_BF16X6: 6}
    # tensor-core products per algorithmic flop: split-bf16 pieces, or the 36 digit
    # products of the binary64 emulation
    ops = {"rank_gemm_tc": pieces.get(prec, 3), "rank_gemm_f64e": 36, "rank_gemm_f64": None,
           "ladder_tc": pieces.get(prec, 3), "ladder_f64e": 36, "ladder_f64": None}
    kernels = {"rank_gemm_tc": "k_tc_gemm: Cholesky-rank doubles GEMMs, split bf16 (tcgen05, fp32 accumulate)",
               "rank_gemm_f64e": "k_tc_gemm (emulation mode) + k_emu_reduce: Cholesky-rank GEMMs "
                                 "in binary64 from exact bf16 integer digits",
               "rank_gemm_f64": "k_dgemm: Cholesky-rank GEMMs on the binary64 FMA units",
               "ladder_tc": "k_tc_gemm: the CCSD-row ladder sum_cd g~_acbd c_cidj, [(ab)][(cd)] x [(cd)][(ij)], "
                            "split bf16 (tcgen05, fp32 accumulate)",
               "ladder_f64e": "k_tc_gemm (emulation mode) + k_emu_reduce: the CCSD-row ladder in binary64",
               "ladder_f64": "k_dgemm: the CCSD-row ladder on the binary64 FMA units"}
    families = {}
    for f, (n, ms, fl) in fams.items():
        if n == 0:
            continue
        ach = fl / (ms / 1e3) / 1e12 if ms > 0 else None
        families[f] = {"launches": n, "total_ms": ms, "avg_launch_ms": ms / n, "flop_per_launch": fl / n,
                       "algorithmic_tflops": ach}
    dom = max(families, key=lambda f: families[f]["total_ms"]) if families else None
    roof = None
    if dom is not None:
        d = families[dom]
        if ops[dom] is None:
            roof = {"bound": "alu", "achieved": d["algorithmic_tflops"], "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": d["algorithmic_tflops"] / FP64_PEAK_TFLOPS,
                    "peak_source": "FP64 DFMA rate from unit counts and clock (152 SMs x 2 FMA/clk x 2.07 GHz)"}
        else:
            peak = bf16_peak / ops[dom]
            roof = {"bound": "tensor", "achieved": d["algorithmic_tflops"], "peak": peak, "unit": "TFLOP/s",
                    "frac": d["algorithmic_tflops"] / peak,
                    "tensor_ops_per_algorithmic_flop": ops[dom],
                    "tensor_issue_tflops": d["algorithmic_tflops"] * ops[dom],
                    "peak_source": f"bf16 dense sustained ({bf16_peak} TFLOP/s, of {src}) / "
                                   f"{ops[dom]} bf16 products per algorithmic product"}
        # DRAM bytes per launch, from one ncu capture of the same kernels on a smaller product
        # (the emulated GEMM and its chunk reduction on the 1500 x 6000 x 6000 product of the
        # dS = 6000 probe: dram__bytes_read.sum + dram__bytes_write.sum = 9.13 GB for
        # 1.08e11 flop). The chunk planes and the operand re-reads grow with M N K like the
        # flops, so the capture scales to a launch by its flops. Other families: not
        # captured on their present kernels (null).
        traffic = emu_traffic(d["flop_per_launch"], d["avg_launch_ms"]) if dom == "rank_gemm_f64e" else None
        if traffic:
            roof.update({"traffic_unit": "bytes per launch", "traffic_gbs": traffic[1],
                         "traffic_source": "ncu capture of the emulated GEMM + reduction on a 1500x6000x6000 "
                                           "product, scaled to the launch by algorithmic flops"})
        roof.update({"traffic": traffic[0] if traffic else None, "kernel": kernels[dom], "family": dom,
                     "achieved_is": "algorithmic 2MNK flops of the contraction per launch / launch time "
                                    "(CUDA events on the library stream)",
                     "launches": d["launches"], "avg_launch_ms": d["avg_launch_ms"],
                     "flop_per_launch": d["flop_per_launch"], "families": families})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision if not split else f"{args.precision}+{args.refine}",
            "data": "synthetic", "config": config_dict(args, args.precision if not split else f"{args.precision}+{args.refine}"),
            "solves_per_s": args.steps * world / t_max,
            "latency_p50_s": float(np.percentile(step_s, 50)), "latency_p99_s": float(np.percentile(step_s, 99)),
            "latency_of": "one whole solve (one step) on rank 0, CUDA events between steps",
            "sigma_per_step": n_sigma / args.steps,
            "sigma_lowp_per_step": n_lowp / args.steps,
            "omega": [float(x) for x in omegas], "e_corr": gs.e_corr,
            "max_abs_omega_err_vs_fp64_gpu_Ha": err_fp64, "fp64_gpu_solve": fp64_solve,
            "roofline": roof, "clocks": clk, "gpu_launches": int(launches), "e2e": e2e,
            "breakdown": breakdown,
            "precision_notes": "split-bf16 phases (ground state, Davidson sigma) then a binary64-class refinement "
                               f"({args.refine}); in the split phase the Davidson vector arithmetic (dot products, "
                               "Gram-Schmidt, Ritz vectors) runs in binary32 and the small subspace eigenproblem "
                               "on the host in binary64; omega and e_corr are those of the refined solve"}
    if WORKLOAD == "three_level":
        line["config"]["larger_workload_excluded"] = larger_workload_excluded(opts)
    if world == 1 and not args.no_cpu_baseline:
        set_blas_threads()
        v, cores, desc, dt = cpu_sample_oracle(system)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc, "seconds": dt}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
