"""Benchmark of the coupled velocity solve: particle-steps per second.

One step = one full time step of the path (cell list and pair search, fused
pair/assembly kernel, Jacobi-PCG to the stated relative residual, Lees-Edwards
position update) on N = 262,144 particles at number density 3 (cubic box,
r_c = 1), alpha = 4, eps = 1, zeta = kT = 1, kappa*tau = 0.5, dt = 0.01,
positions uniform from the seed.  Inputs are synthetic and seeded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed] [--impl reference]

N > 1 (torchrun): each rank advances its own replica (different seed): the path
does not shard, so the ranks are independent replicas (weak scaling, no
collective on the data path); value = all ranks' particle-steps / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "particle-steps/s at 1e-8 CG rel. residual; CG SpMV HBM GB/s vs GB300 peak"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank advances its own replica of the workload (independent positions and noise)."""
    return base_seed + 1000 * rank


def max_over_ranks(local_ms: float, dist=None, device="cpu") -> float:
    """The slowest rank's time: the whole job ends when the last replica does."""
    if dist is None:
        return local_ms
    import torch
    t = torch.tensor([local_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n: int, world: int, steps: int, t_max_ms: float) -> float:
    """Particle-steps/s of all ranks together (weak scaling: N particles per rank)."""
    return n * world * steps / (t_max_ms / 1e3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region.

    start() returns once the first sample has arrived (so sampling is running
    when the timed region begins); stop() keeps the samples that arrived while
    the region ran (at least the first one after it began)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []   # (arrival time, text)
        self.t_start = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", str(self.INTERVAL_MS)]
        if self.gpu_id:
            cmd[1:1] = ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.005)
        self.t_start = time.perf_counter()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t_end = time.perf_counter()
        time.sleep(2.5 * self.INTERVAL_MS / 1e3)   # the sample taken just after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        inside = [ln for t, ln in self.lines if self.t_start <= t <= t_end + 1.5 * self.INTERVAL_MS / 1e3]
        if not inside:
            inside = [ln for t, ln in self.lines if t >= self.t_start][:1]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in inside:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[4:8]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "interval_ms": self.INTERVAL_MS, "reasons": sorted(reasons)}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# persistent solve from one ncu capture of the current kernel on this command's
# workload, keyed by workload, tile configuration (gathers in flight, blocks per
# SM, pipelined, threads per block, on-chip) and burn-in steps (the regime the
# captured launch came from); any other kernel, workload or regime reports null.
PROFILED_TRAFFIC = {("mixed-n262144", 4, 1, False, 512, True, 1000): 172.4e6}
# the same for the large workload (N = 4,194,304), by solver kernel (one capture of the
# DRAM counters alone, one pass, the launch of the first timed step)
LARGE_PROFILED_TRAFFIC = {"k32_cg_persistent<6,1,0,1024>": 53.90e9, "k32_cg_persistent<4,3,0,256,1>": 49.99e9}


def profiled_traffic(workload_name: str, tune, burn_in: int = 0) -> float | None:
    """The capture's DRAM bytes, where it matches this launch's kernel, workload and regime."""
    if not tune:
        return None
    return PROFILED_TRAFFIC.get((workload_name, tune["gathers_in_flight"], tune["blocks_per_sm"],
                                 tune["pipelined"], tune["block_threads"], tune.get("resident", False), burn_in))


def solver_kernel_name(tune) -> str:
    """Name of the persistent solver kernel a tile configuration launches."""
    if tune and tune.get("resident"):
        bt = tune["block_threads"]
        return f"k32_cg_resident<{bt},{2048 // bt}>"
    if tune:
        mf = ",1" if tune.get("matrix_free") else ""
        return (f"k32_cg_persistent<{tune['gathers_in_flight']},{tune['blocks_per_sm']},{int(tune['pipelined'])},"
                f"{tune['block_threads']}{mf}>")
    return "k32_cg_persistent"


def spmv_algorithmic_bytes(n: int, nnz: int, precision: str) -> float:
    """Bytes the solver's SpMV kernel must move per launch (padding excluded):
    per entry its column and weight; per row the slot map, one read of the
    gathered vector (r with D^-1 in the mixed solver, z in FP64), the diagonal,
    and the read and write of q and p (q' = A z + beta q, p' = z + beta p)."""
    if precision == "mixed":
        return n * (4.0 + 16.0 + 4.0 + 32.0 + 32.0) + 8.0 * nnz
    return n * (4.0 + 24.0 + 8.0 + 48.0 + 48.0) + 12.0 * nnz


def update_algorithmic_bytes(n: int, precision: str) -> float:
    """Update kernel: mixed reads p, q, d, r and writes d, r (float4 rows);
    FP64 reads x, p, r, q, D^-1 and writes x, r, z."""
    if precision == "mixed":
        return n * 6 * 16.0
    return n * (4 * 24.0 + 8.0 + 3 * 24.0)


# Algorithmic bytes per particle per iteration of the mixed solve, as the scope
# table of the measurement plan counts them: the SpMV (13.58 entries x 8 B of
# column and FP32 weight, 4 B row pointer, 16 + 16 B of gathered and written
# vectors: 145 B), the FP32 vector updates (~120 B) and the residual
# replacements' share (~215 B every ~15 iterations): ~280 B.
MIXED_BYTES_PER_PARTICLE_ITERATION = 280.0
L2_BYTES = 126.5e6   # GB300 L2
FP64_BYTES_PER_PARTICLE_ITERATION = 450.0


def plan_algorithmic_bytes(n: int, iters: int, precision: str) -> float:
    per = MIXED_BYTES_PER_PARTICLE_ITERATION if precision == "mixed" else FP64_BYTES_PER_PARTICLE_ITERATION
    return per * n * iters


def persistent_algorithmic_bytes(n: int, nnz: int, iters: int, checks: int, init: bool = False) -> float:
    """Bytes one persistent mixed solve must move: per iteration one SpMV and one
    update; per FP64 residual replacement the fold of d into x (x read and
    written, d read and cleared) and the FP64 SpMV r = b - A x (columns and FP64
    weights, one read of x, b and the diagonals, r written).  init: the launch
    also forms r = b - A x0 in double-float (per entry the column, both weight
    parts and a 32-byte x0 record; per row b and x0 records, A_ii in two parts,
    D^-1, and r written as a float4 and a 32-byte record)."""
    per_check = n * (48.0 + 32.0) + n * (4.0 + 24.0 + 24.0 + 24.0 + 8.0 + 4.0 + 16.0) + 12.0 * nnz
    per_init = n * (32.0 + 32.0 + 8.0 + 4.0 + 16.0 + 32.0) + 44.0 * nnz if init else 0.0
    return iters * (spmv_algorithmic_bytes(n, nnz, "mixed") + update_algorithmic_bytes(n, "mixed")) \
        + checks * per_check + per_init


def run_steps(sim, steps, stream, flush):
    """Time `steps` single steps with CUDA events on the simulation's stream,
    flushing L2 before each; returns (total ms, launches, CG iterations, max residual)."""
    import torch
    total_ms, launches, iters, max_res = 0.0, 0, 0, 0.0
    for _ in range(steps):
        flush.zero_()                      # L2 flush between timed steps (512 MB > L2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = sim.step(1)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        launches += info["kernel_launches"]
        iters += info["cg_iterations"]
        max_res = max(max_res, info["last_residual"])
    return total_ms, launches, iters, max_res


def _oracle_steps(job):
    """One host process: `steps` timed oracle steps (after `warm` untimed ones) of a replica of the
    workload with its own seed; returns the per-step seconds."""
    n, L, kappa_tau, tol, seed, steps, warm = job
    import oracle
    import dataclasses
    w = dataclasses.replace(synth.cubic("sample", n, kappa_tau, steps, tol, seed), L=tuple(L))
    p = oracle.Params.from_workload(w)
    pos = synth.uniform_positions(n, w.L, seed)
    delta, times = 0.0, []
    for s in range(warm + steps):
        t0 = time.perf_counter()
        r = oracle.step(p, pos, delta, s, tol=tol, neighbor_method="cells")
        pos, delta = r.pos, r.delta
        if s >= warm:
            times.append(time.perf_counter() - t0)
    return times


def oracle_throughput(workload, n: int, steps: int, warm: int = 0):
    """The CPU oracle as it stands (single-threaded code) on every host core at once: one process
    per core, each stepping its own replica (own seed) of an n-particle box of the workload's
    density, shear rate and tolerance.  Returns (particle-steps/s of all processes together,
    processes, seconds of the slowest process's timed steps)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    procs = max(1, os.cpu_count() or 1)
    L = (synth.box_length(n),) * 3 if n != workload.n else workload.L
    jobs = [(n, L, workload.kappa_tau, workload.tol, workload.seed + 7919 * k, steps, warm) for k in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:   # spawned: this process has used the GPU
        times = pool.map(_oracle_steps, jobs)
    slowest = max(sum(t) for t in times)
    return n * steps * procs / slowest, procs, slowest


def cpu_baseline(workload, precision: str, steps: int = 2):
    """The CPU oracle as it stands on all host cores (one process per core, each a replica of
    the full workload), a bounded sample of 2 steps each."""
    value, procs, slowest = oracle_throughput(workload, workload.n, steps)
    return {"value": value, "unit": "particle-steps/s", "cores": procs, "kind": "oracle",
            "sample": f"{procs} concurrent single-thread oracle processes, each {steps} full steps of its own "
                      f"N={workload.n} replica (cell-list pair search, Jacobi-PCG to {workload.tol:g}) from "
                      f"the uniform start (fewer pairs and CG iterations per step than the steady state the "
                      f"GPU line is timed in); slowest {slowest:.1f} s"}


REFERENCE_SAMPLE_N = 32768   # particles per process and reference step: one oracle step then takes ~0.5 s


def run_reference(args, workload):
    """The CPU oracle as it stands on the same metric, on every host core: each process steps its
    own replica of a bounded sample of the workload (the same density, shear rate, tolerance and
    seed family in a box of REFERENCE_SAMPLE_N particles: the oracle's full step of cell-list
    search, assembly, Jacobi-PCG to the workload's tolerance and sheared update), so that any
    --steps K --warmup W run ends within minutes; value = all processes' particle-steps / the
    slowest process's timed seconds."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    ns = min(workload.n, REFERENCE_SAMPLE_N)
    value, procs, slowest = oracle_throughput(workload, ns, args.steps, args.warmup)
    note = (f"{procs} concurrent single-thread oracle processes (one per host core), each {args.steps} timed "
            f"steps of its own {ns}-particle replica of {workload.name} (same density, shear, tolerance)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * slowest / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload.name, "n": workload.n, "box": workload.L[0],
                       "kappa_tau": workload.kappa_tau, "cg_tol": workload.tol,
                       "precision": "fp64", "sample_n": ns, "processes": procs, "l2": "cpu"},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": procs, "kind": "oracle",
                             "sample": note},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64-comparison", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="override the particle count (diagnostics)")
    ap.add_argument("--workload", default="mixed",
                    choices=["mixed", "lowshear", "plain", "learned", "batch", "large", "config5", "flexible", "vcorr",
                             "fdt"],
                    help="mixed: N=262,144 precision workload at kappa tau 0.5 (the default line); lowshear: "
                         "the same at kappa tau 0.05; plain: the FP64 workload (N=4,096, 1e-10); learned: "
                         "N=262,144 with the learned warm start; batch: 64 replicas; large: N=4,194,304; "
                         "vcorr: the velocity cross-correlation of Fig. vv on the paper's box; fdt: "
                         "A^(1/2) g (FDT-consistent noise) on the N=262,144 system")
    ap.add_argument("--train-steps", type=int, default=520,
                    help="learned workload: solves streamed into the online training (13 trajectories)")
    ap.add_argument("--burn-in", type=int, default=None,
                    help="untimed steps before the warm-up, so that the timed steps come from the trajectory's "
                         "steady state (the uniform start clusters: ~13 -> ~18 pairs per row and 42 -> 56 CG "
                         "iterations by step ~400 of the 2,000-step N = 262,144 runs); default 1000 for the "
                         "N = 262,144 workloads, 0 for plain (its 200 timed steps are the whole run)")
    ap.add_argument("--solver-config", type=int, default=None,
                    help="tile configuration of the persistent mixed solver (sp_set_solver_config) instead of "
                         "autotuning; 9 is the on-chip k32_cg_resident<512,4>, 0 the streaming "
                         "k32_cg_persistent<6,1,0,1024>")
    ap.add_argument("--profile-timed", action="store_true",
                    help="bracket the timed steps of the main line with cudaProfilerStart/Stop, so that "
                         "`ncu --profile-from-start off` captures the steady state and not the burn-in")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "ours" and args.workload not in ("mixed", "lowshear", "plain"):
        return {"learned": run_learned, "batch": run_batch, "large": run_large, "config5": run_large,
                "flexible": run_flexible, "vcorr": run_vcorr, "fdt": run_fdt}[args.workload](args)

    workload = {"mixed": synth.PRECISION, "lowshear": synth.PRECISION_LOW_SHEAR,
                "plain": synth.PLAIN_FP64}[args.workload]
    if args.workload == "plain":
        args.precision = "fp64"
    if args.burn_in is None:
        args.burn_in = 0 if args.workload == "plain" or args.n else 1000
    if args.n:
        workload = synth.cubic(f"n{args.n}", args.n, workload.kappa_tau, workload.steps, workload.tol,
                               workload.seed)
    if args.impl == "reference":
        run_reference(args, workload)
        return

    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_1808_06381_gb300 as ss
    ss.load()
    n, L = workload.n, workload.L
    seed = replica_seed(workload.seed, rank)
    pos0 = synth.uniform_positions(n, L, seed)
    kappa = ss.kappa_from_kappa_tau(workload.kappa_tau)
    def make_sim(precision):
        return ss.Simulation(n, L, kappa, alpha=workload.alpha, eps=workload.eps, zeta=workload.zeta,
                             kT=workload.kT, dt=workload.dt, rc=workload.rc, seed=seed, precision=precision,
                             warm_start="prev", cg_tol=workload.tol, cg_max_iter=2000, device=local_rank,
                             positions=pos0)

    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    gpu_uuid = None
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        pass
    # clocks over the whole GPU phase of the run (the timed region alone is short)
    clocks_run = ClockSampler(gpu_uuid)
    clocks_run.start()

    # the FP64 solver on the same workload, for comparison (same steps, same timing)
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64_comparison:
        sim64 = make_sim("fp64")
        if args.burn_in:
            sim64.step(args.burn_in)
        for _ in range(args.warmup):
            sim64.step(1)
        t64, _, it64, res64 = run_steps(sim64, args.steps, stream, flush)
        fp64 = {"value": n * args.steps / (t64 / 1e3), "ms_per_step": t64 / args.steps,
                "cg_iterations_per_step": it64 / args.steps, "max_true_residual": res64}
        sim64.close()

    sim = make_sim(args.precision)
    if args.burn_in:   # untimed: the trajectory's steady state
        sim.step(args.burn_in)
    # the persistent solver's tile configuration for this system (cached on disk
    # when SHEARSIM_TUNE_CACHE names a file); untimed, like the warm-up
    tune = None
    if args.precision == "mixed":
        tune = (sim.set_solver_config(args.solver_config) if args.solver_config is not None
                else sim.autotune(trials=2))
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()

    clocks = ClockSampler(gpu_uuid)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_timed:
        torch.cuda.profiler.start()
    total_ms, launches, iters, max_res = run_steps(sim, args.steps, stream, flush)
    torch.cuda.synchronize()
    if args.profile_timed:
        torch.cuda.profiler.stop()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()

    t_max = max_over_ranks(total_ms, dist, "cuda")
    value = whole_job_value(n, world, args.steps, t_max)

    # per-kernel timing of one more step (CUDA events on the simulation's
    # stream), then the two loop kernels launched back to back on that system
    prof = sim.profile_step()
    spmv_avg_ms = prof["spmv_probe_ms"]
    algo = spmv_algorithmic_bytes(prof["n"], prof["nnz"], args.precision)
    upd_algo = update_algorithmic_bytes(prof["n"], args.precision)
    peak, peak_kind = measured_peaks()
    achieved = algo / (spmv_avg_ms * 1e-3) / 1e9
    upd_achieved = upd_algo / (prof["update_probe_ms"] * 1e-3) / 1e9
    persistent = None
    if prof["persistent_ms"] > 0 and args.precision == "fp64":
        plan = plan_algorithmic_bytes(prof["n"], prof["cg_iterations"], "fp64")
        pach = plan / (prof["persistent_ms"] * 1e-3) / 1e9
        persistent = {"kernel": "k64_cg_persistent", "bound": "latency", "achieved": pach, "peak": peak,
                      "unit": "GB/s", "frac": pach / peak, "traffic": None,
                      "peak_source": f"hbm_gbs {peak_kind} (burst copy)",
                      "algorithmic_bytes_per_launch": plan,
                      "algorithmic_bytes_rule": f"{FP64_BYTES_PER_PARTICLE_ITERATION:g} B per particle per CG "
                                                "iteration x n x iterations",
                      "avg_launch_ms": prof["persistent_ms"], "cg_iterations": prof["cg_iterations"],
                      "true_residual_checks": prof["true_checks"], "grid": prof["persistent_blocks"],
                      "note": "one cooperative launch per solve; the system stays in L2 and GB300 issues FP64 at "
                              "~2 FMA per clock per SM: bound by the FP64 pipe, the gathers' latency and the grid "
                              "reductions (two per iteration; one in the pipelined form that systems of fewer "
                              "than 512 rows per SM take), so frac is an algorithmic-equivalent bandwidth"}
    elif prof["persistent_ms"] > 0:
        pbytes = persistent_algorithmic_bytes(prof["n"], prof["nnz"], prof["cg_iterations"], prof["true_checks"],
                                              bool(prof.get("persistent_init")))
        pach_detail = pbytes / (prof["persistent_ms"] * 1e-3) / 1e9
        plan = plan_algorithmic_bytes(prof["n"], prof["cg_iterations"], "mixed")
        pach = plan / (prof["persistent_ms"] * 1e-3) / 1e9
        kname = solver_kernel_name(tune)
        resident = bool(tune and tune.get("resident"))
        traffic = profiled_traffic(workload.name, tune, args.burn_in)
        persistent = {"kernel": kname, "bound": "latency" if resident else "hbm", "achieved": pach, "peak": peak,
                      "unit": "GB/s", "frac": pach / peak, "traffic": traffic,
                      "peak_source": f"hbm_gbs {peak_kind} (burst copy)",
                      "algorithmic_bytes_per_launch": plan,
                      "algorithmic_bytes_rule": f"{MIXED_BYTES_PER_PARTICLE_ITERATION:g} B per particle per CG "
                                                "iteration x n x iterations",
                      "avg_launch_ms": prof["persistent_ms"],
                      "cg_iterations": prof["cg_iterations"], "true_residual_checks": prof["true_checks"],
                      "grid": prof["persistent_blocks"],
                      "detailed_bytes_per_launch": pbytes, "detailed_frac": pach_detail / peak,
                      "dram_gbs": traffic / (prof["persistent_ms"] * 1e-3) / 1e9 if traffic else None,
                      "dram_frac": traffic / (prof["persistent_ms"] * 1e-3) / 1e9 / peak if traffic else None,
                      "note": ("one launch per solve; CUDA events on the simulation's stream; rows, vectors "
                               "and in-block entries stay on chip (registers, shared memory), so DRAM "
                               "traffic is a small fraction of the algorithmic bytes: the solve is bound by "
                               "its grid-wide reductions and halo-gather latency, and frac is an "
                               "algorithmic-equivalent bandwidth, not DRAM use (dram_frac is)"
                               if resident else
                               "one launch per solve; CUDA events on the simulation's stream; the "
                               "solver's working set (~60 MB) is L2-resident during the solve")}

    # end to end through the public API: host positions in, step, host positions out in
    # one call (sp_step_host; two pinned host buffers used in turn: each step's output is
    # the next step's input)
    import ctypes  # noqa: F401
    bufs = [torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    sim.get_positions(bufs[0])
    delta, _ = sim.state()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        delta = sim.step_host(bufs[k & 1], delta, 1, bufs[(k + 1) & 1])["delta"]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = whole_job_value(n, world, args.e2e_steps, max_over_ranks(1e3 * e2e_s, dist, "cuda"))
    clk_run = clocks_run.stop()

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(workload, args.precision)
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": workload.name, "n": n, "box": L[0], "density": 3.0,
                       "kappa_tau": workload.kappa_tau, "alpha": workload.alpha, "dt": workload.dt,
                       "cg_tol": workload.tol, "precision": args.precision, "warm_start": "prev",
                       "replicas": world, "l2": "flushed between timed steps (512 MB write)",
                       "burn_in_steps": args.burn_in,
                       "regime": ("steady state: timed after the untimed burn-in" if args.burn_in
                                  else "from the uniform start")},
            "cg_iterations_per_step": iters / args.steps, "max_true_residual": max_res,
            "gpu_launches": launches,
            "roofline": persistent if persistent else {
                "kernel": "k32_spmv" if args.precision == "mixed" else "k64_spmv",
                "bound": "hbm" if algo > L2_BYTES else "latency",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_source": f"hbm_gbs {peak_kind} (burst copy)",
                "algorithmic_bytes_per_launch": algo, "avg_launch_ms": spmv_avg_ms,
                "launches_timed": prof["probe_reps"],
                "note": "CUDA events around back-to-back launches on the solved system; the solver's "
                        f"working set ({algo / 1e6:.1f} MB per SpMV) stays in L2 between launches, so frac "
                        "is an algorithmic-equivalent bandwidth of a latency-bound kernel"
                        if algo <= L2_BYTES else
                        "CUDA events around back-to-back launches on the solved system"},
            "roofline_spmv_kernel": {"kernel": "k32_spmv" if args.precision == "mixed" else "k64_spmv",
                                     "achieved": achieved, "frac": achieved / peak,
                                     "algorithmic_bytes_per_launch": algo, "avg_launch_ms": spmv_avg_ms,
                                     "note": "the two-kernel solver's SpMV, launched back to back"},
            "roofline_update": {"kernel": "k32_update" if args.precision == "mixed" else "k64_update",
                                "achieved": upd_achieved, "frac": upd_achieved / peak,
                                "algorithmic_bytes_per_launch": upd_algo, "avg_launch_ms": prof["update_probe_ms"]},
            "kernel_ms_per_step": {k: prof[k] for k in ("persistent_ms", "spmv_ms", "update_ms", "true_residual_ms",
                                                         "build_ms", "sort_ms", "count_ms", "fill_ms",
                                                         "assemble_ms", "other_ms", "init_ms", "stress_ms",
                                                         "integrate_ms")},
            "autotune": tune,
            "matrix": {"nnz": prof["nnz"], "stored_with_padding": prof["nnz_slots"]},
            "fp64_comparison": fp64,
            "e2e": {"value": e2e_value, "unit": "particle-steps/s", "h2d_bytes_per_step": n * 24 + 8,
                    "d2h_bytes_per_step": n * 24 + int(ss.load().sp_state_record_bytes()),
                    "steps": args.e2e_steps},
            "clocks": clk,
            "clocks_run": clk_run,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


def _common_line(metric_value, n_total, steps, warmup, ms_per_step, dtype, config, extra):
    line = {"metric": METRIC, "value": metric_value, "unit": "particle-steps/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}
    line.update(extra)
    return line


def _sim(ss, w, precision, warm, pos=None, seed=None):
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    return ss.Simulation(w.n, w.L, kappa, alpha=w.alpha, eps=w.eps, zeta=w.zeta, kT=w.kT, dt=w.dt, rc=w.rc,
                         seed=w.seed if seed is None else seed, precision=precision, warm_start=warm,
                         cg_tol=w.tol, cg_max_iter=2000,
                         positions=synth.uniform_positions(w.n, w.L, w.seed) if pos is None else pos)


TRAIN_SEEDS = 13   # trajectories of the precision workload the training streams its solves from


def run_learned(args):
    """Learned warm start at N=262,144, kappa*tau=0.5: the network is trained online on solves
    streamed from TRAIN_SEEDS trajectories of the precision workload (--train-steps solves in all,
    one Adam step per solve, untimed), then K steps of a held-out trajectory are timed with it
    and, from the same state, with a cold start (v0 = 0) and with the previous-velocity start."""
    import torch
    import paper_1808_06381_gb300 as ss
    ss.load()
    w = synth.LEARNED
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    weights, losses, t_train = train_network(ss, args.train_steps)
    # the held-out trajectory three times from the same start and burn-in: with the trained
    # network, with a cold start (v0 = 0) and with the previous velocities; the solver
    # configuration the autotuner picks for the first
    results, tune, clk, launches, prof = {}, None, None, 0, None
    for mode in ("learned", "none", "prev"):
        sim = _sim(ss, w, "mixed", "none" if mode == "none" else "prev")
        if tune is None:
            tune = sim.autotune(trials=1)
        else:
            sim.set_solver_config(tune["config"])
        sim.step(args.warmup)
        if mode == "learned":
            sim.mpnn_enable(weights=weights)
        sim.step(1)   # (the learned form's graph is captured here)
        if mode == "learned":
            clocks = ClockSampler(None)
            clocks.start()
        torch.cuda.synchronize()
        t, nl, iters, res = run_steps(sim, args.steps, stream, flush)
        if mode == "learned":
            clk = clocks.stop()
            launches = nl
            prof = sim.profile_step()
        results[mode] = (t, iters, res)
        sim.close()
    n = w.n
    val = n * args.steps / (results["learned"][0] / 1e3)
    line = _common_line(val, n, args.steps, args.warmup, results["learned"][0] / args.steps, "bf16+f32+f64",
                        {"workload": w.name, "n": n, "kappa_tau": w.kappa_tau, "cg_tol": w.tol,
                         "precision": "mixed", "warm_start": "learned", "train_steps": args.train_steps,
                         "l2": "flushed between timed steps (512 MB write)"},
                        {"cg_iterations_per_step": results["learned"][1] / args.steps,
                         "max_true_residual": results["learned"][2],
                         "comparison": {k: {"value": n * args.steps / (v[0] / 1e3),
                                            "cg_iterations_per_step": v[1] / args.steps,
                                            "max_true_residual": v[2]}
                                        for k, v in results.items()},
                         "training_loss_first_last": [losses[0], losses[-1]] if losses else None,
                         "training": {"solves": len(losses), "trajectories": TRAIN_SEEDS, "seconds": t_train},
                         "mpnn_ms_per_step": prof["mpnn_ms"], "gpu_launches": launches, "clocks": clk,
                         "autotune": tune})
    print(json.dumps(line), flush=True)


def run_batch(args):
    """64 replicas (N log-uniform in [8192, 131072], kappa*tau log-uniform in [0.01, 1]) advanced
    as one batch (one graph per step, one cooperative solve launch) versus the same replicas
    stepped one after another.  The batch's data (~1.3 GB) is larger than L2."""
    import torch
    import paper_1808_06381_gb300 as ss
    ss.load()
    reps = synth.batch_replicas()
    kws = [dict(n=r.n, L=r.L, kappa=ss.kappa_from_kappa_tau(r.kappa_tau), seed=r.seed, cg_tol=r.tol,
                precision="mixed", warm_start="prev", cg_max_iter=2000) for r in reps]
    pos = [synth.uniform_positions(r.n, r.L, r.seed) for r in reps]
    ntot = sum(r.n for r in reps)
    batch = ss.Batch(kws, positions=pos)
    batch.step(args.warmup)
    torch.cuda.synchronize()
    # the untuned configuration (0) first, then the autotuner's choice
    t0 = time.perf_counter()
    batch.step(args.steps)
    t_untuned = time.perf_counter() - t0
    tune = batch.autotune(trials=2)
    batch.step(1)   # the re-captured graph
    torch.cuda.synchronize()
    clocks = ClockSampler(None)
    clocks.start()
    t0 = time.perf_counter()
    infos = batch.step(args.steps)
    t_batch = time.perf_counter() - t0
    clk = clocks.stop()
    iters = sum(x["cg_iterations"] for x in infos)
    worst = max(x["last_residual"] for x in infos)
    launches = sum(x["kernel_launches"] for x in infos)
    blocks = batch.blocks().tolist()
    batch.close()
    # the same replicas, one after another (each its own graph per step)
    sims = [ss.Simulation(positions=pos[k], **kws[k]) for k in range(len(reps))]
    for sm in sims:
        sm.step(args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for sm in sims:
            sm.step(1)
    t_seq = time.perf_counter() - t0
    for sm in sims:
        sm.close()
    val = ntot * args.steps / t_batch
    line = _common_line(val, ntot, args.steps, args.warmup, 1e3 * t_batch / args.steps, "f32+f64",
                        {"workload": "batch-64-replicas", "replicas": len(reps), "n_total": ntot,
                         "n_min": min(r.n for r in reps), "n_max": max(r.n for r in reps),
                         "cg_tol": reps[0].tol, "precision": "mixed", "l2": "working set > L2"},
                        {"cg_iterations_per_replica_step": iters / (len(reps) * args.steps),
                         "max_true_residual": worst, "gpu_launches": launches,
                         "sequential": {"value": ntot * args.steps / t_seq, "ms_per_step": 1e3 * t_seq / args.steps},
                         "speedup_vs_sequential": t_seq / t_batch, "blocks_per_replica": blocks,
                         "untuned": {"config": 0, "value": ntot * args.steps / t_untuned,
                                     "ms_per_step": 1e3 * t_untuned / args.steps},
                         "autotune": tune,
                         "timing": "host wall clock around the synchronising batch call", "clocks": clk})
    print(json.dumps(line), flush=True)


def train_network(ss, steps: int, prior: bool = True):
    """Online training on solves streamed from TRAIN_SEEDS trajectories of the precision workload
    (N = 262,144); returns (weights, losses, seconds).  prior=False: the network's
    previous-velocity feature is 0 (its readout starts at the Jacobi guess b / A_ii), as the
    flexible solve's preconditioner applies it."""
    w = synth.LEARNED
    losses, weights = [], None
    per_seed = max(1, steps // TRAIN_SEEDS)
    t0 = time.perf_counter()
    for k in range(TRAIN_SEEDS):
        seed = synth.PRECISION.seed + 100 + k
        tr = _sim(ss, w, "mixed", "prev", pos=synth.uniform_positions(w.n, w.L, seed), seed=seed)
        tr.step(3)
        tr.mpnn_enable(seed=1, weights=weights)
        if not prior:
            tr.mpnn_set_prior(False)
            if weights is None:
                wt = tr.mpnn_weights()
                wt[len(wt) - 11 + 8], wt[len(wt) - 11 + 9] = 1.0, 0.0
                tr.mpnn_set_weights(wt)
        for _ in range(per_seed):
            tr.step(1)
            losses.append(tr.mpnn_train_step(lr=2e-3))
        weights = tr.mpnn_weights()
        tr.close()
    return weights, losses, time.perf_counter() - t0


SQ_EVERY = 100   # steps between two S(qx, qy) of the large-scale workload


def run_large(args):
    """N = 4,194,304 (box 111.8), mixed solver: the solver's working set (~2 GB) is far larger
    than L2, so this is the HBM-bound regime of the same kernels.  --workload config5 adds the
    large-scale workload's learned warm start (the network trained on solves streamed from
    trajectories of the N = 262,144 workload; its weights do not depend on N) and S(qx, qy) on
    a 256^3 grid every SQ_EVERY steps, inside the timed region (K >= SQ_EVERY) and amortised."""
    import torch
    import paper_1808_06381_gb300 as ss
    ss.load()
    w = synth.LARGE
    learned = args.workload == "config5"
    stream = torch.cuda.current_stream()
    flush = torch.empty(4, dtype=torch.float32, device="cuda")   # inputs are larger than L2
    training = None
    if learned:
        weights, losses, t_train = train_network(ss, args.train_steps)
        training = {"solves": len(losses), "trajectories": TRAIN_SEEDS, "seconds": t_train, "n": synth.LEARNED.n,
                    "loss_first_last": [losses[0], losses[-1]] if losses else None}
    sim = _sim(ss, w, "mixed", "prev")
    tune = (sim.set_solver_config(args.solver_config) if args.solver_config is not None
            else sim.autotune(trials=1))
    sim.step(args.warmup)
    if learned:
        sim.mpnn_enable(weights=weights)
        sim.step(1)
    t_sq = time.perf_counter()
    sim.structure_factor(48, 48, grid=256)
    torch.cuda.synchronize()
    t_sq = time.perf_counter() - t_sq
    clocks = ClockSampler(None)
    clocks.start()
    t, launches, iters, res = 0.0, 0, 0, 0.0
    n_sq, t_sq_in = 0, 0.0
    done = 0
    while done < args.steps:
        chunk = min(SQ_EVERY, args.steps - done)
        tc, lc, ic, rc = run_steps(sim, chunk, stream, flush)
        t += tc
        launches += lc
        iters += ic
        res = max(res, rc)
        done += chunk
        if chunk == SQ_EVERY:   # S(qx, qy) every SQ_EVERY steps, timed with the steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.structure_factor(48, 48, grid=256)
            e1.record(stream)
            e1.synchronize()
            t_sq_in += e0.elapsed_time(e1)
            n_sq += 1
    clk = clocks.stop()
    prof = sim.profile_step()
    peak, peak_kind = measured_peaks()
    plan = plan_algorithmic_bytes(prof["n"], prof["cg_iterations"], "mixed")
    pach = plan / (prof["persistent_ms"] * 1e-3) / 1e9
    pbytes = persistent_algorithmic_bytes(prof["n"], prof["nnz"], prof["cg_iterations"], prof["true_checks"],
                                          bool(prof.get("persistent_init")))
    spmv = spmv_algorithmic_bytes(prof["n"], prof["nnz"], "mixed") / (prof["spmv_probe_ms"] * 1e-3) / 1e9
    traffic = LARGE_PROFILED_TRAFFIC.get(solver_kernel_name(tune))
    sim.close()
    n = w.n
    total = t + t_sq_in
    line = _common_line(n * args.steps / (total / 1e3), n, args.steps, args.warmup, total / args.steps, "f32+f64",
                        {"workload": ("config5-" if learned else "") + w.name, "n": n, "box": w.L[0],
                         "kappa_tau": w.kappa_tau, "cg_tol": w.tol, "precision": "mixed",
                         "warm_start": "learned" if learned else "prev", "l2": "working set > L2",
                         "structure_factor": f"256^3 CIC grid every {SQ_EVERY} steps (timed)"},
                        {"cg_iterations_per_step": iters / args.steps, "max_true_residual": res,
                         "gpu_launches": launches,
                         "roofline": {"kernel": solver_kernel_name(tune), "bound": "hbm", "achieved": pach,
                                      "peak": peak, "unit": "GB/s", "frac": pach / peak, "traffic": traffic,
                                      "peak_source": f"hbm_gbs {peak_kind} (burst copy)",
                                      "algorithmic_bytes_per_launch": plan,
                                      "algorithmic_bytes_rule": f"{MIXED_BYTES_PER_PARTICLE_ITERATION:g} B per "
                                                                "particle per CG iteration x n x iterations",
                                      "avg_launch_ms": prof["persistent_ms"],
                                      "detailed_bytes_per_launch": pbytes,
                                      "dram_gbs": traffic / (prof["persistent_ms"] * 1e-3) / 1e9 if traffic else None,
                                      "dram_frac": (traffic / (prof["persistent_ms"] * 1e-3) / 1e9 / peak
                                                    if traffic else None)},
                         "roofline_spmv_kernel": {"achieved": spmv, "frac": spmv / peak,
                                                  "avg_launch_ms": prof["spmv_probe_ms"]},
                         "kernel_ms_per_step": {k: prof[k] for k in ("persistent_ms", "build_ms", "fill_ms",
                                                                      "assemble_ms", "count_ms", "sort_ms",
                                                                      "other_ms", "mpnn_ms")},
                         "autotune": tune, "structure_factor_ms": 1e3 * t_sq,
                         "structure_factor_in_region": {"calls": n_sq, "ms": t_sq_in},
                         "steps_only_value": n * args.steps / (t / 1e3),
                         "training": training, "clocks": clk})
    print(json.dumps(line), flush=True)


def run_flexible(args):
    """The learned preconditioner on the N = 262,144 system in FP64: flexible CG (FCG(1)) with the
    network applied to the residual at every iteration, against FCG with Jacobi and against the
    FP64 PCG of the time step (one graph launch), all from v0 = 0 to the workload's 1e-8.  The
    network is trained beforehand (untimed) with its previous-velocity feature 0 on solves
    streamed from TRAIN_SEEDS trajectories.  Value: particles per second of the flexible solve
    with the network (solves of the N-particle system per second x N)."""
    import torch
    import paper_1808_06381_gb300 as ss
    ss.load()
    w = synth.PRECISION
    weights, losses, t_train = train_network(ss, args.train_steps, prior=False)
    sim = _sim(ss, w, "fp64", "none")
    sim.step(args.warmup)
    sim.build_neighbors()
    sim.assemble()
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        best, info = None, None
        for _ in range(max(1, args.steps)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best, info

    t_pcg, i_pcg = timed(lambda: sim.solve_velocities())
    t_jac, i_jac = timed(lambda: sim.solve_flexible(0))
    sim.mpnn_enable(weights=weights)
    sim.mpnn_set_prior(False)
    t_net, i_net = timed(lambda: sim.solve_flexible(1))
    sim.close()
    n = w.n
    res = {"pcg_graph": (t_pcg, i_pcg), "fcg_jacobi": (t_jac, i_jac), "fcg_network_every_iteration": (t_net, i_net)}
    line = {"metric": "particle-solves/s of the N=262,144 system to 1e-8 (flexible CG, learned preconditioner)",
            "value": n / (t_net * 1e-3), "unit": "particle-solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_net, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (network bf16+f32)", "data": "synthetic",
            "config": {"workload": "flexible-" + w.name, "n": n, "cg_tol": w.tol, "precision": "fp64",
                       "start": "v0 = 0", "timing": "best of the timed solves, CUDA events"},
            "comparison": {k: {"ms": v[0], "iterations": v[1]["iterations"], "residual": v[1]["residual"],
                               "value": n / (v[0] * 1e-3)} for k, v in res.items()},
            "training": {"solves": len(losses), "trajectories": TRAIN_SEEDS, "seconds": t_train,
                         "prior": "previous-velocity feature 0"},
            "gpu_launches": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


# FP32 operations per pair of the all-pairs velocity correlation, counted from
# its definition: the separation (3), the y image with the sheared x shift (4),
# the x and z images (3 each) and |R|^2 (3); for a pair inside the cut-off also
# the square root, the bin scaling and floor, and the product u . u' (6).
VCORR_OPS_ALL, VCORR_OPS_IN = 16, 6
# DRAM bytes per launch of k_vc_pairs on this workload (one ncu capture); the
# particles stay in L2 and shared memory
VCORR_PROFILED_TRAFFIC = 578304.0
FP32_LANES_PER_SM = 128


def run_vcorr(args):
    """Fig. vv on the paper's box (87.6 x 43.6 x 22 lambda^3, N = 17,191, kappa tau = 0):
    every pair, 120 bins of 0.25 lambda up to 30 lambda.  Value: pairs per second of the
    whole call through the C ABI with the simulation's state resident (CUDA events on its
    stream); e2e: the host-array entry (positions and velocities copied in every call)."""
    import torch
    import paper_1808_06381_gb300 as ss
    ss.load()
    w = synth.PAPER_BOX_VV
    nbins, rmax = 120, 12.25
    stream = torch.cuda.current_stream()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 512 MB > L2
    sim = _sim(ss, w, "mixed", "prev")
    sim.step(20)
    for _ in range(args.warmup):
        sim.velocity_correlation(nbins, rmax)
    clocks = ClockSampler(None)
    clocks.start()
    total, kern = 0.0, 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = sim.velocity_correlation(nbins, rmax)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
        kern += r["pairs_ms"]
    clk = clocks.stop()
    pos, v = sim.get_positions(), sim.get_velocities()
    delta = sim.state()[0]
    kappa = ss.kappa_from_kappa_tau(w.kappa_tau)
    sim.close()
    pairs = r["pairs"]
    t_e2e = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        ss.velocity_correlation(pos, v, w.L, delta, kappa, nbins, rmax)
    t_e2e = (time.perf_counter() - t_e2e) / max(1, args.e2e_steps)
    ms = total / args.steps
    kms = kern / args.steps
    in_range = float(r["counts"].sum()) / pairs
    ops = pairs * (VCORR_OPS_ALL + VCORR_OPS_IN * in_range)
    sm_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = 152 * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    achieved = ops / (kms * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        p = oracle.Params(n=w.n, L=w.L, kappa=kappa)
        t0 = time.perf_counter()
        oracle.velocity_correlation(p, pos, delta, v, nbins, rmax)
        dt = time.perf_counter() - t0
        cpu = {"value": pairs / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
               "sample": f"the whole workload once (N={w.n}, {pairs} pairs), single thread, {dt:.2f} s"}
    line = {"metric": "velocity cross-correlation pairs/s (Fig. vv, all pairs, exact counts)",
            "value": pairs / (ms * 1e-3), "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (simulated state after 20 steps)",
            "config": {"workload": w.name, "n": w.n, "box": list(w.L), "kappa_tau": w.kappa_tau,
                       "nbins": nbins, "rmax": rmax, "l2": "flushed between calls (512 MB write)"},
            "gpu_launches": 6 * args.steps,
            "roofline": {"kernel": "k_vc_pairs", "bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": VCORR_PROFILED_TRAFFIC,
                         "peak_source": f"152 SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz "
                                        "(one FP32 operation per lane per clock)",
                         "ops_per_pair": VCORR_OPS_ALL + VCORR_OPS_IN * in_range, "avg_launch_ms": kms},
            "boundary_pairs": r["boundary_pairs"], "pairs_in_range": int(r["counts"].sum()),
            "e2e": {"value": pairs / t_e2e, "unit": "pairs/s", "h2d_bytes_per_step": 2 * w.n * 24,
                    "d2h_bytes_per_step": nbins * 16 + 16},
            "clocks": clk, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


# DRAM bytes per launch of k_cheb_step_df on this workload (one ncu capture)
FDT_PROFILED_TRAFFIC = 55.94e6


def fdt_algorithmic_bytes(n: int, nnz: int) -> float:
    """One Chebyshev degree step (mixed path, double-float records): per entry the
    column, the weight's two FP32 parts and the gathered 32-byte record of T_k; per row
    the slot map, A_ii's two parts, T_k and T_(k-1) read, T_(k+1) written, xi read and
    written (32 bytes each)."""
    return nnz * (4.0 + 8.0 + 32.0) + n * (4.0 + 8.0 + 5 * 32.0)


def run_fdt(args):
    """xi = p(A) g ~ A^(1/2) g on the N=262,144 mixed system after the warm-up steps
    (degree 32 on [1, Gershgorin max]); value: particles per second of the whole call
    (host arrays in and out, so it is also the end-to-end figure); roofline: the
    degree steps, CUDA events on the simulation's stream."""
    import torch
    import paper_1808_06381_gb300 as ss
    ss.load()
    w = synth.PRECISION
    degree = 32
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 512 MB > L2
    sim = _sim(ss, w, "mixed", "prev")
    sim.step(args.warmup)
    sim.build_neighbors()
    sim.assemble()
    g = np.random.default_rng(w.seed).standard_normal((w.n, 3))
    for _ in range(2):
        sim.sqrt_apply(g, degree)
    clocks = ClockSampler(None)
    clocks.start()
    total, kern = 0.0, 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, lmax, ms = sim.sqrt_apply(g, degree, timing=True)
        total += time.perf_counter() - t0
        kern += ms
    clk = clocks.stop()
    prof = sim.profile_step()
    sim.close()
    ms_call = 1e3 * total / args.steps
    step_ms = kern / args.steps / degree
    nbytes = fdt_algorithmic_bytes(prof["n"], prof["nnz"])
    peak, peak_kind = measured_peaks()
    ach = nbytes / (step_ms * 1e-3) / 1e9
    line = {"metric": "A^(1/2) g (FDT-consistent noise) particles/s, Chebyshev degree 32",
            "value": w.n / (ms_call * 1e-3), "unit": "particles/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_call, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32x2 (double-float)",
            "data": "synthetic (the simulated system after the warm-up steps)",
            "config": {"workload": w.name, "n": w.n, "degree": degree, "lambda_max": lmax,
                       "l2": "flushed between calls (512 MB write)"},
            "gpu_launches": args.steps * (degree + 4),
            "roofline": {"kernel": "k_cheb_step_df", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "traffic": FDT_PROFILED_TRAFFIC,
                         "peak_source": f"hbm_gbs {peak_kind} (burst copy)",
                         "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": step_ms},
            "e2e": {"value": w.n / (ms_call * 1e-3), "unit": "particles/s", "h2d_bytes_per_step": w.n * 24,
                    "d2h_bytes_per_step": w.n * 24 + 8},
            "clocks": clk, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
