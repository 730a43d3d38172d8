"""Benchmark: single-bead Metropolis updates per second of the parallel-tempering engine.

Default workload (one GPU, the long-chain configuration): one PT ensemble of an N = 1000 bead
chain with 128 replicas at geometric temperatures 0.2-3.0, displacement half-width 0.3, an
exchange round after every sweep, an FP64 full-energy recompute every 1000 sweeps and 4096
FP64 histogram bins per temperature slot. One step = 1000 sweeps (128 x 1000 x 1000 = 128 M
single-bead updates); 20 steps are the whole 2e4-sweep run. ``--workload paper-scale`` runs
the N = 100 configuration instead: 4 ensembles (seeds 1-4) of 64 replicas, one step = 1000
sweeps of all four. Under torchrun every rank runs its own ensembles (seeds offset by the
rank): weak scaling, no collective on the data path.

Prints one JSON line (see the repository's benchmark contract). ``--impl reference`` times
the FP64 CPU oracle instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

T_MIN, T_MAX = 0.2, 3.0
SWEEPS_PER_STEP = 1000
# FP32 flops per pair evaluation (FMA = 2): 3 subtractions for the coordinate differences, 5
# for r^2 (a multiply and two FMAs), 1 for sigma^2 / r^2, 2 multiplies for the sixth power, 3
# for s^6 (s^6 - 1) minus the shift, 1 to accumulate; the reciprocal is not counted.
FLOPS_PER_PAIR = 15
METRIC = "single-bead Metropolis updates/sec (all replicas)"
KERNEL_NAMES = {0: "k_sweep", 1: "k_sweep_la", 2: "k_sweep_team", 3: "k_sweep_wpm", 4: "k_sweep_reg",
                5: "k_sweep_grp", 6: "k_sweep_cta"}
KERNEL_DESC = {0: "warp per replica", 1: "lookahead groups of 8 moves", 2: "team of warps per replica",
               3: "warp per move of a group", 4: "warp per replica, chain in registers, deferred double-float",
               5: "CTA per replica, one warp per move of a group, chain in registers",
               6: "CTA per replica, every thread a chain slice and a group of 16 moves in packed FP32x2, control warps"}
UNIT = "updates/s"
# The plain (one-context) workloads: beads, replicas, ensembles per GPU.
PLAIN = {
    "long": dict(N=1000, R=128, E=1, label="long chains (configuration 3)"),
    "paper-scale": dict(N=100, R=64, E=4, label="paper-scale (configuration 2)"),
}
# DRAM bytes read + written per sweep (ncu dram__bytes_read.sum + dram__bytes_write.sum of one
# launch of the kernel as it stands, divided by the sweeps that launch ran), keyed by
# (workload, kernel, launch mode); pairs without a current capture report null
TRAFFIC_BYTES = {("long", "k_sweep_cta", 1): 2926, ("paper-scale", "k_sweep_cta", 1): 2763}


def workload_text(w):
    c = PLAIN[w]
    ens = f"{c['E']} ensembles (seeds 1-{c['E']})" if c["E"] > 1 else "1 ensemble (seed 1)"
    return (f"PT polymer N={c['N']} beads, {c['R']} replicas at T geometric {T_MIN}-{T_MAX}, {ens} per GPU, "
            f"delta 0.3, exchange every sweep, FP64 recompute every 1000 sweeps, 4096 FP64 bins/slot; "
            f"1 step = {SWEEPS_PER_STEP} sweeps")


def updates_per_step(w):
    c = PLAIN[w]
    return c["E"] * c["R"] * c["N"] * SWEEPS_PER_STEP


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws: int, backend: str):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def reduce_max(value: float, dist, device=None) -> float:
    """Max over ranks of a host scalar (no data-path collective: timing only)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def ensemble_params(rank: int, w: str):
    from paper_1107_3490_gb300 import inputs, pt
    c = PLAIN[w]
    made = []
    for e in range(c["E"]):
        seed = c["E"] * rank + e + 1
        T = inputs.temperature_ladder(T_MIN, T_MAX, c["R"])
        x0 = inputs.random_coil(c["N"], c["R"], seed, seed - 1)
        made.append(pt.make_params(c["N"], T, seed, ensemble_id=seed - 1, init_positions=x0,
                                   delta=0.3, recompute_every=1000, n_bins=4096))
    return made


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.file is None:
            return None
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def fp32_peak_tflops(num_sms: int, mhz: float) -> float:
    """FP32 peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return num_sms * 128 * 2 * mhz * 1e6 / 1e12


def _oracle_sample(w: str, threads: int):
    import oracle
    from paper_1107_3490_gb300 import inputs
    c = PLAIN[w]
    T = inputs.temperature_ladder(T_MIN, T_MAX, c["R"])
    return oracle.OracleEnsemble(inputs.random_coil(c["N"], c["R"], 1, 0), T, 1, delta=0.3,
                                 recompute_every=1000, n_bins=4096, threads=threads)


def cpu_baseline(w: str, target_s: float = 15.0, threads: int | None = None):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload:
    its ensemble seed 1, exchange every sweep."""
    c = PLAIN[w]
    threads = threads or os.cpu_count() or 1
    ens = _oracle_sample(w, threads)
    t0 = time.perf_counter()
    ens.run(2, 1)
    per_sweep = (time.perf_counter() - t0) / 2
    n = max(2, int(target_s / max(per_sweep, 1e-6)))
    t0 = time.perf_counter()
    ens.run(n, 1)
    dt = time.perf_counter() - t0
    return {"value": c["R"] * c["N"] * n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"ensemble seed 1 of {c['E']} (N={c['N']}, {c['R']} replicas), {n} sweeps after 2 warm-up "
                      f"sweeps, exchange every sweep, FP64 oracle with {threads} OpenMP threads; {dt:.1f} s"}


def run_reference(args):
    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return 0
    w = args.workload if args.workload in PLAIN else "long"
    c = PLAIN[w]
    threads = os.cpu_count() or 1
    ens = _oracle_sample(w, threads)
    t0 = time.perf_counter()
    ens.run(2, 1)
    per_sweep = (time.perf_counter() - t0) / 2
    budget = 150.0 / max(1, args.steps + args.warmup)  # whole run within a few minutes
    sweeps = max(1, int(budget / max(per_sweep, 1e-6)))
    for _ in range(args.warmup):
        ens.run(sweeps, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ens.run(sweeps, 1)
        times.append(time.perf_counter() - t0)
    upd = c["R"] * c["N"] * sweeps
    value = upd * len(times) / sum(times)
    sample = (f"each step: {sweeps} sweeps of ensemble seed 1 (N={c['N']}, {c['R']} replicas), "
              f"exchange every sweep, FP64 oracle, {threads} OpenMP threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_text(w), "reference_sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    w = args.workload
    c = PLAIN[w]
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(ws, "nccl")
    from paper_1107_3490_gb300 import pt

    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.Stream(device=dev)
    made = ensemble_params(rank, w)
    h = pt.pt_create_batch([p for p, _ in made], stream.cuda_stream)
    if args.kernel >= 0:
        pt.pt_set_sweep_kernel(h, args.kernel)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB of L2

    for _ in range(args.warmup):
        pt.pt_sweep(h, SWEEPS_PER_STEP, 1)
    if args.kernel < 0:
        # untimed, on the warmed-up chain (the state is restored afterwards), then one more
        # warm-up step with the chosen kernel
        kernel = pt.pt_autotune(h, 100, force=True)
        pt.pt_sweep(h, SWEEPS_PER_STEP, 1)
    else:
        kernel = args.kernel
    pt.pt_set_kernel_timing(h, True)
    pt.pt_sweep(h, 64, 1)
    pt.pt_sync(h)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            starts[k].record(stream)
            pt.pt_sweep(h, SWEEPS_PER_STEP, 1)
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kernel_ms, kernel_n = pt.pt_kernel_timing(h)
    lmode = pt.pt_get_launch_mode(h)
    pt.pt_sync(h)
    local_ms = sum(step_ms)
    total_ms = reduce_max(local_ms, dist, dev)
    value = updates_per_step(w) * ws * args.steps / (total_ms / 1e3)
    clocks = clk.summary()

    # ---- end to end through the C-ABI with host buffers: restore the state from pinned host
    # memory, run the step, checkpoint it back to pinned host memory
    nbytes = pt.pt_checkpoint_size(h)
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    pt.pt_checkpoint_into(h, host)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pt.pt_restore_from(h, host, nbytes)
        pt.pt_sweep(h, SWEEPS_PER_STEP, 1)
        pt.pt_checkpoint_into(h, host)
    e2e_s = reduce_max(time.perf_counter() - t0, dist, dev)
    e2e = {"value": updates_per_step(w) * ws * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # ---- roofline of the dominant kernel (the sweep): plain FP32 ALU work
    pairs_per_launch = c["E"] * c["R"] * c["N"] * 2 * (c["N"] - 1)  # pair evaluations per sweep
    achieved = pairs_per_launch * FLOPS_PER_PAIR / (kernel_ms / 1e3) / 1e12
    peak = fp32_peak_tflops(num_sms, 2070.0)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TRAFFIC_BYTES.get((w, KERNEL_NAMES[kernel], lmode)), "traffic_unit": "bytes per sweep",
                "kernel": KERNEL_NAMES[kernel],
                "kernel_ms_per_sweep": kernel_ms, "launches_sampled": kernel_n,
                "launch_mode": "persistent (exchange in kernel)" if lmode == 1 else "graph per sweep",
                "peak_basis": f"{num_sms} SMs x 128 FP32 lanes x 2 flops x 2070 MHz (max SM clock)"}
    if clocks and clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / fp32_peak_tflops(num_sms, clocks["sm_mhz"])
    pt.pt_destroy(h)
    # measured FP32 FMA throughput of this GPU (independent fmaf chains on every warp slot)
    fma_tflops, _ = pt.pt_fp32_fma_rate(stream.cuda_stream)
    roofline["peak_measured_fma"] = fma_tflops
    roofline["frac_of_measured_fma"] = achieved / fma_tflops

    # every step: the target-setting launch, then one cooperative launch and the round-count
    # update (persistent mode) or graphs of 32 (sweep, exchange) launch pairs
    launches_per_step = 3 if lmode == 1 else 1 + -(-SWEEPS_PER_STEP // 32) * 64
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_text(w), "name": c["label"],
                       "parallelism": f"ensembles per GPU, {ws} GPU(s), no collective",
                       "l2": "256 MB buffer written between timed steps (outside the per-step events)",
                       "sweep_kernel": KERNEL_DESC[kernel], "pair_evals_per_s": value * 2 * (c["N"] - 1)},
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "roofline": roofline,
            "clocks": clocks}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _timed(fn):
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


def run_batched(args):
    """256 uneven ensembles (N log-uniform 20-500, 8-64 replicas, T 0.2-3.0) in one context,
    against the plain form (each ensemble its own context, swept one after another) on the
    first ensembles. The batched context runs the autotuned kernel and launch mode; kernel 4
    is also timed in its work-list mode (every sweep of every replica in one launch per call)
    and in per-sweep launches (a CUDA graph of sweep and exchange launches)."""
    import torch
    from paper_1107_3490_gb300 import inputs, pt
    specs = inputs.batched_ensembles(256, n_sweeps=5000)
    made = [pt.make_params(sp.n_beads, sp.temperatures(), sp.seed, ensemble_id=sp.ensemble_id, n_bins=1024)
            for sp in specs]
    steps_sweeps = 100
    upd = sum(sp.n_beads * sp.n_replicas for sp in specs) * steps_sweeps
    h = pt.pt_create_batch([p for p, _ in made])
    kernel = pt.pt_autotune(h, 4)
    mode = pt.pt_get_launch_mode(h)

    def rate():
        for _ in range(args.warmup):
            pt.pt_sweep(h, steps_sweeps, 1)
        pt.pt_sync(h)

        def timed_steps():
            for _ in range(args.steps):
                pt.pt_sweep(h, steps_sweeps, 1)
            pt.pt_sync(h)
        return upd * args.steps / _timed(timed_steps)

    value = rate()
    per_mode = {}
    pt.pt_set_sweep_kernel(h, 4)
    for m, name in ((2, "kernel 4, work list (one launch per call)"), (0, "kernel 4, per-sweep launches (CUDA graph)")):
        pt.pt_set_launch_mode(h, m)
        per_mode[name] = rate()
    pt.pt_destroy(h)
    # plain form on a sample: one ensemble per context and per launch sequence
    sample = specs[:16]
    ctxs = []
    for sp, (p, _) in zip(sample, made[:16]):
        c = pt.pt_create_ex(p)
        pt.pt_autotune(c, 4)
        pt.pt_sweep(c, 10, 1)
        ctxs.append(c)
    for c in ctxs:
        pt.pt_sync(c)
    t = 0.0
    for c in ctxs:
        t += _timed(lambda: (pt.pt_sweep(c, steps_sweeps, 1), pt.pt_sync(c)))
    plain = sum(sp.n_beads * sp.n_replicas for sp in sample) * steps_sweeps / t
    for c in ctxs:
        pt.pt_destroy(c)
    modes = {0: "per-sweep launches", 1: "persistent (all replicas resident)", 2: "work list"}
    launches = {0: 1 + -(-steps_sweeps // 32) * 64, 1: 3, 2: 2}[mode]  # per call
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "256 uneven PT ensembles: N log-uniform 20-500, replicas uniform 8-64, "
                                   "T geometric 0.2-3.0, exchange every sweep; one step = 100 sweeps of all",
                       "sweep_kernel": KERNEL_NAMES[kernel], "launch_mode": modes[mode],
                       "gpu_launches_per_step": launches, "replicas": sum(sp.n_replicas for sp in specs)},
            "per_mode": per_mode,
            "plain_one_ensemble_per_launch": {"value": plain, "unit": UNIT, "sample": "first 16 ensembles, sequential"}}
    print(json.dumps(line), flush=True)
    return 0


def run_served(args):
    """A Poisson stream of PT jobs (N log-uniform 20-1000, 16-128 replicas, budgets
    log-uniform in [s_lo, s_hi] sweeps) through the continuous-batching server, against
    running jobs of the same stream one after another as plain contexts (on a sample). The
    configured stream has 2000 jobs with budgets 1e3-1e5 sweeps (about 8e14 pair
    evaluations, tens of minutes of GPU time); the default here scales the budgets by 1/10
    and the number of jobs by 1/2, and the line states the scale."""
    import threading
    from paper_1107_3490_gb300 import inputs, pt
    n_jobs = args.jobs
    jobs = inputs.served_jobs(n_jobs, s_lo=args.s_lo, s_hi=args.s_hi, rate_hz=args.rate)
    # clients arrive with their start conformations ready (made before the clock starts)
    made = [pt.make_params(j.n_beads, j.temperatures(), j.seed, ensemble_id=j.ensemble_id, n_bins=1024,
                           init_positions=pt.pt_make_coil(j.n_beads, j.n_replicas, j.seed, j.ensemble_id))
            for j in jobs]
    cfg = pt.pt_server_config_init(1000, 16 << 30)
    cfg.round_sweeps = 64
    if args.kernel >= 0:
        cfg.sweep_kernel = args.kernel
    srv = pt.pt_server_create(cfg)
    ids = [0] * n_jobs
    t_start = time.perf_counter()

    def feeder():
        for i, (j, (p, _)) in enumerate(zip(jobs, made)):
            delay = j.arrival_s - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            ids[i] = pt.pt_server_submit(srv, p, j.n_sweeps, 1)

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    lat = []
    for i, j in zip(ids, jobs):
        pt.pt_server_wait(srv, i, 7200.0)
        lat.append(pt.pt_server_result(srv, i, j.n_replicas, 1024)[3])
    makespan = time.perf_counter() - t_start
    upd = sum(j.n_beads * j.n_replicas * j.n_sweeps for j in jobs)
    pairs = sum(j.n_beads * j.n_replicas * j.n_sweeps * 2 * (j.n_beads - 1) for j in jobs)
    pt.pt_server_destroy(srv)
    # plain form: jobs of the stream one after another, each its own context (autotuned)
    sample = list(zip(jobs, made))[:: max(1, n_jobs // 12)][:12]
    t = 0.0
    for j, (p, _) in sample:
        c = pt.pt_create_ex(p)
        pt.pt_autotune(c, 4)
        t += _timed(lambda: (pt.pt_sweep(c, j.n_sweeps, 1), pt.pt_sync(c)))
        pt.pt_destroy(c)
    plain = sum(j.n_beads * j.n_replicas * j.n_sweeps for j, _ in sample) / t
    lat = sorted(lat)
    line = {"metric": METRIC, "value": upd / makespan, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": f"{n_jobs} PT jobs, Poisson arrivals at {args.rate}/s, N log-uniform 20-1000, "
                                   f"replicas uniform 16-128, budgets log-uniform {args.s_lo}-{args.s_hi} sweeps, "
                                   "exchange every sweep; server N_max 1000",
                       "scale_vs_configured": f"jobs {n_jobs}/2000, budgets {args.s_lo}-{args.s_hi} against 1e3-1e5",
                       "arrival_rate_per_s": args.rate, "pair_evaluations": pairs, "updates": upd,
                       "pool_kernels": "k_sweep_reg work list up to 320 beads, k_sweep_cta above"
                       if args.kernel < 0 else KERNEL_NAMES[args.kernel]},
            "latency_s": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                          "max": lat[-1]},
            "makespan_s": makespan,
            "plain_one_job_per_context": {"value": plain, "unit": UNIT,
                                          "sample": f"{len(sample)} jobs spread over the stream, sequential, autotuned"}}
    print(json.dumps(line), flush=True)
    return 0


def run_paper(args):
    """The paper's benchmark protocol (Sec. 4.2): N = 55, 4000 sweeps per replica, an exchange
    round every 1000 sweeps, n_r replicas (T geometric 0.2-3.0). As in the paper the GPU time
    includes copying the start conformations to the device and the results (energies,
    histograms, conformations) back; context creation is excluded like the CPU side's
    initialisation. S_p = t(one host core, FP64 oracle) / t(GPU). The oracle runs independent
    replicas, so its time is measured on a sample of replicas and scaled by n_r."""
    import numpy as np
    import oracle
    from paper_1107_3490_gb300 import inputs, pt
    N, SW, XE = 55, 4000, 1000
    n_rs = [1, 2, 4, 8, 16, 32, 60, 120, 240, 480, 960]
    n_s = 4
    Ts = inputs.temperature_ladder(0.2, 3.0, n_s)
    ens = oracle.OracleEnsemble(inputs.random_coil(N, n_s, 1), Ts, 1, n_bins=1024, e_min=-6.0 * N,
                                e_max=3.0 * N, threads=1)
    t0 = time.perf_counter()
    ens.run(SW, XE)
    cpu_per_rep = (time.perf_counter() - t0) / n_s
    rows = []
    for n_r in n_rs:
        T = inputs.temperature_ladder(0.2, 3.0, n_r) if n_r > 1 else np.array([1.0])
        x0 = inputs.random_coil(N, n_r, 1)
        p, keep = pt.make_params(N, T, 1, init_positions=x0, n_bins=1024, e_min=-6.0 * N, e_max=3.0 * N)
        h = pt.pt_create_ex(p)
        times = []
        for rep in range(args.warmup + 2):
            pt.pt_sync(h)
            t0 = time.perf_counter()
            pt.pt_set_positions(h, x0)
            pt.pt_sweep(h, SW, XE)
            pt.pt_energies(h)
            pt.pt_histograms(h)
            pt.pt_get_positions(h)
            times.append(time.perf_counter() - t0)
        kern = pt.pt_get_sweep_kernel(h)
        pt.pt_destroy(h)
        t_gpu = min(times[args.warmup:])
        t_cpu = cpu_per_rep * n_r
        rows.append({"n_r": n_r, "t_gpu_s": t_gpu, "t_cpu_1core_s": t_cpu, "S_p": t_cpu / t_gpu})
    best = max(rows, key=lambda r: r["S_p"])
    line = {"metric": "speed-up S_p = single-core FP64 oracle time / GPU time", "value": best["S_p"], "unit": "x",
            "n_gpus": 1, "steps": 2, "warmup": args.warmup, "higher_is_better": True,
            "vs_baseline": best["S_p"] / 130.0, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper protocol: N=55, 4000 sweeps per replica, exchange every 1000 sweeps, "
                                   "T geometric 0.2-3.0, n_r = 1..960; GPU time includes the host<->device copies",
                       "best_n_r": best["n_r"], "sweep_kernel": KERNEL_NAMES.get(kern, str(kern)),
                       "per_n_r": rows,
                       "baseline_note": "vs_baseline divides by the paper's best S_p (130x, GTX480 vs one "
                                        "Xeon E5620 core, its own CPU code): context, not a like-for-like ratio"},
            "cpu_baseline": {"value": SW * N / cpu_per_rep, "unit": "updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n_s} replicas x {SW} sweeps, exchange every {XE}, FP64 oracle, 1 thread"}}
    print(json.dumps(line), flush=True)
    return 0


def run_reweight(args):
    """Multiple-histogram reweighting of one ensemble's histograms (64 slots x 4096 bins from a
    GPU run of the N = 100 chain) into C_V(T) and <r_gyr^2>(T) at 400 temperatures: the
    library's host implementation against the FP64 oracle on the same input."""
    import numpy as np
    import oracle.wham as W
    from paper_1107_3490_gb300 import inputs, pt
    R, N, nb = 64, 100, 4096
    T = inputs.temperature_ladder(T_MIN, T_MAX, R)
    e_min, e_max = -8.0 * N, 2.0 * N
    p, keep = pt.make_params(N, T, 1, init_positions=inputs.random_coil(N, R, 1), n_bins=nb, n_therm=2000)
    h = pt.pt_create_ex(p)
    pt.pt_sweep(h, 20000, 1)
    H = pt.pt_histograms(h).reshape(R, nb)
    rg, _ = pt.pt_obs_histograms(h, R * nb)
    pt.pt_destroy(h)
    Tq = np.linspace(T_MIN, T_MAX, 400)
    cnt, osum = H.sum(0), rg.reshape(R, nb).sum(0)

    def native():
        g, f, it = pt.pt_wham(T, H, e_min, e_max, tol=1e-10, max_iter=500000)
        return pt.pt_wham_canonical(g, e_min, e_max, Tq, osum, cnt), it

    def orc():
        g, f, it = W.wham(T, H, e_min, e_max, tol=1e-10, max_iter=500000)
        return W.canonical(g, e_min, e_max, Tq, osum, cnt), it

    native()
    t0 = time.perf_counter()
    c_n, it = native()
    t_n = time.perf_counter() - t0
    t0 = time.perf_counter()
    c_o, _ = orc()
    t_o = time.perf_counter() - t0
    line = {"metric": "multiple-histogram reweighting time", "value": 1e3 * t_n, "unit": "ms", "n_gpus": 0,
            "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{R} slots x {nb} bins (N={N} chain, 20000 sweeps on the GPU), {it} fixed-point "
                                   f"iterations to max|df| < 1e-10, canonical C_V and <r_gyr^2> at 400 temperatures",
                       "host_threads": os.cpu_count(),
                       "max_rel_diff_vs_oracle": float(np.nanmax(np.abs(c_n - c_o) / (np.abs(c_o) + 1e-300)))},
            "cpu_baseline": {"value": 1e3 * t_o, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": "the same histograms through the numpy FP64 oracle"}}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_rate(N, R, T, seed, sweeps, threads, xe=1, ens_id=0):
    """Oracle single-bead updates/s of one ensemble (N, R) over `sweeps` sweeps."""
    import oracle
    from paper_1107_3490_gb300 import inputs
    ens = oracle.OracleEnsemble(inputs.random_coil(N, R, seed, ens_id), T, seed, ensemble_id=ens_id,
                                n_bins=1024, e_min=-8.0 * N, e_max=2.0 * N, threads=threads)
    t0 = time.perf_counter()
    ens.run(sweeps, xe)
    return R * N * sweeps / (time.perf_counter() - t0)


def _gpu_rate(specs, sweeps, warm=20):
    """GPU single-bead updates/s and FP32 flops/s of one batched context over `sweeps` sweeps
    (autotuned kernel, exchange every sweep)."""
    from paper_1107_3490_gb300 import inputs, pt
    made = [pt.make_params(N, inputs.temperature_ladder(tl, th, R), seed, ensemble_id=e,
                           init_positions=inputs.random_coil(N, R, seed, e), n_bins=1024, recompute_every=1000)
            for (N, R, tl, th, seed, e) in specs]
    h = pt.pt_create_batch([p for p, _ in made])
    pt.pt_sweep(h, warm, 1)
    kern = pt.pt_autotune(h, max(4, min(100, sweeps // 4)), force=True)
    pt.pt_sweep(h, 4, 1)
    pt.pt_sync(h)
    t0 = time.perf_counter()
    pt.pt_sweep(h, sweeps, 1)
    pt.pt_sync(h)
    dt = time.perf_counter() - t0
    pt.pt_destroy(h)
    upd = sum(N * R for (N, R, *_) in specs) * sweeps
    flops = sum(N * R * 30 * (N - 1) for (N, R, *_) in specs) * sweeps
    return upd / dt, flops / dt, KERNEL_NAMES.get(kern, str(kern))


def run_table(args):
    """Oracle (all host cores and one core, bounded samples) and GPU single-bead updates/s for
    the five configurations: plain N=30 x 16; N=100 x 64 x 4 ensembles; N=300 and N=1000 x 128;
    256 uneven ensembles; the served job stream (run through the job server)."""
    import numpy as np
    from paper_1107_3490_gb300 import inputs
    cores = os.cpu_count() or 1
    peak = fp32_peak_tflops(152, 2070.0) * 1e12
    rows = []

    def add(name, gpu, flops, kern, orc_all, orc_1, sample, extra=None):
        row = {"config": name, "gpu_updates_s": gpu, "fp32_peak_frac": flops / peak, "sweep_kernel": kern,
               "oracle_updates_s_all_cores": orc_all, "oracle_updates_s_1core": orc_1, "oracle_sample": sample}
        if extra:
            row.update(extra)
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)

    T30 = inputs.temperature_ladder(0.3, 3.0, 16)
    g, f, k = _gpu_rate([(30, 16, 0.3, 3.0, 1, 0)], 1000)
    add("1 plain N=30 x 16 replicas, T 0.3-3.0, 1000 sweeps", g, f, k,
        _oracle_rate(30, 16, T30, 1, 1000, cores), _oracle_rate(30, 16, T30, 1, 300, 1), "full run / 300 sweeps")
    T100 = inputs.temperature_ladder(0.2, 3.0, 64)
    g, f, k = _gpu_rate([(100, 64, 0.2, 3.0, s, s - 1) for s in range(1, 5)], 1000)
    add("2 N=100 x 64 replicas x 4 ensembles, T 0.2-3.0", g, f, k,
        _oracle_rate(100, 64, T100, 1, 400, cores), _oracle_rate(100, 64, T100, 1, 30, 1),
        "ensemble seed 1: 400 sweeps / 30 sweeps")
    T128 = inputs.temperature_ladder(0.2, 3.0, 128)
    for N, sw, so_all, so_1 in ((300, 200, 40, 3), (1000, 40, 4, 1)):
        g, f, k = _gpu_rate([(N, 128, 0.2, 3.0, 1, 0)], sw)
        add(f"3 N={N} x 128 replicas, T 0.2-3.0", g, f, k, _oracle_rate(N, 128, T128, 1, so_all, cores),
            _oracle_rate(N, 128, T128, 1, so_1, 1), f"prefix: {so_all} sweeps / {so_1} sweeps")
    specs = inputs.batched_ensembles(256)
    g, f, k = _gpu_rate([(sp.n_beads, sp.n_replicas, 0.2, 3.0, sp.seed, sp.ensemble_id) for sp in specs], 100)
    o_all = [_oracle_rate(sp.n_beads, sp.n_replicas, sp.temperatures(), sp.seed, 10, cores, ens_id=sp.ensemble_id)
             for sp in specs[:8]]
    o_one = [_oracle_rate(sp.n_beads, sp.n_replicas, sp.temperatures(), sp.seed, 3, 1, ens_id=sp.ensemble_id)
             for sp in specs[:8]]
    w = np.array([sp.n_beads * sp.n_replicas for sp in specs[:8]], dtype=float)
    hm = lambda r: float(w.sum() / np.sum(w / np.array(r)))  # updates over time of the sample
    add("4 batched 256 uneven ensembles (N 20-500, 8-64 replicas)", g, f, k, hm(o_all), hm(o_one),
        "first 8 ensembles: 10 sweeps / 3 sweeps each")
    jobs = inputs.served_jobs(4, s_lo=100, s_hi=1000)
    o_all = [_oracle_rate(j.n_beads, j.n_replicas, j.temperatures(), j.seed, 5, cores, ens_id=j.ensemble_id) for j in jobs]
    o_one = [_oracle_rate(j.n_beads, j.n_replicas, j.temperatures(), j.seed, 2, 1, ens_id=j.ensemble_id) for j in jobs]
    w = np.array([j.n_beads * j.n_replicas for j in jobs], dtype=float)
    rows.append({"config": "5 served job stream (oracle only; GPU: --workload served)",
                 "oracle_updates_s_all_cores": float(w.sum() / np.sum(w / np.array(o_all))),
                 "oracle_updates_s_1core": float(w.sum() / np.sum(w / np.array(o_one))),
                 "oracle_sample": "first 4 jobs of the stream: 5 sweeps / 2 sweeps each"})
    line = {"metric": "single-bead updates/s per configuration (GPU and FP64 oracle)", "unit": "updates/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "configurations 1-4; the served stream has its own workload (--workload served)",
                       "host_cores": cores, "fp32_peak_tflops": peak / 1e12},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=["long", "paper-scale", "batched", "served", "paper", "reweight", "table"],
                    default="long",
                    help="long: the benchmark line (N=1000 x 128 replicas); paper-scale: N=100 x 64 replicas x 4 "
                         "ensembles; batched / served: the uneven-ensemble and job-stream forms; "
                         "paper: the paper's S_p protocol; reweight: histogram reweighting time; "
                         "table: GPU and oracle rates of the five configurations")
    ap.add_argument("--jobs", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=12.0)
    ap.add_argument("--s-lo", dest="s_lo", type=int, default=100)
    ap.add_argument("--s-hi", dest="s_hi", type=int, default=10000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4, 5, 6],
                    help="sweep kernel: -1 autotune (default), 0 warp per replica, 1 lookahead groups, "
                         "2 team of warps, 3 warp per move of a group, 4 chain in registers, 5 groups of moves, "
                         "6 CTA-wide groups of moves")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    from paper_1107_3490_gb300 import build
    build.build()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "paper":
        return run_paper(args)
    if args.workload == "reweight":
        return run_reweight(args)
    if args.workload == "table":
        return run_table(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
