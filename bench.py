"""Throughput of the population-annealing hot path on GB300 (arXiv:2102.06611, Sec. II).

Workload (default): 2D Ising, L = 64 periodic, R = 10^6 replicas (512 B each, packed,
double-buffered), 301 temperatures beta = i / 300, theta = 10 checkerboard Metropolis
sweeps per temperature, nearest-integer resampling, seed 7 (seed 7 + rank on rank > 0).
One bench step = one temperature step of the method: resampling (table, copy numbers,
prefix sum, tree-ordered copy), theta sweeps with the fused measurement, and the step-4
record (families, observables) written on the device.

Metric: Metropolis spin-flip attempts per ns, attempts = N * R_i * theta summed over the
timed steps, R_i read back from the device records after the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

L_DEFAULT, R_DEFAULT, THETA, N_TEMPS, SEED = 64, 1_000_000, 10, 301, 7
METRIC = "Metropolis flips/ns on 1 GB300"
UNIT = "attempts/ns"
KERNELS_PER_STEP = 8  # k_table, k_counts, k_scan, k_copy, k_zero_measure, k_sweep, k_families, k_obs

# Integer roofline of the sweep kernel.  Peak: 152 SMs x 4 partitions x 32 lanes issue 128
# 32-bit integer operations per clock per SM.  Algorithmic 32-bit integer operations per
# attempt of the bit-plane Metropolis step, per 32-site word: 2 Philox4x32-10 calls for 8 bit
# planes (each call 20 widening multiplies counted as 2 ops and 20 three-input XORs: 60 ops),
# 8 planes x 3 ops of the borrow-chain comparison (threshold-bit select, majority, tie
# update), 15 ops of neighbour classes and update; plus one 62-op low-bits draw for the 2^-8
# of sites whose top 8 bits tie with the threshold.
SMS = 152
INT_OPS_PER_SM_CLK = 128.0
OPS_PER_ATTEMPT = (2 * 60 + 8 * 3 + 15) / 32 + 62 / 256
# DRAM bytes per attempt of k_sweep<64> from one ncu capture; None until the current kernel
# has been captured.
SWEEP64_DRAM_BYTES_PER_ATTEMPT = (135.497472e6 + 76.767744e6) / (262144 * 4096 * 10)


def _parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=297)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--L", type=int, default=L_DEFAULT)
    p.add_argument("--R", type=int, default=R_DEFAULT)
    p.add_argument("--theta", type=int, default=THETA)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-schedule-eval", action="store_true")
    p.add_argument("--no-batch-eval", action="store_true",
                   help="skip the bounded 64-run batch figure of the default line")
    p.add_argument("--no-whole-anneal", action="store_true",
                   help="skip the whole-anneal end-to-end figure of the default line")
    p.add_argument("--schedule-arm", choices=["plain", "rule", "learned"], default=None,
                   help="only one whole anneal of the schedule comparison (L=128, R=2e5, seed 1), for profiling")
    p.add_argument("--parallel", choices=["independent", "shard"], default="independent",
                   help="N > 1 ranks: independent populations (default) or one population sharded over the "
                        "ranks by slot ranges")
    p.add_argument("--shards", type=int, default=1,
                   help="--parallel shard: shards held by each rank (several shards of one population on one "
                        "GPU measure the protocol's cost)")
    p.add_argument("--workload", choices=["single", "batch"], default="single",
                   help="single: the L=64, R=1e6 run (default); batch: 64 mixed independent runs")
    p.add_argument("--update", choices=["metropolis", "heatbath"], default="metropolis",
                   help="spin update of the single-run workload (the headline metric is Metropolis)")
    p.add_argument("--resample", choices=["nearest", "poisson", "multinomial"], default="nearest",
                   help="resampling of the single-run workload (the headline metric is nearest-integer)")
    p.add_argument("--batch-steps", type=int, default=0,
                   help="batch workload: temperature steps to run (0: every run to completion)")
    p.add_argument("--no-sequential", action="store_true",
                   help="batch workload: skip the one-after-another comparison")
    p.add_argument("--batch-homog", default=None, metavar="L,R,N",
                   help="batch workload: N runs of one size L, R replicas each, 301 temperatures, theta 10, "
                        "seeds 100.. (profiling; the default is the 64 mixed runs)")
    p.add_argument("--batch-shape", default=None, metavar="UNIFIED,BPS,SCALE",
                   help="batch workload: fix the sweep phase's shape instead of the autotuner's choice")
    return p.parse_args()


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 50):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms",
                 str(self.interval_ms),
                 "-i", str(self.gpu)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------ oracle timing
def oracle_rate(L: int, R_sample: int, steps: int, theta: int, seed: int):
    """The CPU oracle as it stands on one host core: attempts / ns over `steps` temperature
    steps of a population of R_sample replicas (the per-attempt cost does not depend on R)."""
    import oracle
    pa = oracle.PA(L, R_sample, seed)
    pa.init()
    attempts = 0
    t0 = time.perf_counter()
    for i in range(1, steps + 1):
        pa.resample(i / (N_TEMPS - 1))
        pa.sweep(theta)
        attempts += L * L * pa.R * theta
        pa.observables()
    dt = time.perf_counter() - t0
    return attempts / (dt * 1e9), attempts, dt


def _oracle_worker(job):
    L, R_sample, steps, theta, seed = job
    _, att, dt = oracle_rate(L, R_sample, steps, theta, seed)
    return att, dt


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def cpu_baseline(L: int, theta: int) -> dict:
    """The oracle as it stands on the host: one core, and every core of the process's affinity
    set running its own oracle population (a replica-parallel split of the same workload:
    the per-attempt cost does not depend on R).  Worker processes are started with spawn."""
    import multiprocessing as mp
    R_sample, steps = 1000, 6
    v1, att1, dt1 = oracle_rate(L, R_sample, steps, theta, SEED)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(L, R_sample, steps, theta, SEED + 1 + c) for c in range(cores)])
    att_all = sum(a for a, _ in res)
    dt_all = max(d for _, d in res)
    model = cpu_model()
    return {"value": att_all / (dt_all * 1e9), "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": model,
            "sample": f"L={L}, {cores} independent oracle populations of R={R_sample} (one per core, "
                      f"spawned processes), {steps} temperature steps beta=i/300, theta={theta}: "
                      f"{att_all:.3g} attempts, slowest worker {dt_all:.1f} s",
            "single_core": {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": model,
                            "sample": f"L={L}, R={R_sample}, {steps} temperature steps beta=i/300, theta={theta}: "
                                      f"{att1:.3g} attempts in {dt1:.1f} s (single-threaded C oracle)"}}


# ------------------------------------------------------------------------------ schedules
SCHED_L, SCHED_R, SCHED_SEEDS, SCHED_TARGET = 128, 200_000, (1, 2, 3, 4), 1e-4


SCHED_MODES = ("plain", "rule", "learned")


def schedule_eval(dev) -> dict:
    """Second half of the metric: wall time of a whole anneal (beta 0 -> 1, L=128, R=2e5) with
    the plain adaptive schedule (overlap bisection at 0.8, theta = 10), with the same bisection
    plus the measured-decorrelation rule for theta and no network ("rule", the ablation of the
    network), and with the learned one, and each run's free-energy deviation per spin at
    beta = 1 from the exact finite-lattice value (Kaufman's closed form,
    tests/golden/exact_lnZ.json); seeds 1-4."""
    import torch

    from paper_2102_06611_gb300 import PopulationAnnealing
    from paper_2102_06611_gb300.learned import ScheduleMLP, anneal
    from paper_2102_06611_gb300.train_schedule import DEFAULT_WEIGHTS

    with open(os.path.join(ROOT, "tests", "golden", "exact_lnZ.json")) as f:
        exact = json.load(f)["lnZ"][str(SCHED_L)]["1.0"]
    model = ScheduleMLP.load(DEFAULT_WEIGHTS, device=dev)
    out = {"L": SCHED_L, "R": SCHED_R, "seeds": list(SCHED_SEEDS), "target_abs_dbetaf_per_spin": SCHED_TARGET,
           "exact_lnZ_beta1": exact, "runs": []}
    for seed in SCHED_SEEDS:
        run = {"seed": seed}
        for mode in SCHED_MODES:
            pa = PopulationAnnealing(SCHED_L, SCHED_R, seed, device=dev)
            r = anneal(pa, mode, model)
            r["abs_dbetaf_per_spin"] = abs(r["minus_betaF"] - exact) / (SCHED_L * SCHED_L)
            r["reached_target"] = r["abs_dbetaf_per_spin"] <= SCHED_TARGET
            run[mode] = {k: r[k] for k in ("wall_s", "steps", "sweeps", "fallbacks", "extensions",
                                           "abs_dbetaf_per_spin", "reached_target")}
            pa.close()
            del pa
            torch.cuda.empty_cache()
        run["speedup"] = run["plain"]["wall_s"] / run["learned"]["wall_s"]
        run["speedup_over_rule"] = run["rule"]["wall_s"] / run["learned"]["wall_s"]
        out["runs"].append(run)
    for mode in SCHED_MODES:
        out[mode + "_wall_s_total"] = sum(r[mode]["wall_s"] for r in out["runs"])
        out[mode + "_sweeps_total"] = sum(r[mode]["sweeps"] for r in out["runs"])
        out[mode + "_reached_target"] = sum(bool(r[mode]["reached_target"]) for r in out["runs"])
    out["speedup"] = out["plain_wall_s_total"] / out["learned_wall_s_total"]
    out["speedup_over_rule"] = out["rule_wall_s_total"] / out["learned_wall_s_total"]
    return out


# ------------------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2102_06611_gb300 import OBS_BYTES, PopulationAnnealing, pa_obs

    L, R, theta = args.L, args.R, args.theta
    N = L * L
    K, W = args.steps, args.warmup
    assert W + K <= N_TEMPS - 1, "schedule has 300 steps"
    stream = torch.cuda.current_stream(dev)
    from paper_2102_06611_gb300.multi import rank_seed
    pa = PopulationAnnealing(L, R, rank_seed(SEED, rank), device=dev, stream=stream, update=args.update,
                             resample=args.resample)
    records = torch.zeros((K, (OBS_BYTES + 7) // 8), dtype=torch.int64, device=dev)

    def beta(i):
        return i / (N_TEMPS - 1)

    for i in range(1, W + 1):
        pa.resample(beta(i))
        pa.anneal_step(theta)
        pa.record(records[0])
    torch.cuda.synchronize()

    sw_start = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    sw_end = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    t_start.record(stream)
    for s in range(K):
        i = W + 1 + s
        pa.resample(beta(i))
        sw_start[s].record(stream)
        pa.anneal_step(theta)
        sw_end[s].record(stream)
        pa.record(records[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    sweep_ms = sum(a.elapsed_time(b) for a, b in zip(sw_start, sw_end))

    recs = records.cpu().numpy()
    import ctypes
    Rs = []
    for s in range(K):
        o = pa_obs.from_buffer_copy(recs[s].tobytes()[: ctypes.sizeof(pa_obs)])
        assert o.status == 0, f"device error {o.status}"
        Rs.append(o.R)
    attempts = float(N) * float(sum(Rs)) * theta

    # end to end through the public API with host results, over the same temperature steps of
    # a second run with the same seed: each step reads its record (pa_obs, D2H) and
    # synchronises
    pa.close()
    del pa
    pa2 = PopulationAnnealing(L, R, rank_seed(SEED, rank), device=dev, stream=stream, update=args.update,
                              resample=args.resample)
    for i in range(1, W + 1):
        pa2.resample(beta(i))
        pa2.anneal_step(theta)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_att = 0.0
    ev0.record(stream)
    for s in range(K):
        i = W + 1 + s
        pa2.resample(beta(i))
        pa2.anneal_step(theta)
        o = pa2.observables()
        e2e_att += float(N) * o["R"] * theta
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ev0.elapsed_time(ev1)
    e2e = {"value": e2e_att / (e2e_ms * 1e6), "unit": UNIT, "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": ctypes.sizeof(pa_obs), "steps": K,
           "note": "public API per step: pa_resample(beta) + pa_anneal_step(theta) + pa_observables "
                   "(host record, synchronising); beta passes by value, no input tensor is copied"}
    pa2.close()
    del pa2
    torch.cuda.empty_cache()
    whole = None if args.no_whole_anneal else whole_anneal_e2e(args, dev, stream, rank)

    from paper_2102_06611_gb300.multi import aggregate
    ms, sweep_ms, attempts = aggregate(ms, sweep_ms, attempts, device=dev)

    pc = philox_ceiling(dev, stream)
    if rank == 0:
        value = attempts / (ms * 1e6)
        sweep_rate = (attempts / world) / (sweep_ms * 1e6)
        f_mhz = clk["sm_mhz"] or 2070.0
        peak_tops = SMS * INT_OPS_PER_SM_CLK * f_mhz * 1e6 / 1e12           # int32 Tops/s
        achieved_tops = sweep_rate * 1e9 * OPS_PER_ATTEMPT / 1e12
        traffic = (SWEEP64_DRAM_BYTES_PER_ATTEMPT * attempts / world / K
                   if (L == 64 and SWEEP64_DRAM_BYTES_PER_ATTEMPT) else None)
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": K,
            "warmup": W,
            "ms_per_step": ms / K,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u32",
            "data": "synthetic (simple sampling at beta=0, Philox4x32-10 seed 7+rank)",
            "config": {"workload": f"2D Ising PA L={L} R={R} theta={theta} beta=i/300 {args.resample}"
                                   + ("" if args.update == "metropolis" else f" {args.update}"),
                       "L": L, "R": R, "theta": theta, "temperatures": N_TEMPS, "resampling": args.resample,
                       "update": args.update,
                       "parallelism": f"independent runs x{world}" if world > 1 else "single run",
                       "beta_timed": [beta(W + 1), beta(W + K)],
                       "l2": "inputs larger than L2 (2 x %.0f MB spin buffers)" % (R * L * 2 * 4 / 1e6)},
            "roofline": {"bound": "alu", "kernel": f"k_sweep<{L}>", "achieved": sweep_rate,
                         "peak": pc["attempts_per_ns"], "unit": "attempts/ns",
                         "frac": sweep_rate / pc["attempts_per_ns"],
                         "peak_basis": "measured Philox4x32-10 rate alone on this GPU (pa_philox_xor, the "
                                       "sweep's round code, every SM filled) x 16 attempts per call: the "
                                       "generator's share of the bit-plane Metropolis step alone",
                         "traffic": traffic,
                         "traffic_unit": "DRAM bytes per launch (ncu, scaled from R=262144 by attempts)",
                         "philox_ceiling": pc,
                         "dispatch_peak": {"achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s (int32)",
                                           "frac": achieved_tops / peak_tops, "ops_per_attempt": OPS_PER_ATTEMPT,
                                           "peak_attempts_per_ns": peak_tops * 1e3 / OPS_PER_ATTEMPT,
                                           "basis": "152 SM x 128 int32 ops/clk/SM x median SM clock "
                                                    "(sampled); algorithmic ops per attempt of the "
                                                    "bit-plane Metropolis step"}},
            "sweep_share": sweep_ms / ms,
            "clocks": clk,
            "gpu_launches": KERNELS_PER_STEP * K,
            "wall_s": wall,
        }
        if e2e:
            line["e2e"] = e2e
        if whole:
            line["e2e_whole_anneal"] = whole
        if not args.no_batch_eval and world == 1:
            line["batch_c4"] = batch_eval(dev, BATCH_EVAL_STEPS, True)
        if not args.no_schedule_eval and world == 1:
            line["learned_schedule"] = schedule_eval(dev)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(L, theta)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


BATCH_EVAL_STEPS = 20


def whole_anneal_e2e(args, dev, stream, rank: int) -> dict:
    """One whole anneal through the public API, timed end to end on the host clock: pa_init
    from the seed (buffers included), all 300 temperature steps (pa_resample, pa_anneal_step,
    pa_observables with its host record every step), and the final host readback of the level
    histogram."""
    import ctypes

    import torch

    from paper_2102_06611_gb300 import PopulationAnnealing, pa_obs
    from paper_2102_06611_gb300.multi import rank_seed

    L, R, theta = args.L, args.R, args.theta
    N = L * L
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.2)
    t0 = time.perf_counter()
    pa = PopulationAnnealing(L, R, rank_seed(SEED, rank), device=dev, stream=stream, update=args.update,
                             resample=args.resample)
    att = 0.0
    for i in range(1, N_TEMPS):
        pa.resample(i / (N_TEMPS - 1))
        pa.anneal_step(theta)
        att += float(N) * pa.observables()["R"] * theta
    hist = pa.histogram()
    dt = time.perf_counter() - t0
    clk = clocks.stop()
    assert int(hist.sum()) == pa.R
    pa.close()
    del pa
    torch.cuda.empty_cache()
    steps = N_TEMPS - 1
    return {"value": att / (dt * 1e9), "unit": UNIT, "wall_s": dt, "steps": steps,
            "h2d_bytes_per_step": 0, "d2h_bytes_per_step": ctypes.sizeof(pa_obs),
            "d2h_bytes_final": 4 * (N + 1), "clocks": clk,
            "note": "host clock: buffers + pa_init (simple sampling on the GPU) + 300 x (pa_resample, "
                    "pa_anneal_step, pa_observables) + final histogram readback; the configuration and "
                    "beta pass by value, so no input array is copied"}


def philox_ceiling(dev, stream) -> dict:
    """The rate of Philox4x32-10 calls alone on this GPU (pa_philox_xor: the sweep's round code,
    every SM filled), and the sweep rate it allows: 2 calls give the bit planes of 32 attempts."""
    import ctypes

    import torch

    from paper_2102_06611_gb300 import _lib
    lib = _lib.lib()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    n, calls = sms * 2048, 2048
    out = torch.empty(n, dtype=torch.int32, device=dev)
    ms = []
    for rep in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        assert lib.pa_philox_xor(7, n, calls, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream)) == _lib.PA_OK
        e1.record(stream)
        torch.cuda.synchronize()
        if rep > 0:
            ms.append(e0.elapsed_time(e1))
    best = min(ms)
    rate = n * calls / (best * 1e6)
    return {"kernel": "pa_philox_xor", "calls_per_ns": rate, "attempts_per_ns": 16 * rate,
            "basis": f"{n} threads x {calls} Philox4x32-10 calls, best of 5 (CUDA events); "
                     "2 calls = the 8 bit planes of 32 attempts"}


# ------------------------------------------------------------------------------ reference arm
def _reference_worker(job):
    """One host core: the oracle population of one worker for W untimed and K timed steps."""
    L, theta, R_sample, seed, W, K = job
    import oracle
    pa = oracle.PA(L, R_sample, seed)
    pa.init()
    for i in range(1, W + 1):
        pa.resample(i / (N_TEMPS - 1))
        pa.sweep(theta)
    att = 0
    t0 = time.perf_counter()
    for s in range(K):
        pa.resample((W + 1 + s) / (N_TEMPS - 1))
        pa.sweep(theta)
        pa.observables()
        att += L * L * pa.R * theta
    return att, time.perf_counter() - t0


def run_reference(args):
    """The CPU oracle as it stands, timed on the host: the benchmark's reference arm.  Every
    core of the process's affinity set runs its own oracle population (spawned processes, a
    replica-parallel split of the workload); the rate is the summed attempts over the slowest
    worker's time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    L, theta = args.L, args.theta
    R_sample = 120
    W, K = args.warmup, args.steps
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_reference_worker, [(L, theta, R_sample, SEED + c, W, K) for c in range(cores)])
    att = sum(a for a, _ in res)
    dt = max(d for _, d in res)
    v = att / (dt * 1e9)
    sample = (f"L={L}, {cores} oracle populations of R={R_sample} (one per core; a bounded sample of the "
              f"R={args.R} population), theta={theta}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": K,
        "warmup": W, "ms_per_step": dt * 1e3 / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i8", "data": "synthetic",
        "config": {"workload": f"2D Ising PA L={L} R={args.R} theta={theta} beta=i/300 nearest-integer",
                   "L": L, "R": args.R, "theta": theta},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def batch_eval(dev, steps: int = 0, sequential: bool = True, homog: str | None = None,
               shape: str | None = None) -> dict:
    """64 independent runs (mixed L, R, temperature count, theta), batched (one graph replay per
    temperature step) and, for comparison, the same runs one after another through the
    single-run API; `steps` > 0 bounds both to the first `steps` temperature steps.  `homog`
    ("L,R,N") replaces the mix by N runs of one size; `shape` ("UNIFIED,BPS,SCALE") fixes the
    sweep phase's shape."""
    import ctypes

    import torch

    from paper_2102_06611_gb300 import OBS_BYTES, PopulationAnnealing, pa_obs
    from paper_2102_06611_gb300.batch import Batch, RunSpec, mixed_runs

    if homog:
        hL, hR, hN = (int(x) for x in homog.split(","))
        specs = [RunSpec(hL, hR, 100 + i, N_TEMPS, THETA) for i in range(hN)]
        what = f"{hN} independent runs of L={hL}, R={hR}, {N_TEMPS} temperatures, theta {THETA}, seeds 100-{99 + hN}"
    else:
        specs = mixed_runs()
        what = ("64 independent runs: L in {8..64}, R log-uniform [1e3, 2e5], 51-301 temperatures, "
                "theta in {1, 5, 10}, seeds 100-163")
    n = len(specs)
    total_steps = max(s.n_temps for s in specs) - 1
    steps = min(total_steps, steps) if steps > 0 else total_steps
    words = (OBS_BYTES + 7) // 8
    b = Batch(specs, device=dev)
    if shape:
        b.set_shape(*(int(x) for x in shape.split(",")))
    rec = torch.zeros((steps, n, words), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for s in range(steps):
        b.step()
        b.record(rec[s])
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    recs = rec.cpu().numpy()
    attempts = 0.0
    for s in range(steps):
        for r in range(n):
            o = pa_obs.from_buffer_copy(recs[s, r].tobytes()[: ctypes.sizeof(pa_obs)])
            if o.step == s + 1:
                assert o.status == 0, f"run {r}: device error {o.status}"
                attempts += float(specs[r].L ** 2) * o.R * specs[r].theta
    tuning = b.tuning()
    b.close()
    del b
    torch.cuda.empty_cache()
    ms_seq = None
    if sequential:
        ctxs = [PopulationAnnealing(sp.L, sp.R, sp.seed, device=dev) for sp in specs]
        torch.cuda.synchronize()
        t0.record(stream)
        for sp, pa in zip(specs, ctxs):
            for i in range(1, min(sp.n_temps, steps + 1)):
                pa.resample(i / (sp.n_temps - 1))
                pa.anneal_step(sp.theta)
        t1.record(stream)
        torch.cuda.synchronize()
        ms_seq = t0.elapsed_time(t1)
        for pa in ctxs:
            pa.close()
        del ctxs
        torch.cuda.empty_cache()
    return {"value": attempts / (ms * 1e6), "unit": UNIT, "runs": n, "steps": steps,
            "steps_bounded": steps < total_steps, "batch_ms": ms, "attempts": attempts,
            "workload": what + (f"; first {steps} temperature steps of every run" if steps < total_steps else ""),
            "sequential_single_run": ({"value": attempts / (ms_seq * 1e6), "unit": UNIT, "ms": ms_seq}
                                      if ms_seq else None),
            "gain_over_sequential": ms_seq / ms if ms_seq else None, "tuning": tuning,
            "gpu_launches": 11 * steps}


def run_batch(args):
    """The batched workload alone (--workload batch)."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    r = batch_eval(dev, args.batch_steps, not args.no_sequential, args.batch_homog, args.batch_shape)
    what = f"{r['runs']} runs of one size" if args.batch_homog else "64 mixed runs"
    line = {"metric": METRIC + f" ({what}, batched)", "value": r["value"], "unit": UNIT,
            "n_gpus": 1, "steps": r["steps"], "warmup": 0, "ms_per_step": r["batch_ms"] / r["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": r["workload"], "runs": r["runs"]},
            "sequential_single_run": r["sequential_single_run"], "gain_over_sequential": r["gain_over_sequential"],
            "batch_ms": r["batch_ms"], "tuning": r["tuning"], "gpu_launches": r["gpu_launches"]}
    print(json.dumps(line), flush=True)


def run_sharded(args):
    """One population of R replicas split over world x --shards shards by contiguous slot ranges
    (NCCL between ranks, direct copies between shards of one rank); a step is the same
    temperature step as the default workload, for the whole population."""
    import ctypes

    import torch
    import torch.distributed as dist

    from paper_2102_06611_gb300 import OBS_BYTES, pa_obs
    from paper_2102_06611_gb300.shard import DistTransport, LocalTransport, ShardedRun, gpu_shards

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    L, R, theta, k = args.L, args.R, args.theta, max(1, args.shards)
    N = L * L
    P = world * k
    K, W = args.steps, args.warmup
    assert W + K <= N_TEMPS - 1, "schedule has 300 steps"
    transport = LocalTransport() if world == 1 else DistTransport(shards_per_rank=k)
    engines = gpu_shards(L, R, SEED, list(range(rank * k, (rank + 1) * k)), P, resample=args.resample,
                         update=args.update, device=dev, stream=stream)
    run = ShardedRun(engines, P, transport)
    first = engines[rank * k]
    records = torch.zeros((K, (OBS_BYTES + 7) // 8), dtype=torch.int64, device=dev)

    def beta(i):
        return i / (N_TEMPS - 1)

    for i in range(1, W + 1):
        run.resample(beta(i))
        run.anneal_step(theta)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(K):
        run.resample(beta(W + 1 + s))
        run.anneal_step(theta)
        first.record(records[s])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    recs = records.cpu().numpy()
    Rs = []
    for s in range(K):
        o = pa_obs.from_buffer_copy(recs[s].tobytes()[: ctypes.sizeof(pa_obs)])
        assert o.status == 0, f"device error {o.status}"
        Rs.append(o.R)
    attempts = float(N) * float(sum(Rs)) * theta  # the whole population's, the same on every rank
    from paper_2102_06611_gb300.multi import aggregate
    ms, _, _ = aggregate(ms, 0.0, 0.0, device=dev)
    if rank == 0:
        value = attempts / (ms * 1e6)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms / K, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic (simple sampling at beta=0, Philox4x32-10 seed 7)",
                "config": {"workload": f"2D Ising PA L={L} R={R} theta={theta} beta=i/300 {args.resample}"
                                       + ("" if args.update == "metropolis" else f" {args.update}"),
                           "L": L, "R": R, "theta": theta, "temperatures": N_TEMPS,
                           "parallelism": f"one population sharded by slot ranges: {P} shards "
                                          f"({k} per rank, {world} rank(s))",
                           "beta_timed": [beta(W + 1), beta(W + K)],
                           "l2": "inputs larger than L2 (%.0f MB of spins per shard)" % (R / P * L * 2 * 4 * 2 / 1e6)},
                "clocks": clk,
                "gpu_launches": (KERNELS_PER_STEP + 4 + (4 if args.resample == "multinomial" else 0)) * K * k}
        print(json.dumps(line), flush=True)
    for e in engines.values():
        e.close()
    if world > 1:
        dist.destroy_process_group()


def run_schedule_arm(args):
    """One whole anneal of one arm of the schedule comparison (L=128, R=2e5, seed 1)."""
    import torch

    from paper_2102_06611_gb300 import PopulationAnnealing
    from paper_2102_06611_gb300.learned import ScheduleMLP, anneal
    from paper_2102_06611_gb300.train_schedule import DEFAULT_WEIGHTS

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    model = ScheduleMLP.load(DEFAULT_WEIGHTS, device=dev)
    pa = PopulationAnnealing(SCHED_L, SCHED_R, SCHED_SEEDS[0], device=dev)
    r = anneal(pa, args.schedule_arm, model)
    pa.close()
    print(json.dumps({"arm": args.schedule_arm, "L": SCHED_L, "R": SCHED_R, "seed": SCHED_SEEDS[0],
                      **{k: r[k] for k in ("wall_s", "steps", "sweeps", "extensions", "fallbacks")}}), flush=True)


def main():
    args = _parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.schedule_arm:
        run_schedule_arm(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.parallel == "shard":
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
