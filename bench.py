"""Benchmark of the stochastic-LLG hysteresis-loop path on GB300.

Workload (a step): the full-resolution magnetite rod at b = 1 (8x24x56 = 10752 cells of
a0 = 0.839 nm), 256 noise realisations, T = 310 K, alpha = 0.1, dt = 2 fs, field swept
+-1500 Oe at 100 Oe/ns; one step advances all 256 rods by one sample interval (5000 Heun steps,
1 Oe of sweep) in one persistent launch of the resident engine and writes one M(H) sample per rod.
Inputs are synthetic (the rods start saturated along +z; the noise is Philox-generated).

Reported: cell-steps/s (value), loops/s, the plain one-launch-per-half-step engine on the same
workload, the small-rod (b = 4, 4 realisations) resident/plain ratio, an end-to-end figure through
the C ABI with host buffers, the roofline of the resident kernel, and the FP64 oracle timed on the
host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sLLG cell-steps/s and loops/s on 1 GB300 (batched vs plain); adjoint grads/s"
UNIT = "cell-steps/s"
WORKLOAD = "rod_b1_256real"
L2_BYTES = 129 * 1024 * 1024
SM_COUNT_NOMINAL = 152
ALU_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0
# Algorithmic 32-bit lane operations of one cell-step (FMA-fused count of the method's
# arithmetic: Philox4x32-10 98, uniforms 12, Box-Muller 20, two effective fields 40, two torques
# 30, predictor with renormalisation and accumulator 12, corrector with renormalisation 9).
ALU_OPS_PER_CELL_STEP = 221
# measured FP32 lane issue rate (lane-ops/s) of this run's GPU, set by run_ours
ALU_PEAK = {"value": None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the side measurements")
    ap.add_argument("--ladder-full", choices=["ci", "all"], default=None,
                    help="run every job of the uneven ladder to the end of its loop in batched "
                         "graph calls and print one JSON line (ci: without the b = 1 jobs at "
                         "10 Oe/ns); not part of the default benchmark")
    ap.add_argument("--profile-case", default=None,
                    help="run a small untimed case for a profiler (b1, b1-plain, b4, b4-rows, slab, "
                         "adjoint, tangent) and exit")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def realisation_offset(rank: int, n_real: int) -> int:
    """First noise key of a rank's ensemble: ranks simulate disjoint realisations."""
    return rank * n_real


def weak_scaling_value(local_seconds: float, cell_steps_per_rank: float, device="cpu"):
    """Whole-job throughput of a weak-scaling run: the cell-steps of all ranks divided by the
    slowest rank's time (a max-reduction of the timings, the only collective; no data moves
    between ranks).  Returns (value, max_seconds)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total = float(t.item())
    return cell_steps_per_rank * world / total, total


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: a temporary file, or LLG_BENCH_CLOCKS_DIR to keep them
        import tempfile
        out_dir = os.environ.get("LLG_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"llg_bench_clocks_gpu{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_grid(pkg, cfg, engine):
    from workloads import MAGNETITE as M
    g = pkg.Grid(*cfg["dims"], a0=M["a0"], b=cfg["b"], periodic=cfg.get("periodic", 0))
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"], T=M["T"])
    g.set_scaling(mode=cfg["mode"], Tc=M["Tc"])
    g.set_sweep(H_start=cfg["H_start"], H_turn=cfg["H_turn"], rate=cfg["rate"], dt=cfg["dt"],
                sample_dH=cfg["sample_dH"])
    g.set_engine(engine)
    return g


def timed_steps(torch, fn, K, W, flush):
    """W warm-up calls, then K calls each bracketed by CUDA events on the current stream, with an
    L2 flush (a write larger than L2) between calls outside the timed window."""
    st = torch.cuda.current_stream()
    for _ in range(W):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(K):
        flush.add_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    return times


def _oracle_problem(cfg):
    from oracle import oracle as O
    from workloads import MAGNETITE as M
    O.build()
    return O, O.material_problem(*cfg["dims"], a0=M["a0"], b=cfg["b"], A0=M["A0"], K0=M["K0"],
                                 Ms=M["Ms"], alpha=M["alpha"], T=M["T"], dt=cfg["dt"],
                                 mode=cfg["mode"], Tc=M["Tc"], H_start_Oe=cfg["H_start"],
                                 H_turn_Oe=cfg["H_turn"], rate_Oe_per_ns=cfg["rate"])


def _oracle_steps_for(O, p, cfg, n_real, threads, budget_s):
    """Heun steps of n_real rods that take about budget_s on the host cores (from a 20-step
    calibration run)."""
    m = O.uniform_state(n_real, p.ncells)
    t0 = time.perf_counter()
    O.run(p, m, seed=cfg["seed"], n_steps=20, threads=threads)
    per_step = (time.perf_counter() - t0) / 20
    return max(20, int(budget_s / max(per_step, 1e-9)))


def _oracle_timed(O, p, cfg, n_real, steps, threads):
    """Seconds of one oracle run of n_real rods from +z over `steps` Heun steps."""
    m = O.uniform_state(n_real, p.ncells)
    t0 = time.perf_counter()
    O.run(p, m, seed=cfg["seed"], n_steps=steps, threads=threads)
    return time.perf_counter() - t0


def cpu_oracle_rate(cfg, budget_s=12.0):
    """The FP64 oracle on the host cores on a bounded sample of the workload: rods of the same
    size, a short window of Heun steps.  Returns (cell-steps/s, threads, description)."""
    threads = os.cpu_count() or 1
    O, p = _oracle_problem(cfg)
    n_real = threads
    steps = _oracle_steps_for(O, p, cfg, n_real, threads, budget_s)
    el = _oracle_timed(O, p, cfg, n_real, steps, threads)
    rate = n_real * p.ncells * steps / el
    return rate, threads, (f"{n_real} b={cfg['b']} rods ({p.ncells} cells) x {steps} Heun steps "
                           f"from +z, FP64, {el:.1f} s")


# ------------------------------------------------------------------------------------------------
def run_reference(args):
    """--impl reference: the FP64 CPU oracle (the only other implementation of the method here)
    timed on the host cores.  A step is a bounded sample of the workload -- one rod per host
    thread over a fixed number of Heun steps, sized so the whole run takes a few minutes -- and
    the line reports what was measured: its time per step and its cell-steps/s.  The time the
    oracle would need for one full step of the GPU arm (256 rods x one sample interval) is
    extrapolated from that rate and labelled as such."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from workloads import CONFIGS
    cfg = CONFIGS[WORKLOAD]
    threads = os.cpu_count() or 1
    per_step_budget = max(2.0, min(20.0, 100.0 / max(1, args.steps + args.warmup)))
    O, p = _oracle_problem(cfg)
    n_real = threads
    heun = _oracle_steps_for(O, p, cfg, n_real, threads, per_step_budget)
    for _ in range(args.warmup):
        _oracle_timed(O, p, cfg, n_real, max(20, heun // 4), threads)
    secs = [_oracle_timed(O, p, cfg, n_real, heun, threads) for _ in range(args.steps)]
    total = sum(secs)
    ncell = math.prod(cfg["dims"])
    value = n_real * ncell * heun * args.steps / total
    steps_per_sample = round(cfg["sample_dH"] / (cfg["rate"] * 1e9 * cfg["dt"]))
    gpu_step_cells = cfg["n_real"] * ncell * steps_per_sample
    desc = (f"{n_real} b={cfg['b']} rods ({ncell} cells) x {heun} Heun steps from +z per step, FP64, "
            f"{total / args.steps:.1f} s per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "rods": n_real, "cells_per_rod": ncell,
                   "heun_steps_measured": heun,
                   "sample": "rods and steps measured per step (a bounded sample of the workload)",
                   "extrapolated": True,
                   "extrapolated_ms_per_full_step": 1e3 * gpu_step_cells / value,
                   "full_step": f"{cfg['n_real']} rods x {steps_per_sample} Heun steps",
                   "l2": "not applicable (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import paper_1912_00310_gb300 as pkg
    from workloads import CONFIGS

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    cfg = CONFIGS[WORKLOAD]
    n_real = cfg["n_real"]
    ncell = math.prod(cfg["dims"])
    g = make_grid(pkg, cfg, pkg.ENGINE_RESIDENT)
    S_per_step = g.sample_every  # Heun steps per bench step (one sample)
    # each rank simulates its own 256 realisations (keys offset by rank): weak scaling
    g.reset(seed=cfg["seed"], n_real=n_real, real_offset=realisation_offset(rank, n_real))
    samples = torch.zeros((n_real, g.n_samples), device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, device="cuda")

    def step():
        g.advance(S_per_step, samples)

    clocks = Clocks(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = timed_steps(torch, step, args.steps, args.warmup, flush)
    clk = clocks.stop()
    g.sync(600)
    local_total = sum(times)
    cells_per_step = n_real * ncell * S_per_step
    value, total = weak_scaling_value(local_total, cells_per_step * args.steps,
                                      device="cuda" if world > 1 else "cpu")
    if world > 1:
        torch.distributed.barrier()
    # one ensemble over all ranks: the sample columns written so far, summed over ranks (an
    # all-reduce of per-sample sums and sums of squares; outside the timed region)
    from paper_1912_00310_gb300 import ensemble
    k_done = args.warmup + args.steps
    cols = samples[:, 1:k_done + 1].float().cpu().numpy()
    n_tot, s1, s2 = ensemble.sample_moments(cols)
    mean_mz = s1 / n_tot
    se_mz = ((s2 - s1 * s1 / n_tot) / max(1, n_tot - 1) / n_tot) ** 0.5
    ens = {"realisations": n_tot, "samples": int(cols.shape[1]),
           "mean_mz_last": float(mean_mz[-1]), "se_mz_last": float(se_mz[-1]),
           "reduction": "per-sample sums over ranks (all-reduce), llg_loop_moments"}

    steps_per_loop = g.steps_per_loop
    loops_per_s = value / (ncell * steps_per_loop)
    launch_s = local_total / args.steps  # one persistent launch per step
    achieved = ALU_OPS_PER_CELL_STEP * cells_per_step / launch_s
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal = sm_count * ALU_LANES_PER_SM * MAX_SM_MHZ * 1e6
    # measured denominator: the FP32 lanes' issue rate on this GPU (outside the timed region)
    alu = pkg.measure_alu_peak(dev)
    peak = alu["ffma_lane_ops_per_s"]
    ALU_PEAK["value"] = peak

    extra = {}
    if not args.quick:
        extra = side_measurements(args, torch, pkg, cfg, g, samples, S_per_step, flush)
        local_rate = cells_per_step * args.steps / local_total
        extra["plain_same_workload"]["resident_over_plain"] = (
            local_rate / extra["plain_same_workload"]["value"])

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            r, threads, desc = cpu_oracle_rate(cfg)
            cpu = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rods_per_gpu": n_real, "cells_per_rod": ncell,
                       "heun_steps_per_step": S_per_step, "engine": "resident (plane-pipelined)",
                       "parallelism": f"replicas x{world} (independent realisations)",
                       "l2": "flushed between steps (write of 2x L2)"},
            "loops_per_s": loops_per_s,
            "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                         "unit": "Gop/s", "frac": achieved / peak, "traffic": measured_traffic(),
                         "traffic_unit": "bytes per launch (ncu dram read + write)",
                         "kernel": "rod_pipelined_nx_kernel<3, 8, 24, 56>",
                         "ops_per_cell_step": ALU_OPS_PER_CELL_STEP,
                         "peak_basis": "measured: FP32 FMA issue microbenchmark (llg_measure_alu_peak) "
                                       f"at {alu['ffma_sm_mhz']:.0f} MHz",
                         "int_mix_lane_ops_per_s": alu["int_lane_ops_per_s"] / 1e9,
                         "nominal_peak": nominal / 1e9,
                         "nominal_basis": f"{sm_count} SMs x {ALU_LANES_PER_SM} lanes x {MAX_SM_MHZ:.0f} MHz"},
            "clocks": clk,
            "gpu_launches": args.steps,
            "cpu_baseline": cpu,
            "ensemble": ens,
        }
        line.update(extra)
        print(json.dumps(line))
    g.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def side_measurements(args, torch, pkg, cfg, g, samples, S_per_step, flush):
    """End-to-end through the C ABI with host buffers, the plain engine on the same workload, and
    the small-rod resident/plain ratio."""
    import numpy as np
    out = {}
    n_real = cfg["n_real"]
    ncell = math.prod(cfg["dims"])
    # e2e: per step, the state goes host -> device, one sample interval runs, and the state and
    # the new sample come back to the host (pinned buffers)
    m_host = torch.empty((n_real, ncell, 3), dtype=torch.float32).pin_memory()
    s_host = torch.empty((n_real,), dtype=torch.float32).pin_memory()
    g.get_state(m_host)
    step_idx = [g.step]

    def e2e_step():
        g.set_state(m_host, step_idx[0])
        g.advance(S_per_step, samples)
        k = (step_idx[0] + S_per_step) // S_per_step
        s_host.copy_(samples[:, min(k, g.n_samples - 1)], non_blocking=True)
        g.get_state(m_host)  # synchronises
        step_idx[0] += S_per_step

    for _ in range(2):
        e2e_step()
    _, world, _ = dist_env()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    el = time.perf_counter() - t0
    # whole-job rate over all ranks: every rank's cell-steps over the slowest rank's time
    e2e_value, _ = weak_scaling_value(el, n_real * ncell * S_per_step * args.steps,
                                      device="cuda" if world > 1 else "cpu")
    out["e2e"] = {"value": e2e_value, "unit": UNIT,
                  "h2d_bytes_per_step": m_host.numel() * 4,
                  "d2h_bytes_per_step": m_host.numel() * 4 + s_host.numel() * 4}
    # plain engine on the same b = 1 workload, bounded window
    gp = make_grid(pkg, cfg, pkg.ENGINE_PLAIN)
    gp.reset(seed=cfg["seed"], n_real=n_real)
    win = 50
    ts = timed_steps(torch, lambda: gp.advance(win, samples), 3, 1, flush)
    plain_rate = n_real * ncell * win * 3 / sum(ts)
    gp.close()
    # small rods (b = 4, 4 realisations, config of the plain-Heun workload)
    from workloads import CONFIGS
    c1 = CONFIGS["rod_b4_4real"]
    ncell1 = math.prod(c1["dims"])
    res = {}
    for name, eng, win1 in (("resident", pkg.ENGINE_RESIDENT, 20000), ("plain", pkg.ENGINE_PLAIN, 500)):
        g1 = make_grid(pkg, c1, eng)
        g1.reset(seed=c1["seed"], n_real=c1["n_real"])
        s1 = torch.zeros((c1["n_real"], g1.n_samples), device="cuda")
        t1 = timed_steps(torch, lambda: g1.advance(win1, s1), 3, 1, flush)
        res[name] = c1["n_real"] * ncell1 * win1 * 3 / sum(t1)
        spl = g1.steps_per_loop
        g1.close()
    out["plain_same_workload"] = {"value": plain_rate, "unit": UNIT,
                                  "resident_over_plain": None}
    out["rods_b4_608"] = small_rods_many(args, torch, pkg, flush)
    out["ladder_batch"] = ladder_batch(args, torch, pkg, flush)
    out["slab_512x512x56"] = slab_stream(args, torch, pkg, flush)
    out["adjoint_b4"] = adjoint_calibration(args, torch, pkg)
    out["small_rod_b4_4real"] = {
        "resident_cell_steps_per_s": res["resident"], "plain_cell_steps_per_s": res["plain"],
        "resident_over_plain": res["resident"] / res["plain"],
        "resident_loops_per_s": res["resident"] / (ncell1 * spl),
        "plain_loops_per_s": res["plain"] / (ncell1 * spl)}
    return out


KERNEL_SOURCES = ("paper_1912_00310_gb300/csrc/k_rod.cu", "paper_1912_00310_gb300/csrc/physics.cuh",
                  "paper_1912_00310_gb300/csrc/reduce.cuh")


def measured_traffic():
    """DRAM bytes per launch of the resident kernel from the committed ncu capture, or None when
    the kernel sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_rod_b1_256real.txt")
    try:
        kv = dict(line.split()[:2] for line in open(path) if line.strip() and not line.startswith("#"))
        h = hashlib.sha256()
        for f in KERNEL_SOURCES:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() == kv.get("kernel_sources_sha256"):
            return float(kv["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def hbm_peak_gbs():
    """Measured HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json beside this file, else a
    fallback of 6800 GB/s (an earlier copy measurement on a GB300)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = json.load(f).get("hbm_gbs")
        if v:
            return float(v), "measured"
    except (OSError, ValueError):
        pass
    return 6800.0, "fallback"


def small_rods_many(args, torch, pkg, flush):
    """The two-phase kernel on a full GPU of small rods: 608 b = 4 rods (2 x 6 x 14 cells, four per
    SM), the plain-Heun workload's material and sweep, launch shape chosen by the autotuner."""
    from workloads import CONFIGS
    c1 = dict(CONFIGS["rod_b4_4real"])
    n_real, W = 608, 20000
    g = make_grid(pkg, c1, pkg.ENGINE_RESIDENT)
    g.reset(seed=c1["seed"], n_real=n_real)
    tuned = g.autotune(trial_steps=2000)
    g.reset(seed=c1["seed"], n_real=n_real)
    S = torch.zeros((n_real, g.n_samples), device="cuda")
    ts = timed_steps(torch, lambda: g.advance(W, S), args.steps, 1, flush)
    rate = n_real * g.ncells * W * args.steps / sum(ts)
    shape = {k: g.tuning(k) for k in ("kind", "rods_per_cta", "cells_per_thread")}
    g.close()
    return {"rods": n_real, "cells_per_rod": math.prod(c1["dims"]), "heun_steps_per_call": W, "value": rate,
            "unit": UNIT, "autotuned_rate": tuned, "launch_shape": shape,
            "alu_frac": ALU_OPS_PER_CELL_STEP * rate / (ALU_PEAK["value"] or
                                                        (152 * ALU_LANES_PER_SM * MAX_SM_MHZ * 1e6))}


def ladder_batch(args, torch, pkg, flush):
    """The uneven ladder: b in {1,2,4,8} x rate in {1000,100,10} Oe/ns x alpha in
    {0.05,0.1,0.5,1.0}, 64 realisations each (3072 loops), advanced W Heun steps per call in one
    graph launch, against the same jobs run one after another with the plain engine."""
    from workloads import CONFIGS, DT_BY_B, MAGNETITE as M, ROD_DIMS
    c3 = CONFIGS["ladder_batch"]
    jobs, specs = [], []
    for b in c3["bs"]:
        for rate in c3["rates"]:
            for alpha in c3["alphas"]:
                g = pkg.Grid(*ROD_DIMS[b], a0=M["a0"], b=b)
                g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=alpha, T=M["T"])
                g.set_scaling(mode=c3["mode"], Tc=M["Tc"])
                g.set_sweep(H_start=c3["H_start"], H_turn=c3["H_turn"], rate=rate, dt=DT_BY_B[b],
                            sample_dH=c3["sample_dH"])
                g.set_engine(pkg.ENGINE_RESIDENT)
                g.reset(seed=c3["seed"], n_real=c3["n_real"], real_offset=len(jobs) * c3["n_real"])
                jobs.append(g)
                specs.append((b, rate, alpha))
    tuned = {}
    for g, (b, _, _) in zip(jobs, specs):
        if b not in tuned:
            tuned[b] = g.autotune(trial_steps=100)
        else:
            g.autotune(trial_steps=100)  # cached: same shape
    samples = [torch.zeros((c3["n_real"], g.n_samples), device="cuda") for g in jobs]
    W = 1000
    cells = sum(c3["n_real"] * g.ncells for g in jobs)
    ts = timed_steps(torch, lambda: pkg.run_batch(jobs, W, samples), args.steps, 1, flush)
    rate = cells * W * args.steps / sum(ts)
    loops_per_s = sum(c3["n_real"] * W / g.steps_per_loop for g in jobs) * args.steps / sum(ts)
    # the same jobs, one after another, with the plain engine (a short window each)
    Wp = 20
    t_plain = 0.0
    for g in jobs:
        g.set_engine(pkg.ENGINE_PLAIN)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for g, S in zip(jobs, samples):
        g.advance(2, S)
    torch.cuda.synchronize()
    e0.record(st)
    for g, S in zip(jobs, samples):
        g.advance(Wp, S)
    e1.record(st)
    e1.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    plain_rate = cells * Wp / t_plain
    for g in jobs:
        g.close()
    return {"jobs": len(jobs), "loops": len(jobs) * c3["n_real"], "heun_steps_per_call": W,
            "cell_steps_per_call": cells * W, "value": rate, "unit": UNIT,
            "loops_per_s": loops_per_s, "plain_sequential_cell_steps_per_s": plain_rate,
            "batched_over_plain": rate / plain_rate,
            "autotuned_cell_steps_per_s_by_b": {str(k): v for k, v in tuned.items()},
            "launch": "one CUDA graph per call (one kernel node per job, longest first)"}


def ladder_full(which):
    """Every job of the uneven ladder (b x rate x alpha, 64 realisations each) run to the end of
    its loop through the batching layer: graph calls of up to 2e6 Heun steps per job until every
    loop is complete.  'ci' leaves out the b = 1 jobs at 10 Oe/ns (3e8 steps per loop)."""
    import time
    import torch
    import paper_1912_00310_gb300 as pkg
    from workloads import CONFIGS, DT_BY_B, MAGNETITE as M, ROD_DIMS
    c3 = CONFIGS["ladder_batch"]
    jobs = []
    for b in c3["bs"]:
        for rate in c3["rates"]:
            if which == "ci" and b == 1 and rate == 10.0:
                continue
            for alpha in c3["alphas"]:
                g = pkg.Grid(*ROD_DIMS[b], a0=M["a0"], b=b)
                g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=alpha, T=M["T"])
                g.set_scaling(mode=c3["mode"], Tc=M["Tc"])
                g.set_sweep(H_start=c3["H_start"], H_turn=c3["H_turn"], rate=rate, dt=DT_BY_B[b],
                            sample_dH=c3["sample_dH"])
                g.set_engine(pkg.ENGINE_RESIDENT)
                g.reset(seed=c3["seed"], n_real=c3["n_real"], real_offset=len(jobs) * c3["n_real"])
                g.autotune(trial_steps=100)
                g.reset(seed=c3["seed"], n_real=c3["n_real"], real_offset=len(jobs) * c3["n_real"])
                jobs.append(g)
    samples = [torch.zeros((c3["n_real"], g.n_samples), device="cuda") for g in jobs]
    for S in samples:
        S[:, 0] = 1.0
    cell_steps = sum(c3["n_real"] * g.ncells * g.steps_per_loop for g in jobs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    calls = 0
    while True:
        done = pkg.run_batch(jobs, 2_000_000, samples)
        calls += 1
        if not any(done):
            break
        torch.cuda.synchronize()
        left = sum(1 for g in jobs if g.step < g.steps_per_loop)
        print(f"ladder_full: call {calls}, {time.perf_counter() - t0:.1f} s, {left} of {len(jobs)} "
              f"jobs unfinished", file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    finished = all(g.step == g.steps_per_loop for g in jobs)
    loops = len(jobs) * c3["n_real"]
    finite = all(bool(torch.isfinite(S).all()) for S in samples)
    for g in jobs:
        g.close()
    print(json.dumps({"leg": "ladder_full", "variant": which, "jobs": len(jobs), "loops": loops,
                      "all_loops_complete": finished, "samples_finite": finite,
                      "cell_steps": cell_steps, "seconds": sec, "graph_calls": calls,
                      "loops_per_s": loops / sec, "cell_steps_per_s": cell_steps / sec,
                      "unit": UNIT}), flush=True)


def slab_stream(args, torch, pkg, flush):
    """The 512x512x56 periodic slab with the streaming engine: one fused Heun step per launch."""
    from workloads import CONFIGS
    c4 = dict(CONFIGS["slab_512x512x56"], sample_dH=1.0)
    g = make_grid(pkg, c4, pkg.ENGINE_STREAM)
    g.reset(seed=c4["seed"], n_real=1)
    S = torch.zeros((1, g.n_samples), device="cuda")
    W = 100
    ts = timed_steps(torch, lambda: g.advance(W, S), args.steps, 1, flush)
    t_step = sum(ts) / (W * args.steps)
    rate = g.ncells / t_step
    peak, basis = hbm_peak_gbs()
    alg = 24.0 * rate / 1e9   # 12 B in + 12 B out per cell-step
    phys = 32.0 * rate / 1e9  # float4 state in and out
    ncells = g.ncells
    g.close()
    return {"cells": ncells, "value": rate, "unit": UNIT, "ms_per_heun_step": 1e3 * t_step,
            "hbm_algorithmic_gbs": alg, "hbm_float4_gbs": phys, "hbm_peak_gbs": peak,
            "hbm_peak_basis": basis, "hbm_frac_algorithmic": alg / peak,
            "alu_frac": ALU_OPS_PER_CELL_STEP * rate / (ALU_PEAK["value"] or (152 * ALU_LANES_PER_SM * MAX_SM_MHZ * 1e6)),
            "alu_peak_basis": "measured" if ALU_PEAK["value"] else "nominal",
            "l2": "state (470 MB ping-pong) larger than L2"}


def adjoint_calibration(args, torch, pkg):
    """Gradient evaluations per second of the calibration workload: b = 4 rod, 64 realisations,
    a 20k-step window at 1000 Oe/ns, checkpoints every 512 steps, mismatch against a fixed loop
    (the same window's mean loop of the b = 1 rod, 64 realisations)."""
    import numpy as np
    from workloads import CONFIGS, DT_BY_B, MAGNETITE as M, ROD_DIMS
    c5 = CONFIGS["adjoint_b4"]
    # target: the b = 1 rod's mean loop over the same field window
    t1 = pkg.Grid(*ROD_DIMS[1], a0=M["a0"], b=1)
    t1.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"], T=M["T"])
    t1.set_scaling(mode=c5["mode"], Tc=M["Tc"])
    t1.set_sweep(H_start=c5["H_start"], H_turn=c5["H_turn"], rate=c5["rate"], dt=DT_BY_B[1], sample_dH=1.0)
    t1.set_engine(pkg.ENGINE_RESIDENT)
    t1.reset(seed=c5["seed"] + 1, n_real=c5["n_real"])
    S1 = torch.zeros((c5["n_real"], t1.n_samples), device="cuda")
    S1[:, 0] = 1.0
    window_oe = c5["window_steps"] * c5["rate"] * 1e9 * c5["dt"]
    t1.advance(int(round(window_oe / (c5["rate"] * 1e9 * DT_BY_B[1]))), S1)
    t1.sync(600)
    target = S1.double().mean(0).cpu().numpy()
    t1.close()
    g = pkg.Grid(*c5["dims"], a0=M["a0"], b=c5["b"])
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"], T=M["T"])
    g.set_scaling(mode=c5["mode"], Tc=M["Tc"])
    g.set_sweep(H_start=c5["H_start"], H_turn=c5["H_turn"], rate=c5["rate"], dt=c5["dt"], sample_dH=1.0)
    g.set_engine(pkg.ENGINE_RESIDENT)
    g.reset(seed=c5["seed"], n_real=c5["n_real"])
    tgt = np.zeros(g.n_samples)
    tgt[:len(target)] = target[:g.n_samples]
    g.loss_grad(c5["window_steps"], tgt, 0, c5["ckpt_every"])  # warm-up
    t0 = time.perf_counter()
    n_eval = max(1, args.steps)
    for _ in range(n_eval):
        L, grad = g.loss_grad(c5["window_steps"], tgt, 0, c5["ckpt_every"])
    t_grad = (time.perf_counter() - t0) / n_eval
    # the forward-mode method on the same workload (one pass carrying the three tangents)
    g.set_tuning(pkg.TUNE_GRAD_METHOD, 1)
    Lt, gt = g.loss_grad(c5["window_steps"], tgt, 0, c5["ckpt_every"])  # warm-up
    t0 = time.perf_counter()
    for _ in range(n_eval):
        Lt, gt = g.loss_grad(c5["window_steps"], tgt, 0, c5["ckpt_every"])
    t_tan = (time.perf_counter() - t0) / n_eval
    g.set_tuning(pkg.TUNE_GRAD_METHOD, 0)
    S = torch.zeros((c5["n_real"], g.n_samples), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.advance(c5["window_steps"], S)
    g.sync(600)
    t_fwd = time.perf_counter() - t0
    g.close()
    return {"grads_per_s": 1.0 / t_grad, "s_per_grad": t_grad, "forward_only_s": t_fwd,
            "grad_over_forward": t_grad / t_fwd, "loss": L, "grad": [float(x) for x in grad],
            "method": "reverse-mode adjoint, checkpoints every ckpt_every steps",
            "tangent": {"grads_per_s": 1.0 / t_tan, "s_per_grad": t_tan, "grad_over_forward": t_tan / t_fwd,
                        "loss": Lt, "grad": [float(x) for x in gt],
                        "max_rel_diff_vs_adjoint": float(max(abs(a - b) / abs(a) for a, b in zip(grad, gt)))},
            "cell_steps_per_grad": c5["n_real"] * math.prod(c5["dims"]) * c5["window_steps"],
            "timing": "host wall clock per synchronous llg_loop_area_grad call"}


def profile_case(name):
    """A small untimed case of one kernel family, sized for an ncu capture (a few launches,
    tens of MB on the device)."""
    import torch
    import paper_1912_00310_gb300 as pkg
    from workloads import CONFIGS
    torch.cuda.set_device(0)
    if name in ("b1", "b1-plain"):
        # 160 rods: more than one wave of 152 SMs, so the balanced schedule of the benchmark's
        # 256-rod launch is exercised on a small case
        cfg = dict(CONFIGS["rod_b1_256real"])
        n_real, steps = 160, (200 if name == "b1" else 5)
        eng = pkg.ENGINE_RESIDENT if name == "b1" else pkg.ENGINE_PLAIN
    elif name == "b4-rows":
        # 608 b = 4 rods with the row kernel's default shape (one rod per CTA), no autotuning
        cfg = dict(CONFIGS["rod_b4_4real"])
        n_real, steps, eng = 608, 2000, pkg.ENGINE_RESIDENT
    elif name == "b4":
        # 608 b = 4 rods with the autotuned launch shape
        cfg = dict(CONFIGS["rod_b4_4real"])
        n_real, steps, eng = 608, 2000, pkg.ENGINE_RESIDENT
    elif name == "slab":
        # the 512x512x56 periodic slab (14.7M cells, 470 MB of state buffers), a few Heun steps
        cfg = dict(CONFIGS["slab_512x512x56"], sample_dH=1.0)
        n_real, steps, eng = 1, 4, pkg.ENGINE_STREAM
    elif name in ("adjoint", "tangent"):
        # the calibration workload's rod and ensemble on a 2000-step window, two gradients: the
        # adjoint (stored window: one recompute launch and one reverse launch per gradient) or
        # the tangent method (one launch per gradient)
        import numpy as np
        c5 = CONFIGS["adjoint_b4"]
        g = make_grid(pkg, dict(c5, sample_dH=1.0), pkg.ENGINE_RESIDENT)
        g.set_tuning(pkg.TUNE_GRAD_METHOD, 1 if name == "tangent" else 0)
        g.reset(seed=0, n_real=c5["n_real"])
        target = 0.9 + 0.05 * np.cos(np.arange(g.n_samples) / 7.0)
        for _ in range(2):
            g.loss_grad(2000, target, 0, c5["ckpt_every"])
        g.close()
        print(f"profile case {name}: 64 rods x 2000-step window x 2 gradients done")
        return 0
    else:
        raise SystemExit(f"unknown profile case {name}")
    g = make_grid(pkg, cfg, eng)
    g.reset(seed=0, n_real=n_real)
    if name == "b4":
        g.autotune(trial_steps=500)
        g.reset(seed=0, n_real=n_real)
    S = torch.zeros((n_real, g.n_samples), device="cuda")
    for _ in range(3):
        g.advance(steps, S)
    g.sync(600)
    g.close()
    print(f"profile case {name}: {n_real} rods x {steps} steps x 3 launches done")
    return 0


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.ladder_full:
        return ladder_full(args.ladder_full)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
