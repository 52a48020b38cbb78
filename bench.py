"""Benchmark of the PDDSparse hot path on GB300: Monte Carlo assembly of
G(w) u = b(w) (Eq. 24-25) plus its FP64 solve (Eq. 23).

Default workload: config 3, the largest single-GPU configuration -- 16
independent BVPs on [0,4]^2 (subdomain grids 4x4 to 32x32, m = 8, variable
sigma, c = -1, per-knot budgets log-uniform in [1e4, 1e5], dt = 1e-5,
105,813 knots, ~1.56e12 path-steps) assembled in ONE persistent launch
replayed from a CUDA graph, then 16 FP64 solves.  One step = that whole batch.
``--config cfg2`` times the single manufactured problem (8x8 subdomains, 833
knots, N = 1e5, dt = 1e-5) instead.  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--config cfg3]

N > 1 runs under torchrun, one process per GPU; every rank assembles an
independent replica (its own seed), so per-GPU work is fixed (weak scaling)
and no collective touches the data path (a barrier and a max-reduction of the
timings only).  ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import inspect
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Counted FP32 operations per Euler-Maruyama path-step of the path kernel
# (FMA = 2, every other FP32 add/mul/compare/min/max = 1, each hardware
# transcendental = 1), read off paper_2301_05780_gb300/csrc/pdds_path.cu:
#   Box-Muller share per step 17, exit test 4, EM update 17 (with Y, Z) or 6,
#   coefficients: MANUFACTURED 39, VARSIGMA 32, TABLE 26 (two bilinear lookups), LAPLACE 0,
#   CONSTANT 0.
FLOPS_PER_STEP = {0: 27, 1: 77, 2: 70, 3: 64, 4: 38}
SMS_GB300 = 152
FP32_LANES_PER_SM = 128


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Every source compiled into the path kernel: the template, the headers it
# includes from csrc/ and the six files that instantiate it.
PATH_KERNEL_SOURCES = ("path_kernel.cuh", "pdds_internal.h", "pdds_mlp.cuh", "pdds_rbf.cuh",
                       "pdds_path_em.cu", "pdds_path_cv.cu", "pdds_path_cvt.cu",
                       "pdds_path_ext.cu", "pdds_path_ext_cv.cu", "pdds_path_ext_cvt.cu")


def kernel_source_hash() -> str:
    """Hash of the path kernel's sources: a committed ncu summary carries the
    hash of the sources it was taken on, and its figures are reported only
    while the hash still matches."""
    h = hashlib.sha256()
    for f in PATH_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2301_05780_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# Committed ncu summary of each single-launch workload's path kernel.
PROFILES = {"cfg2": "path_kernel_cfg2_ncu.txt", "cfg3": "path_kernel_cfg3_batch_ncu.txt",
            "cfg4": "path_kernel_cfg4_tabulated_ncu.txt"}


def profiled_value(config: str, key: str):
    """A `key: value` figure of the committed ncu summary of this workload's
    path kernel, if the summary was taken on the current kernel source; else
    None."""
    if config not in PROFILES:
        return None
    p = os.path.join(ROOT, "profiles", PROFILES[config])
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_v = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", txt)
    if not (m_hash and m_v) or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_v.group(1))


def profiled_traffic(config: str):
    """DRAM bytes per launch of the path kernel (committed ncu summary)."""
    return profiled_value(config, "dram_bytes_per_full_launch")


def issue_roofline(config: str, path_steps_per_s: float, sm_max_mhz: float):
    """The path kernel is bound by instruction issue: warp instructions per
    path-step from the committed ncu summary times the live path-step rate,
    against 152 SMs x 4 schedulers x one warp instruction per cycle."""
    wi = profiled_value(config, "warp_instructions_per_path_step")
    if wi is None:
        return None
    peak = SMS_GB300 * 4 * sm_max_mhz * 1e6
    achieved = path_steps_per_s * wi
    return {"warp_instructions_per_path_step": wi, "achieved_warp_inst_per_s": achieved,
            "peak_warp_inst_per_s": peak, "frac": achieved / peak,
            "source": "instructions per path-step from the committed ncu summary of this kernel "
                      "source; peak = 152 SMs x 4 schedulers x 1 warp instruction/cycle x max SM "
                      "clock"}


# Directory for the raw nvidia-smi samples (--clocks-dir); a temporary one
# when unset.  The JSON line carries their summary either way.
CLOCKS_DIR = None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.proc = None
        d = CLOCKS_DIR or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_gpu{gpu_index}_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank r's independent replica (rank 0 keeps the workload seed)."""
    return (base + 1000003 * rank) % 2**64


def reduce_timing(total_ms: float, path_steps: float, device="cpu"):
    """Whole-job timing over ranks: the slowest rank's time and the sum of the
    path-steps all ranks processed (timing only; no data-path collective)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, path_steps
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    s = torch.tensor([path_steps], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t[0]), float(s[0])


def exact_solution(coef_id: int, xy: np.ndarray):
    """Closed-form u at the knots for the workloads that have one (None for the
    tabulated coefficient fields, which have no exact solution)."""
    x, y = xy[:, 0], xy[:, 1]
    if coef_id == 0:
        return np.exp(x) * np.sin(y)
    if coef_id == 1:
        return np.sin(np.pi * x) * np.cos(np.pi * y) + x * y
    if coef_id == 2:
        return np.exp(x / 4) * np.cos(y / 2)
    if coef_id == 5:
        r = np.sqrt(1 + x * x / 100 + y * y / 50)
        q = np.sin(3 * x / 25 + y / 20) + np.sin(x / 20 - 3 * y / 25)
        return 3 + np.sin(r) / 3 + np.tanh(q) / 3
    return None


def workload(name: str):
    from paper_2301_05780_gb300 import workloads as W
    return W.all_configs()[name]()


# ------------------------------------------------------------------ CPU arm
def oracle_sample(w, rows_wanted: int, threads: int, frac: float = 1.0):
    """Times the FP64 oracle on `rows_wanted` evenly spaced rows of w at the
    per-knot budget (times frac, at least one path); returns (path_steps,
    seconds, rows)."""
    import oracle
    tabs = w.tables if w.tables is not None else (None, None)
    O = oracle.Problem(w.grid, w.coef_id, w.params, sigma_tab=tabs[0], c_tab=tabs[1])
    rows = np.linspace(0, O.n - 1, rows_wanted).round().astype(np.int32)
    N = w.budgets(O.n) if w.budget_seed is not None else np.full(O.n, w.n_paths, np.int64)
    N = np.maximum(1, np.round(N * frac)).astype(np.int64)
    t0 = time.perf_counter()
    _, _, st, _ = O.assemble(N, w.dt, w.seed, w.k_max, rows=rows, threads=threads)
    return int(st[0]), time.perf_counter() - t0, rows


def cpu_baseline(w, budget_s: float = 15.0):
    threads = os.cpu_count() or 1
    steps, secs, rows = oracle_sample(w, threads, threads)       # calibration
    rate = steps / secs
    per_row = steps / len(rows)
    want = int(max(threads, min(w.extra.get("n_rows", 10**9), budget_s * rate / per_row)))
    want = min(want, 4000)
    steps, secs, rows = oracle_sample(w, want, threads)
    if secs < 0.5 * budget_s and want < 4000:   # the calibration overestimated a row's cost
        want = int(min(4000, want * budget_s / max(secs, 1e-3)))
        steps, secs, rows = oracle_sample(w, want, threads)
    distinct = len(set(rows.tolist()))
    what = (f"{len(rows)} evenly spaced rows" if distinct == len(rows) else
            f"{len(rows)} rows ({distinct} distinct, each recomputed)")
    return {"value": steps / secs, "unit": "path-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{what} of {w.name} at N={w.n_paths}, "
                      f"dt={w.dt:g} ({steps:.3e} path-steps in {secs:.1f} s, FP64, "
                      f"{threads} threads)"}


def cpu_baseline_batch(ws, budget_s: float = 15.0):
    """The oracle on `threads` evenly spaced rows of every problem of a batch,
    each row at the same fraction of its own per-knot budget: a 1 % pass
    calibrates the fraction that fills the time budget."""
    threads = os.cpu_count() or 1

    def sweep(frac):
        steps = secs = 0.0
        for w in ws:
            s_, t_, _ = oracle_sample(w, threads, threads, frac)
            steps, secs = steps + s_, secs + t_
        return steps, secs

    _, secs = sweep(0.01)
    frac = float(min(1.0, max(0.01, 0.01 * budget_s / max(secs, 1e-9))))
    steps, secs = sweep(frac)
    return {"value": steps / secs, "unit": "path-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{threads} evenly spaced rows of each of the {len(ws)} problems, each at "
                      f"{100 * frac:.1f} % of its per-knot budget ({steps:.3e} path-steps in "
                      f"{secs:.1f} s, FP64, {threads} threads)"}


def run_reference_batch(args):
    """The oracle on the batched config-3 workload: every step is a bounded
    sample of the 16 problems (`threads` evenly spaced rows of each, every row
    at the same fraction of its own per-knot budget), the fraction chosen by a
    short calibration pass so that one step takes about 4 s of host time."""
    ws = workload("cfg3")
    threads = os.cpu_count() or 1

    def sweep(frac):
        steps = secs = 0.0
        for w in ws:
            s_, t_, _ = oracle_sample(w, threads, threads, frac)
            steps, secs = steps + s_, secs + t_
        return steps, secs

    _, secs = sweep(0.002)
    frac = float(min(1.0, max(0.001, 0.002 * 4.0 / max(secs, 1e-9))))
    for _ in range(args.warmup):
        sweep(frac)
    tot_steps, tot_s = 0.0, 0.0
    for _ in range(args.steps):
        s_, t_ = sweep(frac)
        tot_steps += s_
        tot_s += t_
    v = tot_steps / tot_s
    sample = (f"{threads} evenly spaced rows of each of the {len(ws)} problems per step, each at "
              f"{100 * frac:.2f} % of its per-knot budget (FP64 oracle, {threads} threads)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "path-steps/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cfg3_batch16", "problems": len(ws), "dt": ws[0].dt,
                       "sample_budget_fraction": frac},
            "cpu_baseline": {"value": v, "unit": "path-steps/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "path-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    if args.config == "cfg3":
        return run_reference_batch(args)
    w = workload(args.config)
    threads = os.cpu_count() or 1
    rows_per_step = max(threads, 2 * threads)
    for _ in range(args.warmup):
        oracle_sample(w, threads, threads)
    tot_steps, tot_s = 0, 0.0
    for _ in range(args.steps):
        s, t, rows = oracle_sample(w, rows_per_step, threads)
        tot_steps += s
        tot_s += t
    v = tot_steps / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "path-steps/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample_rows_per_step": rows_per_step,
                       "paths_per_knot": w.n_paths, "dt": w.dt},
            "cpu_baseline": {"value": v, "unit": "path-steps/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"{rows_per_step} evenly spaced rows per step of {w.name} "
                                       f"at N={w.n_paths} (FP64 oracle, {threads} threads)"},
            "e2e": {"value": v, "unit": "path-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
METRIC = "path-steps/s & G,b assembly time at fixed interface RMS error; % of FP32 peak"


def run_gpu(args):
    import torch
    from paper_2301_05780_gb300 import pdds

    rank, local, world = dist_env()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args.config)
    w.seed = replica_seed(w.seed, rank)       # independent replica per rank
    if args.paths:
        w.n_paths = args.paths
    P = pdds.Problem(w, device=local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    if args.no_autotune:
        launch = pdds.pdds_get_launch(P.ctx)
    else:
        launch = pdds.pdds_autotune(P.ctx, w.n_paths, w.dt, w.seed)  # before warm-up, untimed
    pdds.pdds_set_timing(P.ctx, True)

    def step(step_ev=None, asm_ev=None):
        # the step's events bracket assembly + solve only; one pdds_stats after
        # them reads the counters and the path-kernel time of the assembly, so
        # no host synchronization falls between the two calls
        if step_ev:
            step_ev[0].record(stream)
        if asm_ev:
            asm_ev[0].record(stream)
        P.assemble(stream)
        if asm_ev:
            asm_ev[1].record(stream)
        P.solve(rtol=1e-12, maxit=5000, stream=stream)
        if step_ev:
            step_ev[1].record(stream)
        return pdds.pdds_stats(P.ctx)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # the whole pdds_assemble call (CSR/b clearing, unit prefix, path kernel, finalize)
    asm_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    path_ms, steps_done, launches, errors, iters = [], 0, 0, 0, []
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()                    # evict L2 between timed steps
            st = step(ev[i], asm_ev[i])
            path_ms.append(st["path_kernel_ms"])
            steps_done += st["path_steps"]
            launches += st["kernel_launches"]
            errors += st["device_error"]
            iters.append(st["solve_iters"])
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    asm_ms = [a.elapsed_time(b) for a, b in asm_ev]
    total_ms = sum(step_ms)
    total_ms_max, steps_all = reduce_timing(total_ms, float(steps_done), device="cuda")
    value = steps_all / (total_ms_max * 1e-3)

    # ---- end to end through the host-buffer C-ABI call (pinned buffers)
    n, nnz = P.n, P.nnz
    pin = dict(pin_memory=True)
    Nh = torch.full((n,), w.n_paths, dtype=torch.int64, **pin)
    rp = torch.empty(n + 1, dtype=torch.int32, **pin)
    col = torch.empty(nnz, dtype=torch.int32, **pin)
    val = torch.empty(nnz, dtype=torch.float64, **pin)
    bh = torch.empty(n, dtype=torch.float64, **pin)
    uh = torch.empty(n, dtype=torch.float64, **pin)
    pdds.pdds_set_timing(P.ctx, False)
    e2e_steps = 0 if args.no_baseline else max(2, min(args.steps, 5))
    if e2e_steps:
        pdds.pdds_assemble_solve_host(P.ctx, 0, w.dt, w.seed, 1e-12, 5000, rp, col, val, bh, uh,
                                      n_per_knot=Nh)
        torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pdds.pdds_assemble_solve_host(P.ctx, 0, w.dt, w.seed, 1e-12, 5000, rp, col, val, bh, uh,
                                      n_per_knot=Nh)
    e2e_s = (time.perf_counter() - t0) / max(e2e_steps, 1)
    e2e_val = steps_done / args.steps / e2e_s * world if e2e_steps else None
    h2d = n * 8
    d2h = (n + 1) * 4 + nnz * 4 + nnz * 8 + 2 * n * 8

    # interface error against the manufactured solution (last timed step)
    xy = pdds.pdds_knot_coords(P.ctx)
    u = P.u.cpu().numpy()
    ex = exact_solution(w.coef_id, xy)
    rms = None if ex is None else float(np.sqrt(np.mean((u - ex) ** 2)))

    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0
    peaks, src = measured_peaks()
    clk_s = clk.summary()
    fpk = FLOPS_PER_STEP[w.coef_id]
    kernel_s = float(np.mean(path_ms)) * 1e-3
    flops_launch = steps_done / args.steps * fpk
    achieved = flops_launch / kernel_s / 1e12
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = SMS_GB300 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    cpu = None if args.no_baseline else cpu_baseline(w)
    line = {
        "metric": METRIC, "value": value, "unit": "path-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "knots": n, "paths_per_knot": w.n_paths, "dt": w.dt,
                   "path_steps_per_step": steps_done / args.steps,
                   "assembly_ms": float(np.mean(path_ms)),
                   "assemble_call_ms": {"median": float(np.median(asm_ms)),
                                        "min": float(np.min(asm_ms)),
                                        "reps": len(asm_ms)},
                   "solve_iters": int(np.median(iters)), "interface_rms_error": rms,
                   "accumulation": "f64", "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "launch": {"block": launch[0], "unit_paths": launch[2],
                              "exit_batch": launch[3],
                              "chosen_by": "default" if args.no_autotune else "pdds_autotune"}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(args.config),
                     "kernel": "path_kernel", "flops_per_path_step": fpk,
                     "issue": issue_roofline(args.config, steps_done / args.steps / kernel_s,
                                             sm_max),
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                    f"({src} max SM clock)"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "path-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk_s,
        "device_errors": errors,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 10 for the batched config 3, 20 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cfg3",
                    choices=["cfg1", "cfg2", "cfg3", "cfg4", "cfg5", "cfg5_network", "e1", "e1_bias"],
                    help="workload (default: config 3, the largest single-GPU configuration)")
    ap.add_argument("--paths", type=int, default=0,
                    help="override paths per knot (small profiling cases; not a bench line)")
    ap.add_argument("--no-baseline", action="store_true",
                    help="skip the CPU-oracle baseline and the end-to-end leg (profiling runs)")
    ap.add_argument("--cv", default="table", choices=["table", "network"],
                    help="control variate of the e1 pipeline: tabulated grad u0 or the network")
    ap.add_argument("--train-steps", type=int, default=1500,
                    help="Adam steps of the e1 pipeline's network fit")
    ap.add_argument("--launch", default=None,
                    help="cfg5_network, e1: fixed launch shape 'block,unit_paths,exit_batch' "
                         "(cfg5_network: no autotune; profiling runs)")
    ap.add_argument("--net-engine", default="tcgen05", choices=["tcgen05", "mma_sync"],
                    help="tensor-core engine of the in-path network (cfg5_network)")
    ap.add_argument("--train-engine", default="tc", choices=["fp32", "tc"],
                    help="training kernel of the network fits (e1, cfg5): FP32 SIMT or tcgen05")
    ap.add_argument("--fit-data", default="knots", choices=["knots", "knots+boundary"],
                    help="what the e1 pipeline's network is fitted to: the warm-up nodal values, "
                         "plus g on the boundary")
    ap.add_argument("--interp", default="linear", choices=["linear", "rbf"],
                    help="stencil interpolation of the e1 pipeline (Sec. 2.1 RBF or linear)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shape (profiling runs count launches)")
    ap.add_argument("--clocks-dir", default=None,
                    help="keep the raw nvidia-smi samples of the timed region in this directory")
    args = ap.parse_args()
    global CLOCKS_DIR
    if args.clocks_dir:
        os.makedirs(args.clocks_dir, exist_ok=True)
        CLOCKS_DIR = args.clocks_dir
    if args.steps is None:
        args.steps = 10 if args.config == "cfg3" else 20
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "cfg5":
        return run_cv_study(args)
    if args.config == "cfg5_network":
        return run_cv_network(args)
    if args.config == "cfg3":
        return run_batch(args)
    if args.config == "e1":
        return run_e1(args)
    if args.config == "e1_bias":
        return run_e1_bias(args)
    return run_gpu(args)


def run_batch(args):
    """Config 3: 16 independent BVPs with per-knot budgets in ONE persistent
    launch (captured once into a CUDA graph and replayed) plus the 16 FP64
    solves; one step = that whole batch.  Under torchrun every rank runs an
    independent replica of the batch (its own seed): weak scaling, no
    data-path collective."""
    import torch
    from paper_2301_05780_gb300 import pdds

    rank, local, world = dist_env()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ws = workload("cfg3")
    seed = replica_seed(ws[0].seed, rank)
    for w in ws:
        w.seed = seed
    probs = [pdds.Problem(w, device=local) for w in ws]
    if args.paths:
        for P in probs:
            P.n_per_knot = torch.clamp(P.n_per_knot, max=args.paths)
    c0 = probs[0].ctx
    # The batch's launch shape, measured on one GB300 at the full budgets (the
    # per-problem autotuner does not cover batches): 128-thread CTAs, units of
    # 2048 paths, exit batch 4 ran 1 % faster than 256 / 4096 / 4 and ahead of
    # 128 / 4096 / 4, 128 / 2048 / 2 and 192 / 2048 / 4.
    if not args.no_autotune:
        pdds.pdds_set_launch(c0, 128, 0, 2048, 4)
    launch = pdds.pdds_get_launch(c0)
    pdds.pdds_set_timing(c0, True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    args_b = ([P.ctx for P in probs], [P.G for P in probs], [P.b for P in probs], 0,
              [P.n_per_knot for P in probs], ws[0].dt, seed)

    def step(ev=None):
        # events around the batched assembly and the 16 solves; the counters
        # and the batched graph's time are read once, after them
        if ev:
            ev[0].record(stream)
        pdds.pdds_assemble_batch(*args_b, stream=stream)
        for P in probs:
            P.solve(rtol=1e-12, maxit=5000, stream=stream)
        if ev:
            ev[1].record(stream)
        return pdds.pdds_stats(c0)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    kms, steps, t_ms, launches, errors = [], 0, 0.0, 0, 0
    # problem 0's counters restart with every batched launch; the other
    # contexts only solve, and their launch counters keep adding up
    others0 = [pdds.pdds_stats(P.ctx)["kernel_launches"] for P in probs[1:]]
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()                    # evict L2 between timed steps
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            st = step((a, b_))
            launches += st["kernel_launches"]
            errors += st["device_error"]
            torch.cuda.synchronize()
            t_ms += a.elapsed_time(b_)
            kms.append(st["path_kernel_ms"])
            steps += st["path_steps"]
    launches += sum(pdds.pdds_stats(P.ctx)["kernel_launches"] - k0
                    for P, k0 in zip(probs[1:], others0))
    t_max, steps_all = reduce_timing(t_ms, float(steps), device="cuda")
    value = steps_all / (t_max * 1e-3)

    # ---- end to end through the host-buffer C-ABI batch call (pinned buffers):
    # budgets up; G, b and u of all 16 problems down, every step
    pin = dict(pin_memory=True)
    Nh = [P.n_per_knot.cpu().pin_memory() for P in probs]
    rp = [torch.empty(P.n + 1, dtype=torch.int32, **pin) for P in probs]
    col = [torch.empty(P.nnz, dtype=torch.int32, **pin) for P in probs]
    val = [torch.empty(P.nnz, dtype=torch.float64, **pin) for P in probs]
    bh = [torch.empty(P.n, dtype=torch.float64, **pin) for P in probs]
    uh = [torch.empty(P.n, dtype=torch.float64, **pin) for P in probs]
    pdds.pdds_set_timing(c0, False)
    ctxs = [P.ctx for P in probs]
    e2e_steps = 0 if args.no_baseline else max(2, min(args.steps, 3))

    def e2e_call():
        return pdds.pdds_assemble_solve_batch_host(ctxs, 0, ws[0].dt, seed, 1e-12, 5000, rp, col,
                                                   val, bh, uh, n_per_knot=Nh, stream=stream)
    e2e_val, e2e_check = None, None
    if e2e_steps:
        e2e_call()                                    # captures its graph (untimed)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        e2e_path_steps = 0
        for _ in range(e2e_steps):
            e2e_call()
            e2e_path_steps += pdds.pdds_stats(c0)["path_steps"]
        e2e_s = time.perf_counter() - t0
        e2e_max, e2e_all = reduce_timing(e2e_s * 1e3, float(e2e_path_steps), device="cuda")
        e2e_val = e2e_all / (e2e_max * 1e-3)
        # the host copies hold the same G, b, u as the device call on the same streams
        u_dev = probs[0].u.cpu().numpy()
        e2e_check = {"copies_declared": True,
                     "u0_max_abs_diff_vs_device_call": float(np.abs(uh[0].numpy() - u_dev).max())}
    h2d = sum(P.n * 8 for P in probs)
    d2h = sum((P.n + 1) * 4 + P.nnz * 4 + P.nnz * 8 + 2 * P.n * 8 for P in probs)

    # interface error against the closed form (last timed step, all problems)
    err = np.concatenate([P.u.cpu().numpy() - exact_solution(w.coef_id, pdds.pdds_knot_coords(P.ctx))
                          for P, w in zip(probs, ws)])
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0
    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = SMS_GB300 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    fpk = FLOPS_PER_STEP[ws[0].coef_id]
    kernel_s = float(np.mean(kms)) * 1e-3
    achieved = steps / args.steps * fpk / kernel_s / 1e12
    line = {"metric": METRIC, "value": value, "unit": "path-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "cfg3_batch16", "problems": len(ws),
                       "H": [w.grid["Hx"] for w in ws], "knots": sum(P.n for P in probs),
                       "paths": sum(P.total_paths() for P in probs), "dt": ws[0].dt,
                       "path_steps_per_step": steps / args.steps,
                       "batched_kernel_ms": float(np.mean(kms)),
                       "solve": "16 FP64 BiCGSTAB solves to 1e-12 inside each step",
                       "interface_rms_error": float(np.sqrt(np.mean(err ** 2))),
                       "accumulation": "f64", "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "launch": {"block": launch[0], "unit_paths": launch[2],
                                  "exit_batch": launch[3], "kind": "one persistent kernel for "
                                  "all 16 problems, replayed from a CUDA graph",
                                  "chosen_by": "default" if args.no_autotune else
                                  "measured launch-shape sweep at full budgets"}},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": profiled_traffic("cfg3"),
                         "kernel": "path_kernel", "flops_per_path_step": fpk,
                         "issue": issue_roofline("cfg3", steps / args.steps / kernel_s, sm_max),
                         "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                        f"({src} max SM clock)"},
            "cpu_baseline": None if args.no_baseline else cpu_baseline_batch(ws),
            "e2e": {"value": e2e_val, "unit": "path-steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "call": "pdds_assemble_solve_batch_host (pinned host buffers)"},
            "e2e_check": e2e_check,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "device_errors": errors}
    print(json.dumps(line), flush=True)
    return 0


def run_cv_network(args):
    """Config 5 with the in-path network control variate (Eq. 37; the
    network's gradient on the tensor cores in every step): a step is one
    assembly + solve at N paths per knot (default 1881, the CV study's budget
    for the plain estimator's error) with the seeded initial network v_theta
    (the kernel's cost does not depend on the parameter values)."""
    import torch
    from paper_2301_05780_gb300 import pdds
    torch.cuda.set_device(0)
    w = workload("cfg5")
    w.n_paths = args.paths or 1881
    P = pdds.Problem(w)
    from paper_2301_05780_gb300 import workloads as W
    theta = torch.tensor(W.mlp_init(), dtype=torch.float32, device="cuda")
    engine = {"tcgen05": pdds.NET_TCGEN05, "mma_sync": pdds.NET_MMA_SYNC}[args.net_engine]
    pdds.pdds_set_network_engine(P.ctx, engine)
    pdds.pdds_set_control_variate(P.ctx, theta)
    if args.launch:
        blk, un, ba = (int(v) for v in args.launch.split(","))
        pdds.pdds_set_launch(P.ctx, blk, 0, un, ba)
    launch = (pdds.pdds_get_launch(P.ctx) if args.no_autotune or args.launch
              else pdds.pdds_autotune(P.ctx, w.n_paths, w.dt, w.seed))
    pdds.pdds_set_timing(P.ctx, True)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        P.assemble(stream)
        pdds.pdds_stats(P.ctx)
    kms, steps, t_ms = [], 0, 0.0
    with Clocks(0) as clk:
        for _ in range(args.steps):
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            P.assemble(stream)
            P.solve(rtol=1e-10, maxit=5000, stream=stream)
            b_.record(stream)
            st = pdds.pdds_stats(P.ctx)
            torch.cuda.synchronize()
            t_ms += a.elapsed_time(b_)
            kms.append(st["path_kernel_ms"])
            steps += st["path_steps"]
    line = {"metric": METRIC, "value": steps / (t_ms * 1e-3), "unit": "path-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic",
            "config": {"workload": "cfg5_network_cv", "knots": P.n, "paths_per_knot": w.n_paths,
                       "dt": w.dt, "path_steps_per_step": steps / args.steps,
                       "kernel_ms": float(np.mean(kms)),
                       "launch": {"block": launch[0], "unit_paths": launch[2],
                                  "exit_batch": launch[3], "grid": st["path_grid"],
                                  "threads": st["path_block"]},
                       "network": "seeded initial v_theta (2-64-64-1, SiLU)",
                       "network_engine": args.net_engine},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_cv_study(args):
    """Config 5: plain estimator vs the learned control variate, time to the
    same interfacial statistical error (one JSON line; not the default bench)."""
    import torch
    from paper_2301_05780_gb300 import cv
    torch.cuda.set_device(0)
    w = workload("cfg5")
    n_plain = args.paths or w.n_paths
    res = cv.study(w, n_plain, train_engine=args.train_engine)
    plain = res["plain"]
    line = {"metric": METRIC, "value": plain["path_steps"] / (plain["kernel_ms"] * 1e-3),
            "unit": "path-steps/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": plain["assembly_solve_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "knots": res["knots"], "dt": w.dt,
                       "paths_per_knot": n_plain},
            "cpu_baseline": None if args.no_baseline else cpu_baseline(w),
            "cv_study": res}
    print(json.dumps(line), flush=True)
    return 0


# The paper's reported E1 figures (Sec. 5.2.1; other hardware and RBF
# stencils): Phase I and Phase III interfacial errors, the mean variance
# reduction factor and the mean estimated bias at h0.
PAPER_E1 = {"phase1": {"max": 0.074, "rmse": 0.016, "frac_below_eps": 0.4898},
            "phase3": {"max": 0.0224, "rmse": 0.0044, "frac_below_eps": 0.9703},
            "mean_vrf": 31.37, "mean_bias_at_h0": 3e-5}


def _e1_exact_grad(grid: dict, per_interval: int = 2):
    """grad u of Eq. 43 at the nodes of a grid of `per_interval` nodes per knot
    spacing over Omega (the look-up-table grid of the e1 pipeline), by central
    differences of the closed form in FP64 (step 1e-4: error ~1e-10)."""
    nx = per_interval * grid["Hx"] * grid["m"] + 1
    ny = per_interval * grid["Hy"] * grid["m"] + 1
    X, Y = np.meshgrid(np.linspace(grid["x0"], grid["x1"], nx),
                       np.linspace(grid["y0"], grid["y1"], ny))
    d = 1e-4

    def u(x, y):
        return exact_solution(5, np.stack([x.ravel(), y.ravel()], 1)).reshape(x.shape)
    gx = (u(X + d, Y) - u(X - d, Y)) / (2 * d)
    gy = (u(X, Y + d) - u(X, Y - d)) / (2 * d)
    return np.stack([gx, gy], axis=-1).astype(np.float32)


def run_e1_bias(args):
    """The calibration estimates of Sec. 4.1-4.2 on the paper's problem, on
    every 10th knot with the exact nodal u as patch data (so that only the
    path discretisation and the sampling enter):
      * Eq. 36's estimate of E[phi_EM - phi_GM] at h = 0.08, 0.04, 0.02 with
        N = 1000 (the paper's N0') and N = 64,000 paths per knot: its mean,
        the mean of |gap| / 2 (Eq. 35, what the pipeline reports) and the
        sampling noise of the gap, sd(phi_EM - phi_GM) / sqrt(N);
      * the predicted variance-reduction factor 1 / (1 - rho^2) of Eq. 39 at
        h = 0.08, N = 1000, with the exact grad u of Eq. 43 as the look-up table
        (the best any warm-up solution can give)."""
    import torch
    from paper_2301_05780_gb300 import pdds
    torch.cuda.set_device(0)
    w = workload("e1")
    P = pdds.Problem(w)
    n = P.n
    xy = pdds.pdds_knot_coords(P.ctx)
    u0 = torch.tensor(exact_solution(w.coef_id, xy), dtype=torch.float64, device=P.dev)
    rows = np.arange(0, n, 10)
    mom = torch.empty(n, pdds.CAL_NMOM, dtype=torch.float64, device=P.dev)

    def calibrate(h, N, seed):
        budgets = np.zeros(n, dtype=np.int64)
        budgets[rows] = N
        pdds.pdds_calibrate(P.ctx, u0, mom, 0, torch.from_numpy(budgets).to(P.dev), h, seed)
        M = mom.cpu().numpy()[rows]
        cnt = M[:, 0]
        gap = M[:, 1] / cnt
        var_d = np.maximum(M[:, 2] - cnt * gap ** 2, 0.0) / (cnt - 1)
        mphi = M[:, 3] / cnt
        var_phi = np.maximum(M[:, 4] - cnt * mphi ** 2, 0.0) / (cnt - 1)
        mxi = M[:, 5] / cnt
        var_xi = np.maximum(M[:, 6] - cnt * mxi ** 2, 0.0) / (cnt - 1)
        cov = (M[:, 7] - cnt * mphi * mxi) / (cnt - 1)
        rho2 = np.where(var_phi * var_xi > 0, cov ** 2 / np.maximum(var_phi * var_xi, 1e-300), 0.0)
        return gap, np.sqrt(var_d / cnt), rho2

    runs = []
    with Clocks(0) as clk:
        for h in (0.08, 0.04, 0.02):
            for N in (1000, 64000):
                gap, noise, _ = calibrate(h, N, w.seed + 1)
                runs.append({"h": h, "N": N, "mean_gap": float(gap.mean()),
                             "mean_abs_gap_half": float(np.abs(gap).mean() / 2),
                             "rms_gap": float(np.sqrt(np.mean(gap ** 2))),
                             "mean_noise_of_gap": float(noise.mean()),
                             # E|gap| / 2 of a zero-mean Gaussian gap with that noise
                             "pure_noise_abs_gap_half": float(noise.mean() * math.sqrt(2 / math.pi) / 2)})
        pdds.pdds_set_control_variate_grid(P.ctx, torch.from_numpy(_e1_exact_grad(w.grid)).cuda())
        _, _, rho2 = calibrate(0.08, 1000, w.seed + 1)
        pdds.pdds_set_control_variate_grid(P.ctx, None)
    line = {"metric": "calibration estimates (Eq. 35-36, 39) on the paper's problem",
            "config": {"workload": w.name, "rows": int(len(rows)), "patch_data": "exact u"},
            "bias_runs": runs,
            "vrf_exact_gradient_table": {"h": 0.08, "N": 1000,
                                         "mean_predicted_vrf": float(np.mean(1 / np.maximum(1 - rho2, 1e-12))),
                                         "median_predicted_vrf": float(np.median(1 / np.maximum(1 - rho2, 1e-12)))},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_e1(args):
    """The paper's experiment (Sec. 5.1) through the calibrated three-phase
    pipeline (warm-up, mixed GM/EM calibration with Eq. 40-41, production
    with per-knot N_i, h_i, GM exits and the control variate).  A step is one
    whole pipeline; the line's value is the path-steps of all three phases
    over the pipeline's wall time."""
    import torch
    from paper_2301_05780_gb300 import calibrated
    torch.cuda.set_device(0)
    w = workload("e1")
    x = w.extra
    kw = dict(eps=x["eps"], n0=args.paths or x["n0"], h0=x["h0"], n_job=x["n_job"],
              rbf=args.interp == "rbf", cv_kind=args.cv, train_steps=args.train_steps,
              boundary_samples=args.fit_data == "knots+boundary", train_engine=args.train_engine)
    if args.launch:  # else the pipeline's own launch shape
        kw["launch"] = tuple(int(v) for v in args.launch.split(","))
    for _ in range(args.warmup):
        calibrated.run(w, **kw)
    runs = []
    with Clocks(0) as clk:
        for _ in range(args.steps):
            runs.append(calibrated.run(w, **kw))
    out = runs[-1]
    ue = exact_solution(w.coef_id, out["xy"])
    e1 = calibrated.error_summary(out["phase1"]["u"], ue, x["eps"])
    e3 = calibrated.error_summary(out["phase3"]["u"], ue, x["eps"])
    total_ms = [r["phase1"]["ms"] + r.get("fit", {}).get("ms", 0.0) + r["phase2"]["ms"] +
                r["phase3"]["ms"] for r in runs]
    steps = [r["phase1"]["path_steps"] + r["phase2"]["path_steps"] + r["phase3"]["path_steps"]
             for r in runs]
    p2 = out["phase2"]
    line = {"metric": METRIC, "value": float(np.sum(steps) / (np.sum(total_ms) * 1e-3)),
            "unit": "path-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(total_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "knots": out["knots"], "eps": x["eps"],
                       "n0": kw["n0"], "h0": x["h0"], "n_job": x["n_job"],
                       "interpolation": out["interpolation"], "rbf_shape": out.get("rbf_shape"),
                       "control_variate": args.cv, "train_steps": args.train_steps,
                       "fit_data": args.fit_data, "train_engine": args.train_engine,
                       "launch": list(kw.get("launch", inspect.signature(calibrated.run)
                                             .parameters["launch"].default)),
                       "note": "path-steps simulated in the three phases (the calibration's "
                               "mixed GM/EM paths once, to their naive exits)"},
            "pipeline": {
                "phase1": {"ms": out["phase1"]["ms"], "path_steps": out["phase1"]["path_steps"],
                           "errors": e1},
                "fit_ms": out.get("fit", {}).get("ms"),
                "phase2": {"ms": p2["ms"], "path_steps": p2["path_steps"],
                           "mean_bias_bound": p2["mean_bias_bound"],
                           "mean_predicted_vrf": p2["mean_predicted_vrf"],
                           "knots_with_h_below_h0": p2["knots_with_h_below_h0"],
                           "N_mean": float(np.mean(p2["N"])), "N_max": int(np.max(p2["N"])),
                           "h_min": float(np.min(p2["h"]))},
                "phase3": {"ms": out["phase3"]["ms"], "path_steps": out["phase3"]["path_steps"],
                           "paths": out["phase3"]["paths"], "errors": e3,
                           "truncated": out["phase3"]["truncated"]},
                "paper": PAPER_E1},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
