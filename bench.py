"""Benchmark: MLMC exp(tA)v to 1e-3 relative error on one GB300.

Workload (the metric's configuration): total communicability x = exp(beta A) 1
of a seeded Barabasi-Albert graph, n = 100000, m = 4, beta = 1/lambda_max
(power iteration), FP32 walk weights with Kahan sums and an FP64 final sum,
4 initial levels above l0 (Eq. 16), relative RMS tolerance 1e-3.

One step = one pass of the whole hot path: rebuild the split quantities and
alias tables on the device from the resident CSR, then mlmc_expmv to the
tolerance (pilot, optimal M_l, top-ups, extra levels, final FP64 sum).  Each
step uses a new seed.  `value` is walk-steps/s (one walk-step = one event =
one holding-time draw; jumps + 1 per walk) over the device-timed steps;
ms_per_step is the time to tolerance.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the paper's Algorithm 2 interval loop,
OpenMP over rows) on bounded samples of the same workload.
N > 1 (torchrun): every rank solves its own replica of the workload with its
own seeds (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "walk-steps/s; time to 1e-3 rel err vs FP64 exp(tA)v, learned vs plain, 1 GB300"
UNIT = "walk-steps/s"
L2_FLUSH_BYTES = 256 << 20


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _workload():
    import mlmc_inputs as I
    return I.workload_c2()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[5 + k].lower() in ("active", "1"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle walker on the host cores (bounded sample)
# ---------------------------------------------------------------------------
def _oracle_sample(w, l0: int, seconds: float = 15.0, seed: int = 1):
    """Time the oracle's Algorithm 2 (OpenMP over rows) on a bounded sample
    of the workload: all levels l0..l0+3 on a growing prefix of the rows,
    one walk per row per level, until ~`seconds` of CPU work is done.
    Returns (events/s, cores, sample description)."""
    from oracle import walker as W
    prec = W.FP32 if w.precision == "fp32" else W.FP64
    wk = W.Walker(w.a, w.t, w.v, seed=seed, precision=prec)
    cores = W.max_threads()
    levels = list(range(l0, l0 + w.num_levels))
    rows = min(w.a.n, 2048)
    events = 0
    elapsed = 0.0
    passes = 0
    while True:
        t0 = time.perf_counter()
        ev = 0
        for l in levels:
            _, _, jumps, _ = wk.mlmcl(l, l > l0, passes, 1, rows=(0, rows))
            ev += jumps + rows
        dt = time.perf_counter() - t0
        events += ev
        elapsed += dt
        passes += 1
        if elapsed >= seconds or passes >= 10000:
            break
        if dt < seconds / 20 and rows < w.a.n:
            rows = min(w.a.n, rows * 2)
    sample = (f"oracle Algorithm 2 (interval loop), levels {levels[0]}-{levels[-1]}, "
              f"{passes} passes of 1 walk per row per level over up to {rows} rows, "
              f"{events} events in {elapsed:.1f} s")
    return events / elapsed, cores, sample


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    from oracle import reference as R
    from oracle import walker as W
    W.build()
    w = _workload()
    tb = W.build_tables(w.a, w.t)
    l0 = R.choose_l0(tb.dl / w.t if w.t > 0 else tb.dl, tb.L, w.t)
    for _ in range(args.warmup):
        _oracle_sample(w, l0, seconds=2.0, seed=99)
    vals, samples = [], []
    t0 = time.perf_counter()
    for k in range(args.steps):
        v, cores, sample = _oracle_sample(w, l0, seconds=args.ref_seconds, seed=k + 1)
        vals.append(v)
        samples.append(sample)
    wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": w.name, "n": w.a.n, "nnz": w.a.nnz,
                                         "t": w.t, "tol": w.tol, "l0": l0},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": samples[-1]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if dist is not None:
        dist.barrier()
    g.build()
    from paper_1904_12754_gb300 import mlmc as M

    w = _workload()
    stream = torch.cuda.current_stream()
    sched = M.schedule_default(precision=M.FP32_KAHAN if w.precision == "fp32" else M.FP64,
                               num_levels=w.num_levels, max_levels=10, pilot_walks=64)
    t_plan = time.perf_counter()
    plan = M.Plan.from_csr(w.a, w.t, sched, rel_tol=w.tol, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t_plan
    info = plan.info()
    n = w.a.n
    dv = torch.from_numpy(w.v).cuda()
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    seed0 = 1_000_003 * (rank + 1)

    # table build alone (a1 + a2), for the record
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.rebuild()
    e1.record(stream)
    torch.cuda.synchronize()
    table_ms = e0.elapsed_time(e1)

    def step(seed):
        plan.rebuild()
        plan.expmv(dv, dx, seed)
        levels, est = plan.stats()
        return levels, est

    for k in range(args.warmup):
        step(seed0 + 7919 * (k + 1))
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = plan.launch_count()
    step_ms, events, walk_s, walk_launch_events, ests, nlevels = [], 0, 0.0, [], [], []
    jumps_total, walks_total = 0, 0
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between steps (256 MB write), outside the timing
        ev_s, ev_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev_s.record(stream)
        levels, est = step(seed0 + k)
        ev_e.record(stream)
        ev_e.synchronize()
        step_ms.append(ev_s.elapsed_time(ev_e))
        for lv in levels:
            walks = lv["walks_per_row"] * n
            events += walks + lv["jumps"]
            jumps_total += lv["jumps"]
            walks_total += walks
            walk_s += lv["seconds"]
        ests.append(est)
        nlevels.append(len(levels))
    t_wall = time.perf_counter() - t_wall
    launches = plan.launch_count() - launches0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()

    total_ms = float(sum(step_ms))
    # whole-job aggregate: sum of events over ranks / max time over ranks
    if dist is not None:
        t = torch.tensor([total_ms, float(events)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_ms_all, events_all = float(tmax[0]), float(t[1])
    else:
        total_ms_all, events_all = total_ms, float(events)
    value = events_all / (total_ms_all * 1e-3)

    # accuracy of the last step against the FP64 judge (CPU baseline leg)
    x_last = dx.cpu().numpy()

    # end to end through the public API with host buffers (pinned): the
    # library copies v in and x out inside mlmc_expmv.
    vh = torch.from_numpy(w.v.copy()).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_events = 0
    t_e2e = time.perf_counter()
    for k in range(args.steps):
        plan.rebuild()
        plan.expmv(vh, xh, seed0 + 500 + k)
        levels, _ = plan.stats()
        e2e_events += sum(lv["walks_per_row"] * n + lv["jumps"] for lv in levels)
    t_e2e = time.perf_counter() - t_e2e
    e2e_value = e2e_events / t_e2e
    if dist is not None:
        t = torch.tensor([t_e2e, float(e2e_events)], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        e2e_value = float(t[1]) / float(tmax[0])

    peaks, peak_kind = _peaks()
    # Walk kernel roofline.  The walk is gather + integer/FP32 ALU work per
    # event; with this workload's tables resident in L2 the issue pipe, not
    # HBM, is the bound.  achieved = warp instructions per
    # event (constant of this kernel build, from the committed ncu profile)
    # x events / walk-kernel time; peak = 152 SMs x 4 schedulers x 1 warp
    # instruction/clock x the SM clock sampled during the run.
    inst_per_event = INST_PER_EVENT_FP32
    walk_launches = sum(nlevels)  # approximate: pilot + top-ups counted below
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_ginst = 152 * 4 * sm_mhz * 1e6 / 1e9
    events_per_s_walk = (events / walk_s) if walk_s > 0 else 0.0
    if inst_per_event:
        achieved = inst_per_event * events_per_s_walk / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_ginst, "unit": "Gwarp-inst/s",
                "frac": achieved / peak_ginst, "traffic": TRAFFIC_PER_EVENT and
                TRAFFIC_PER_EVENT * events / max(1, walk_launch_count(levels, nlevels)),
                "peak_source": f"152 SMs x 4 issue/clk x {sm_mhz:.0f} MHz sampled",
                "inst_per_event": inst_per_event}
    else:
        # gather model: 16 B meta at the start + 8 B v[end] per walk, 16 B
        # alias entry + 16 B meta per jump (FP32 records)
        alg_bytes = 24 * walks_total + 32 * jumps_total
        achieved = alg_bytes / walk_s / 1e9 if walk_s > 0 else 0.0
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "peak_source": f"{peak_kind} hbm_gbs"}
    roof["walk_kernel_events_per_s"] = events_per_s_walk
    roof["walk_kernel_share_of_step"] = (walk_s * 1e3 / total_ms) if total_ms > 0 else None

    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import reference as R
        cv, cores, sample = _oracle_sample(w, info["l0"], seconds=args.ref_seconds)
        t_ref = time.perf_counter()
        ref = R.expmv_taylor(w.a.scipy(), w.t, w.v)
        t_ref = time.perf_counter() - t_ref
        err = float(np.linalg.norm(x_last - ref) / np.linalg.norm(ref))
        cpu = {"value": cv, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "fp64_reference_s": t_ref}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "n": n, "nnz": w.a.nnz, "t": w.t,
                       "lambda_max": w.extra.get("lambda_max"), "tol": w.tol, "l0": info["l0"],
                       "levels_used": nlevels, "precision": "fp32 walk + kahan, fp64 final",
                       "l2": "flushed between steps (256 MB write outside the timed events)",
                       "parallelism": f"replicas{world}" if world > 1 else "1 GPU"},
            "time_to_tol_s": total_ms_all / args.steps / 1e3,
            "est_rel_err": float(np.mean(ests)), "rel_err_vs_fp64": err,
            "table_build_ms": table_ms, "plan_create_s": t_plan,
            "walks_per_step": walks_total / args.steps, "jumps_per_step": jumps_total / args.steps,
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "peaks": {"source": peak_kind, "hbm_gbs": peaks.get("hbm_gbs")},
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


# Warp instructions per event of the FP32 walk kernel and DRAM bytes per
# event, from the ncu capture summarised in profiles/ (None until measured).
INST_PER_EVENT_FP32 = None
TRAFFIC_PER_EVENT = None


def walk_launch_count(levels, nlevels) -> int:
    return max(1, sum(nlevels))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
