"""Benchmark: MLMC exp(tA)v walk-steps/s and time to 1e-3 relative error on
one GB300.

Workload (the metric's configuration): total communicability x = exp(beta A) 1
of a seeded Barabasi-Albert graph, n = 100000, m = 4, beta = 1/lambda_max
(power iteration), FP32 walk weights with Kahan sums and an FP64 final sum,
4 initial levels from l0 (Eq. 16), relative RMS tolerance 1e-3.

One step = one pass of the whole hot path with a new seed: rebuild the split
quantities and alias tables on the device from the resident CSR; learn the
tilt (pilot walks, MLP training on the tensor cores, tilted-clock proposal
tables); mlmc_expmv to the tolerance (pilot, optimal M_l, top-ups, extra
levels, final FP64 sum).  `value` = the solve's walk-steps (one walk-step =
one event = one holding-time draw; jumps + 1 per walk) / the step's time, and
time_to_tol.learned_s = the step time.  With beta = 1/lambda_max the plain
walk's weight e^{beta int d} has a variance that grows like e^{beta d_max}
(hub sojourns; beta d_max = 32 here), so the plain walk is run beside it for a
fixed budget and its time to 1e-3 is projected from the error it reaches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload kernel|batch|learned|precision|levels|complexity|source|forward|c1

--impl reference times the CPU oracle (the paper's Algorithm 2 interval loop,
OpenMP over rows) on bounded samples of the same workload.
N > 1 (torchrun): one problem sharded over the ranks (each rank walks its part
of every level's walks; the level sums are all-reduced before each controller
decision): strong scaling.
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


def _fp64_judge(a, t, v, f=None):
    """FP64 exp(tA)v from the library routine scipy.sparse.linalg.
    expm_multiply (Al-Mohy and Higham's truncated Taylor with scaling), the
    reference each result's error is stated against.  With a constant source
    f: u(t) = exp(tA)v + int_0^t exp(sA)f ds, the first n entries of exp(tB)
    [v; 1] for the augmented B = [[A, f], [0, 0]]."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import expm_multiply
    m = a.scipy().tocsr()
    if f is None:
        return expm_multiply(t * m, np.asarray(v, dtype=np.float64))
    n = m.shape[0]
    b = sp.bmat([[m, sp.csr_matrix(np.asarray(f, dtype=np.float64).reshape(n, 1))],
                 [None, sp.csr_matrix((1, 1))]], format="csr")
    y = expm_multiply(t * b, np.append(np.asarray(v, dtype=np.float64), 1.0))
    return y[:n]


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate_over_ranks(dist, elapsed: float, count: float, device="cpu"):
    """Whole-job figures of a multi-rank run: (max elapsed over ranks, sum of
    counts over ranks).  Without a process group, the rank's own pair."""
    if dist is None:
        return float(elapsed), float(count)
    import torch
    t = torch.tensor([float(elapsed), float(count)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def share_law(plan, dist, rank: int, coll="cpu"):
    """Install rank 0's learned law on every rank of a sharded solve: its
    time pieces K, then its h (K x n), both broadcast from rank 0 (the ranks
    must walk the same law)."""
    import torch
    k = torch.tensor([plan.tilt_pieces()], dtype=torch.int64, device=coll)
    dist.broadcast(k, 0)
    k = int(k.item())
    h = torch.zeros((k, plan.n), dtype=torch.float32, device=coll)
    if rank == 0:
        h.copy_(torch.from_numpy(np.asarray(plan.export_h()).reshape(k, plan.n)))
    dist.broadcast(h, 0)
    hh = h.cpu().numpy() if coll == "cpu" else h
    if k > 1:
        plan.set_tilt_pieces(hh, 0.1)
    else:
        plan.set_tilt(hh.reshape(plan.n), 0.1, clocks=True)


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
def _oracle_sample(w, l0: int, seconds: float = 15.0, seed: int = 1, nthreads: int = 0):
    """Time the oracle's Algorithm 2 (OpenMP over rows) on a bounded sample
    of the workload: all levels l0..l0+3 on a growing prefix of the rows,
    one walk per row per level, until ~`seconds` of CPU work is done.
    Returns (events/s, cores, sample description)."""
    from oracle import walker as W
    prec = W.FP32 if w.precision == "fp32" else W.FP64
    wk = W.Walker(w.a, w.t, w.v, seed=seed, precision=prec)
    cores = nthreads if nthreads > 0 else W.max_threads()
    levels = list(range(l0, l0 + w.num_levels))
    rows = min(w.a.n, 2048)
    events = 0
    elapsed = 0.0
    passes = 0
    while True:
        t0 = time.perf_counter()
        ev = 0
        for l in levels:
            _, _, jumps, _ = wk.mlmcl(l, l > l0, passes, 1, rows=(0, rows), nthreads=nthreads)
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
    # one rank per GPU; with more ranks than GPUs (a host-side gloo check of
    # the sharded path) ranks share devices, whose kernels never wait on
    # one another: the exchange is the host all-reduce
    torch.cuda.set_device(local % torch.cuda.device_count())
    dist = None
    coll = "cuda"
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(args.dist_backend)
        coll = "cuda" if args.dist_backend == "nccl" else "cpu"
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
                               num_levels=w.num_levels, max_levels=10, pilot_walks=64,
                               time_budget_s=args.step_budget)
    t_plan = time.perf_counter()
    plan = M.Plan.from_csr(w.a, w.t, sched, rel_tol=w.tol, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t_plan
    info = plan.info()
    n = w.a.n
    exchange = None
    if dist is not None:
        from paper_1904_12754_gb300.shard import DistExchange
        exchange = DistExchange(plan)        # one problem, sharded over the ranks
    dv = torch.from_numpy(w.v).cuda()
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    seed0 = 1_000_003

    # table build alone (a1 + a2), for the record
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.rebuild()
    e1.record(stream)
    torch.cuda.synchronize()
    table_ms = e0.elapsed_time(e1)

    mlp_launches = [0]
    learn_log = []

    def step(seed, v_in, x_out):
        """One pass of the hot path: tables, learned proposal with tilted
        clocks (pilot walks, MLP training, proposal tables), the MLMC solve
        to the tolerance.  Sharded runs learn on every rank and take rank
        0's h, so that every rank walks the same law."""
        plan.rebuild()
        with M.MLP(seed=3, stream=stream.cuda_stream) as net:
            net.learn_tilt(plan, v_in, seed=seed, pilot_walks=args.pilot, steps=args.mlp_steps,
                           batch=args.mlp_batch, clocks=True, rounds=args.rounds,
                           time_pieces=bool(args.time_pieces))
            mlp_launches[0] += net.launch_count()
        learn_log.append(plan.learn_report() + (plan.tilt_pieces(),))
        if dist is not None:
            share_law(plan, dist, rank, coll)
        rc = plan.expmv(v_in, x_out, seed, allow_not_converged=True)
        levels, est = plan.stats()
        plan.set_tilt(None)
        return rc, levels, est

    log(f"plan created in {t_plan:.2f} s (table build {table_ms:.2f} ms), l0 = {info['l0']}, "
        f"ranks {world}")
    for k in range(args.warmup):
        t0 = time.perf_counter()
        rc, _, est = step(seed0 + 7919 * (k + 1), dv, dx)
        log(f"warm-up {k}: {time.perf_counter() - t0:.2f} s, rc {rc}, est {est:.3g}")
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = plan.launch_count()
    mlp_launches[0] = 0
    step_ms, events, walk_s, ests, nlevels, conv = [], 0, 0.0, [], [], []
    jumps_total, walks_total = 0, 0
    level_log = []
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between steps (256 MB write), outside the timing
        ev_s, ev_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev_s.record(stream)
        rc, levels, est = step(seed0 + k, dv, dx)
        ev_e.record(stream)
        ev_e.synchronize()
        step_ms.append(ev_s.elapsed_time(ev_e))
        for k_l, lv in enumerate(levels):
            walks = lv["walks_per_row"] * n
            events += walks + lv["jumps"]
            jumps_total += lv["jumps"]
            walks_total += walks
            walk_s += lv["seconds"]
            level_log.append(dict(lv, coarse=k_l > 0, walks=walks))
        log(f"step {k}: {step_ms[-1] / 1e3:.3f} s, levels {len(levels)}, rc {rc}, "
            f"est rel err {est:.2e}")
        ests.append(est)
        nlevels.append(len(levels))
        conv.append(rc == 0)
    launches = plan.launch_count() - launches0 + mlp_launches[0]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()

    total_ms = float(sum(step_ms))
    # whole-job aggregate.  Sharded: the walk-steps are counted once (every
    # rank's stats describe the whole solve), the time is the slowest rank's.
    total_ms_all, _ = aggregate_over_ranks(dist, total_ms, events, coll)
    value = events / (total_ms_all * 1e-3)
    x_last = dx.cpu().numpy()

    # end to end through the public API with host buffers (pinned): v is
    # copied in by the learning and the solve, x out by the solve
    vh = torch.from_numpy(w.v.copy()).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_events = 0
    t_e2e = time.perf_counter()
    for k in range(args.steps):
        _, levels, _ = step(seed0 + 500 + k, vh, xh)
        e2e_events += sum(lv["walks_per_row"] * n + lv["jumps"] for lv in levels)
    t_e2e = time.perf_counter() - t_e2e
    log(f"e2e: {t_e2e:.2f} s for {args.steps} step(s)")
    t_e2e_all, _ = aggregate_over_ranks(dist, t_e2e, e2e_events, coll)
    e2e_value = e2e_events / t_e2e_all

    peaks, peak_kind = _peaks()
    # the law of the last timed step: the capture constants describe the
    # one-law kernel and the 8-piece one (a law with time pieces runs its
    # own variant)
    pieces = learn_log[args.warmup + args.steps - 1][2]
    roof = walk_roofline(level_log, walk_s, clocks, peaks, total_ms, proposal=True,
                         capture=w.name.startswith("ba_n100000_m4") and (
                             pieces == 1 or (pieces == 8 and PIECES_CAPTURE_CURRENT)),
                         pieces=pieces)

    # The plain walk on the same plan and budget: its error estimate after
    # the budget, and the time 1e-3 would take at its measured variance
    # (the error falls like 1/sqrt(time)).
    sched_p = M.schedule_default(precision=M.FP32_KAHAN if w.precision == "fp32" else M.FP64,
                                 num_levels=w.num_levels, max_levels=10, pilot_walks=64,
                                 time_budget_s=args.plain_budget)
    with M.Plan.from_csr(w.a, w.t, sched_p, rel_tol=w.tol, stream=stream.cuda_stream) as plan_p:
        if exchange is not None:
            exchange.attach(plan_p)
        sec_p, est_p, conv_p, ev_p = _timed_solve(plan_p, dv, dx, seed0 + 777)
    plain = {"budget_s": args.plain_budget, "seconds": sec_p, "est_rel_err": est_p,
             "converged": conv_p, "walk_steps_per_s": ev_p / sec_p,
             "projected_time_to_tol_s": sec_p * (est_p / w.tol) ** 2,
             "projection": "seconds x (est_rel_err / tol)^2 at the measured variance; a lower "
                           "bound here: the plain walk's heavy-tailed weights make its own error "
                           "estimate unreliable"}
    log(f"plain: {sec_p:.2f} s, est {est_p:.3g}, projected {plain['projected_time_to_tol_s']:.3g} s")

    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cv, cores, sample = _oracle_sample(w, info["l0"], seconds=args.ref_seconds)
        cv1, _, sample1 = _oracle_sample(w, info["l0"], seconds=5.0, seed=2, nthreads=1)
        _oracle_sample(w, info["l0"], seconds=0.1, seed=3, nthreads=cores)  # restore the thread count
        t_ref = time.perf_counter()
        ref = _fp64_judge(w.a, w.t, w.v)
        t_ref = time.perf_counter() - t_ref
        err = float(np.linalg.norm(x_last - ref) / np.linalg.norm(ref))
        cpu = {"value": cv, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "fp64_reference_s": t_ref, "single_thread_value": cv1,
               "single_thread_sample": sample1}

    if rank == 0:
        tt = [ms / 1e3 for ms in step_ms]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps,
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n": n, "nnz": w.a.nnz, "t": w.t,
                       "lambda_max": w.extra.get("lambda_max"), "tol": w.tol, "l0": info["l0"],
                       "levels_used": nlevels, "precision": "fp32 walk + kahan, fp64 final",
                       "step": "table build + learned tilted proposal (pilot walks, MLP "
                               "training, proposal tables) + MLMC solve to the tolerance",
                       "learning": {"rounds": args.rounds, "pilot_walks": args.pilot,
                                    "mlp_steps": args.mlp_steps, "mlp_batch": args.mlp_batch,
                                    "alpha": 0.1,
                                    "time_piece_candidates": bool(args.time_pieces),
                                    "chosen_law_per_timed_step": [
                                        c for c, _, _ in learn_log[args.warmup:args.warmup + args.steps]],
                                    "time_pieces_per_timed_step": [
                                        k for _, _, k in learn_log[args.warmup:args.warmup + args.steps]],
                                    "pilot_var_per_walk_last_timed_step":
                                        learn_log[args.warmup + args.steps - 1][1]},
                       "l2": "flushed between steps (256 MB write outside the timed events)",
                       "parallelism": f"shard{world}" if world > 1 else "1 GPU"},
            "time_to_tol": {"learned_s": statistics.median(tt), "learned_runs_s": tt,
                            "learned_converged": all(conv),
                            "learned_est_rel_err": float(np.mean(ests)),
                            "learned_rel_err_vs_fp64": err,
                            "plain_s": None, "plain": plain},
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


# ---------------------------------------------------------------------------
# Walk-kernel roofline: ALU (issue) bound with this workload's tables in L2.
# Algorithmic operations of the FP32 walk, counted from the kernel source
# (each integer/FP32 operation, compare, select, load, exp = 1):
#   Philox draw   42  (10 rounds x 2 wide multiplies and 2 three-input xors, 2
#                     counter words; the round keys are formed once per launch).
#                     The FP32 layout needs one draw per jump plus one
#                     block per four walks for their first holding times
#                     (rows with 1/(tL) >= 1, nearly all rows here; a walk in
#                     another row that never jumps also draws once, which
#                     this count leaves out)
#   holding time  31  (uniform 4; -ln(u) 24: range reduction 10, degree-8
#                     polynomial 10, ln 2 terms 4; scale + add + compare 3), for
#                     every event except the first of a walk that never jumps
#   still test     2  per walk: the first uniform's index against the row's
#                     threshold index
#   every jump    22 (levels above l0) / 15 (l0): grid index, counts, bucket,
#                 alias gather and select, sign, next-state gather
#   walk end      31 / 24 for a walk that jumped (exponents, exp/expm1, Kahan
#                 and pair sums); 1 for a walk that never jumped
# peak = SMs x 128 lanes x SM clock (one operation per lane per clock), the SM
# count read from the device.
# ---------------------------------------------------------------------------
OPS_DRAW = 42
OPS_HOLD = 31
OPS_STILL_TEST = 2
OPS_JUMP = {True: 22, False: 15}
OPS_END_JUMPED = {True: 31, False: 24}
OPS_END_STILL = 1
# A proposal walk's jump also loads the entry's log-ratios and adds one to
# the exponent (the row record comes from the record table, not the entry).
OPS_JUMP_PROPOSAL = 2
# From one ncu capture (--set full, one launch) of the proposal walk kernel
# on this workload: a launch of 4.1e8 walks at l0 (4096 per row, 5.22e8
# events) after an L2 flush, with the learned tilted clocks.  DRAM bytes per
# launch (the proposal tables are read once, everything else hits L2: 98.3%),
# issue-slot use and instructions per event.  Set to None when the kernel
# changes.
TRAFFIC_CAPTURE = 28.834e6
ISSUE_CAPTURE = {"issue_active": 0.761, "threads_per_instruction": 26.78,
                 "warp_instructions_per_event": 3.10, "l2_hit": 0.983,
                 "dram_bytes_per_event": 0.055, "launch_ms": 1.755,
                 "capture": "k_walk<FP32, proposal> at l0, BA n=1e5, 4096 walks per row, "
                            "bench.py --workload kernel --kernel-tilt --time-pieces 0"}
# The same capture of the walk with the learned law of 8 time pieces (the law
# the default step installs on this graph): the same launch (4.1e8 walks,
# 1.16e8 jumps, 5.26e8 events).  Its 8 table sets (218 MB) exceed L2, so
# the tables are read from DRAM about five times over.  Taken before the
# pieces' row records were stored state-major: not reported for the present
# kernel (PIECES_CAPTURE_CURRENT).
PIECES_CAPTURE_CURRENT = False
TRAFFIC_CAPTURE_PIECES = 1.278e9
ISSUE_CAPTURE_PIECES = {"issue_active": 0.701, "threads_per_instruction": 17.50,
                        "warp_instructions_per_event": 8.71, "l2_hit": 0.891,
                        "dram_bytes_per_event": 2.43, "launch_ms": 5.816,
                        "capture": "k_walk<FP32, proposal, 8 time pieces> at l0, BA n=1e5, 4096 "
                                   "walks per row, bench.py --workload kernel --kernel-tilt"}


def walk_roofline(level_log, walk_s, clocks, peaks, total_ms, num_sms=None, proposal=False,
                  capture=False, pieces=1):
    """capture: the capture constants above describe this kernel and workload.
    pieces: the time pieces of the proposal (its carry-overs are not in the
    op model, so the ops per event are a lower bound with pieces > 1)."""
    ops = 0.0
    events = 0
    launches = 0
    gather = 0.0
    for lv in level_log:
        c = lv["coarse"]
        ev = lv["walks"] + lv["jumps"]
        still = lv.get("still_walks", 0)
        ops += OPS_DRAW * (lv["jumps"] + lv["walks"] / 4.0) + OPS_HOLD * (ev - still) \
            + OPS_STILL_TEST * lv["walks"] \
            + (OPS_JUMP[c] + (OPS_JUMP_PROPOSAL if proposal else 0)) * lv["jumps"] \
            + OPS_END_JUMPED[c] * (lv["walks"] - still) + OPS_END_STILL * still
        # table gathers: alias entry + the new state's row record per jump,
        # v at the end state per walk that jumped (FP32 layout); a proposal
        # entry adds its two log-ratios (8 B)
        gather += (40.0 if proposal else 32.0) * lv["jumps"] + 4.0 * (lv["walks"] - still)
        events += ev
        launches += lv.get("launches", 0)
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if num_sms is None:
        import torch
        num_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = num_sms * 128 * sm_mhz * 1e6 / 1e9
    achieved = ops / walk_s / 1e9 if walk_s > 0 else 0.0
    hbm = peaks.get("hbm_gbs")
    gather_gbs = gather / walk_s / 1e9 if walk_s > 0 else 0.0
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
            "frac": achieved / peak if peak else None,
            "traffic": (TRAFFIC_CAPTURE_PIECES if pieces == 8 else TRAFFIC_CAPTURE) if capture else None,
            "traffic_per": ("launch of 4.1e8 walks at l0 after an L2 flush (the capture's launch)"
                            if capture else None),
            "kernel": "k_walk<FP32%s%s> (mlmc_walk.cu)" % (
                ", proposal" if proposal else "",
                f", {pieces} time pieces" if pieces > 1 else ""),
            "peak_source": f"{num_sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (SM count of the device, "
                           "median SM clock sampled in the run)",
            "issue": (ISSUE_CAPTURE_PIECES if pieces == 8 else ISSUE_CAPTURE) if capture else None,
            "ops_per_event": ops / events if events else None,
            "walk_launches": launches,
            "avg_launch_ms": 1e3 * walk_s / launches if launches else None,
            "walk_events_per_s": events / walk_s if walk_s > 0 else None,
            "walk_kernel_share_of_step_time": (1e3 * walk_s / total_ms) if total_ms > 0 else None,
            "gather": {"achieved": gather_gbs, "unit": "GB/s", "peak": hbm,
                       "peak_source": "HBM copy of measured (the tables are L2-resident here)",
                       "frac": gather_gbs / hbm if hbm else None,
                       "bytes_per_event": gather / events if events else None}}


def log(msg: str):
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# Secondary workload: batching (256 Laplacian instances, 1-8 right-hand sides)
# ---------------------------------------------------------------------------
def run_batch_workload(args):
    """Batched solver against a loop of single-plan solves on the same
    inputs (every instance and right-hand side, same seeds, same tolerance).
    Prints one JSON line; not the default benchmark."""
    import torch
    import mlmc_inputs as I
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    stream = torch.cuda.current_stream()
    inst = I.workload_c3(n_hi=args.batch_nmax)
    tol = args.tol
    sched = M.schedule_default(precision=M.FP32_KAHAN, num_levels=3, max_levels=10, pilot_walks=64,
                               time_budget_s=600.0)
    plans, probs = [], []
    t0 = time.perf_counter()
    for w, rhs in inst:
        p = M.Plan.from_csr(w.a, w.t, sched, rel_tol=tol, stream=stream.cuda_stream)
        plans.append(p)
        for r in range(rhs.shape[0]):
            probs.append((p, torch.from_numpy(np.ascontiguousarray(rhs[r])).cuda()))
    torch.cuda.synchronize()
    t_plans = time.perf_counter() - t0
    rows = sum(p.n for p in plans)
    log(f"{len(plans)} instances, {len(probs)} problems, {rows} rows; plans in {t_plans:.1f} s")
    xs = [torch.zeros(p.n, dtype=torch.float64, device="cuda") for p, _ in probs]
    seeds = [7 + 13 * k for k in range(len(probs))]

    def events_of(levels, n):
        return sum(lv["walks_per_row"] * n + lv["jumps"] for lv in levels)

    # plain: one mlmc_expmv per problem
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_events, plain_conv = 0, 0
    for k, (p, v) in enumerate(probs):
        rc = p.expmv(v, xs[k], seeds[k], allow_not_converged=True)
        lv, _ = p.stats()
        plain_events += events_of(lv, p.n)
        plain_conv += rc == 0
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    log(f"plain loop: {t_plain:.2f} s, {plain_conv}/{len(probs)} converged")
    # batched
    t0 = time.perf_counter()
    batch = M.Batch([p for p, _ in probs], sched, rel_tol=tol, stream=stream.cuda_stream)
    t_create = time.perf_counter() - t0
    batch.expmv([v for _, v in probs], xs, seeds, allow_not_converged=True)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.expmv([v for _, v in probs], xs, seeds, allow_not_converged=True)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    info = batch.info()
    batch_events = sum(events_of(batch.stats(k)[0], p.n) for k, (p, _) in enumerate(probs))
    ests = [batch.stats(k)[1] for k in range(len(probs))]
    log(f"batch: {t_batch:.2f} s, {info['rounds']} rounds, {info['converged']}/{len(probs)} converged")
    line = {"metric": "time to per-instance rel. RMS tolerance, batched vs plain", "unit": "s",
            "value": t_batch, "higher_is_better": False, "n_gpus": 1, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"256 Laplacian instances (2D/3D), n log-uniform in "
                                   f"[1e3, {args.batch_nmax:g}], t ~ U[0.1, 2], 1-8 right-hand sides",
                       "tol": tol,
                       "problems": len(probs), "rows": rows},
            "batched": {"seconds": t_batch, "walk_steps_per_s": batch_events / t_batch,
                        "rounds": info["rounds"], "gpu_seconds": info["gpu_seconds"],
                        "converged": info["converged"], "max_est_rel_err": max(ests),
                        "create_s": t_create, "walks_per_lane_by_bucket": batch.autotune(),
                        "round_kernel_block": batch.block()},
            "plain": {"seconds": t_plain, "walk_steps_per_s": plain_events / t_plain,
                      "converged": plain_conv},
            "speedup": t_plain / t_batch}
    print(json.dumps(line), flush=True)
    batch.close()
    for p in plans:
        p.close()


# ---------------------------------------------------------------------------
# Secondary workloads: learned proposal, precision path
# ---------------------------------------------------------------------------
def _level0_variance(plan, v_dev, reps, seed):
    import torch
    n = plan.n
    s = torch.zeros(n, dtype=torch.float64, device="cuda")
    tot = torch.zeros(8, dtype=torch.float64, device="cuda")
    plan.mlmcl(plan.info()["l0"], False, 1 << 40, reps, v_dev, seed, s, tot)
    torch.cuda.synchronize()
    sv = s.cpu().numpy()
    y2 = float(tot[0])
    return (y2 - float(sv @ sv) / reps) / (reps - 1), float(np.linalg.norm(sv / reps))


def _timed_solve(plan, v_dev, x_dev, seed):
    import torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = plan.expmv(v_dev, x_dev, seed, allow_not_converged=True)
    e1.record(stream)
    e1.synchronize()
    levels, est = plan.stats()
    events = sum(lv["walks_per_row"] * plan.n + lv["jumps"] for lv in levels)
    return e0.elapsed_time(e1) / 1e3, est, rc == 0, events


def run_learned_workload(args):
    """The learned proposal with tilted clocks (mlmc_learn_tilt) against the
    plain walk on the same inputs: time to the tolerance, learning included,
    and the error against the FP64 judge.  A plain solve that stops at its
    budget reports its projected time (budget x (estimated error / tol)^2)."""
    import torch
    import mlmc_inputs as I
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    st = torch.cuda.current_stream().cuda_stream
    out = {"metric": "time to rel. RMS tolerance, learned tilted proposal vs plain MLMC",
           "n_gpus": 1, "dtype": "f32", "data": "synthetic", "workloads": {}}

    def one(w, tol, plain_budget, learned_budget, name):
        log(f"{name}: n={w.a.n} nnz={w.a.nnz}")
        ref = _fp64_judge(w.a, w.t, w.v)
        nref = np.linalg.norm(ref)
        dv = torch.from_numpy(w.v).cuda()
        dx = torch.zeros(w.a.n, dtype=torch.float64, device="cuda")
        res = {"tol": tol}
        sched = M.schedule_default(precision=M.FP32_KAHAN, num_levels=4, max_levels=10,
                                   time_budget_s=plain_budget)
        with M.Plan.from_csr(w.a, w.t, sched, rel_tol=tol, stream=st) as plan:
            var_p, _ = _level0_variance(plan, dv, 64, 11)
            tp, ep, cp, evp = _timed_solve(plan, dv, dx, 21)
            xp = dx.cpu().numpy()
        res["plain"] = {"seconds": tp, "est_rel_err": ep, "converged": cp,
                        "rel_err_vs_fp64": float(np.linalg.norm(xp - ref) / nref),
                        "walk_steps_per_s": evp / tp, "level0_var_per_walk": var_p,
                        "time_to_tol_s": tp if cp else None,
                        "projected_time_to_tol_s": tp * (ep / tol) ** 2}
        sched = M.schedule_default(precision=M.FP32_KAHAN, num_levels=4, max_levels=10,
                                   time_budget_s=learned_budget)
        runs = []
        with M.Plan.from_csr(w.a, w.t, sched, rel_tol=tol, stream=st) as plan:
            for rep in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                with M.MLP(seed=3, stream=st) as net:
                    loss = net.learn_tilt(plan, dv, seed=5 + rep, pilot_walks=args.pilot,
                                          steps=args.mlp_steps, batch=args.mlp_batch, clocks=True,
                                          rounds=args.rounds, time_pieces=bool(args.time_pieces))
                torch.cuda.synchronize()
                t_learn = time.perf_counter() - t0
                chosen, pilot_var = plan.learn_report()
                var_l, _ = _level0_variance(plan, dv, 64, 11)
                tl, el, cl, evl = _timed_solve(plan, dv, dx, 31 + rep)
                xl = dx.cpu().numpy()
                runs.append({"learn_s": t_learn, "solve_s": tl, "time_to_tol_s": t_learn + tl,
                             "est_rel_err": el, "converged": cl, "train_loss": loss,
                             "rel_err_vs_fp64": float(np.linalg.norm(xl - ref) / nref),
                             "level0_var_per_walk": var_l, "walk_steps_per_s": evl / tl,
                             "pilot_var_per_walk": pilot_var, "chosen_law": chosen,
                             "time_pieces": plan.tilt_pieces()})
                log(f"{name} learned run {rep}: {t_learn:.2f} + {tl:.2f} s, est {el:.3g}, "
                    f"converged {cl}")
                plan.set_tilt(None)
        res["learned"] = runs
        conv = [r["time_to_tol_s"] for r in runs if r["converged"]]
        res["learned_median_time_to_tol_s"] = statistics.median(conv) if conv else None
        res["learned_converged_runs"] = len(conv)
        ref_t = res["plain"]["time_to_tol_s"] or res["plain"]["projected_time_to_tol_s"]
        if conv:
            res["speedup_incl_learning"] = ref_t / statistics.median(conv)
        out["workloads"][name] = res
        log(f"{name}: plain {tp:.2f} s (est {ep:.3g}), learned median "
            f"{res['learned_median_time_to_tol_s']}")
        return res

    c5 = one(I.workload_c5(), 1e-3, args.plain_budget, args.step_budget,
             "ba_n1e6_m8_beta_inv_lambda_max")
    c4 = one(I.workload_c4(), 1e-3, 300.0, 300.0, "convdiff3d_128_bump")
    out["value"] = c5.get("learned_median_time_to_tol_s")
    out["unit"] = "s (learned time to 1e-3 on BA n=1e6 m=8, learning included)"
    out["higher_is_better"] = False
    print(json.dumps(out), flush=True)


def run_precision_workload(args):
    """FP32 + Kahan walk against the all-FP64 walk on the convection-
    diffusion workload, each with its error against the FP64 Taylor judge."""
    import torch
    import mlmc_inputs as I
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    st = torch.cuda.current_stream().cuda_stream
    w = I.workload_c4()
    ref = _fp64_judge(w.a, w.t, w.v)
    nref = np.linalg.norm(ref)
    dv = torch.from_numpy(w.v).cuda()
    dx = torch.zeros(w.a.n, dtype=torch.float64, device="cuda")
    res = {}
    for name, prec in (("fp32_kahan", M.FP32_KAHAN), ("fp64", M.FP64)):
        sched = M.schedule_default(precision=prec, num_levels=4, max_levels=10,
                                   time_budget_s=args.step_budget)
        with M.Plan.from_csr(w.a, w.t, sched, rel_tol=args.tol, stream=st) as plan:
            sec, est, conv, events = _timed_solve(plan, dv, dx, 7)
            levels, _ = plan.stats()
        x = dx.cpu().numpy()
        res[name] = {"seconds": sec, "walk_steps_per_s": events / sec, "est_rel_err": est,
                     "converged": conv, "rel_err_vs_fp64_taylor": float(np.linalg.norm(x - ref) / nref),
                     "levels": len(levels)}
        log(f"{name}: {sec:.2f} s, est {est:.3g}, err {res[name]['rel_err_vs_fp64_taylor']:.3g}")
    out = {"metric": "precision path: FP32+Kahan vs FP64 walk, error vs FP64 Taylor",
           "config": {"workload": w.name, "n": w.a.n, "nnz": w.a.nnz, "t": w.t, "tol": args.tol},
           "n_gpus": 1, "data": "synthetic", **res,
           "value": res["fp64"]["seconds"] / res["fp32_kahan"]["seconds"],
           "unit": "x (FP64 time / FP32 time)", "higher_is_better": True}
    print(json.dumps(out), flush=True)


def run_kernel_workload(args):
    """The walk kernel alone (Algorithm 2's MLMCL launch, mlmc_mlmcl): the
    metric's graph and precision, 4096 walks per row at l0 (about 4e8 walks
    in one launch) and at l0 + 1 (coarse-coupled), each launch timed with
    CUDA events on the plan's stream after an L2 flush.  This is the burst
    figure of the dominant kernel and the command the kernel profiles run."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    import mlmc_inputs as I
    if args.kernel_matrix == "lap3d":
        # long walks: unscaled 7-point Laplacian, t L_ii = 6 (about 7 events
        # per walk), the instance family of the batched workload
        a = I.laplacian_3d(64)
        w = I.Workload(name="lap3d_g64_t1_fp32", a=a, t=1.0, v=I.uniform_v(a.n, 20190429),
                       precision="fp32", num_levels=3, tol=1e-3, extra={})
    elif args.kernel_matrix == "c4":
        w = I.workload_c4()          # FP32 tables ~233 MB: larger than L2
    elif args.kernel_matrix == "c5":
        w = I.workload_c5()          # FP32 tables ~272 MB: larger than L2
    else:
        w = _workload()
    w.precision = args.kernel_precision
    stream = torch.cuda.current_stream()
    sched = M.schedule_default(precision=M.FP32_KAHAN if w.precision == "fp32" else M.FP64,
                               walks_per_lane=args.walks_per_lane, block_threads=args.block,
                               l2_persist=args.l2_persist)
    plan = M.Plan.from_csr(w.a, w.t, sched, rel_tol=w.tol, stream=stream.cuda_stream)
    l0 = plan.info()["l0"]
    n = w.a.n
    dv = torch.from_numpy(w.v).cuda()
    if args.kernel_tilt:
        # the walk the default workload's solve runs: learned tilted clocks
        with M.MLP(seed=3, stream=stream.cuda_stream) as net:
            net.learn_tilt(plan, dv, seed=5, pilot_walks=args.pilot, steps=args.mlp_steps,
                           batch=args.mlp_batch,
                           clocks=True, rounds=args.rounds, time_pieces=bool(args.time_pieces))
    l2win = plan.l2_window()
    sums = torch.zeros(n, dtype=torch.float64, device="cuda")
    tot = torch.zeros(5, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    reps = args.kernel_reps
    res = {}
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    for name, level, coarse in (("l0", l0, False), ("l0+1", l0 + 1, True)):
        for k in range(args.warmup):
            plan.mlmcl(level, coarse, 0, reps, dv, 11 + k, sums, tot)
        torch.cuda.synchronize()
        ms, events, jumps, walks, still = [], 0.0, 0.0, 0.0, 0.0
        for k in range(args.steps):
            flush.fill_(float(k))
            tot.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.mlmcl(level, coarse, reps * (k + 1), reps, dv, 1000 + k, sums, tot)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            t = tot.cpu().numpy()
            jumps += t[1]
            walks += t[2]
            still += t[4]
        events = walks + jumps
        total_s = 1e-3 * sum(ms)
        res[name] = {"level": level, "coarse": coarse, "walks_per_row": reps,
                     "launch_ms": ms, "walks": walks / args.steps, "jumps": jumps / args.steps,
                     "still_walks": still / args.steps, "events_per_s": events / total_s}
        log(f"{name}: {statistics.median(ms):.3f} ms per launch, {events / total_s:.4g} events/s")
    clocks = sampler.stop()
    peaks, _ = _peaks()
    lv = [dict(coarse=False, walks=res["l0"]["walks"], jumps=res["l0"]["jumps"],
               still_walks=res["l0"]["still_walks"], launches=1)]
    # the op model and its ALU peak describe the FP32 walk; the FP64 walk is
    # bound by the FP64 pipe (its counters are in the kernel's ncu summary)
    pieces = plan.tilt_pieces() if args.kernel_tilt else 1
    roof = walk_roofline(lv, 1e-3 * statistics.mean(res["l0"]["launch_ms"]), clocks, peaks,
                         statistics.mean(res["l0"]["launch_ms"]), proposal=args.kernel_tilt,
                         capture=args.kernel_tilt and args.kernel_matrix == "ba" and (
                             pieces == 1 or (pieces == 8 and PIECES_CAPTURE_CURRENT)),
                         pieces=pieces) if w.precision == "fp32" else None
    out = {"metric": "walk kernel alone: walk-steps/s at l0 (one launch, L2 flushed before it)",
           "value": res["l0"]["events_per_s"], "unit": UNIT, "higher_is_better": True,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "dtype": "f32" if w.precision == "fp32" else "f64",
           "data": "synthetic",
           "config": {"workload": w.name, "n": n, "nnz": w.a.nnz, "t": w.t, "l0": l0,
                      "walks_per_row": reps, "l2": "flushed before each launch",
                      "walks_per_lane": args.walks_per_lane or "default",
                      "block": args.block or "default", "l2_window": l2win,
                      "walk": "learned tilted clocks and jumps" if args.kernel_tilt else "plain",
                      "precision": w.precision},
           "levels": res, "roofline": roof, "clocks": clocks}
    print(json.dumps(out), flush=True)
    plan.close()

# ---------------------------------------------------------------------------
# Level statistics and complexity (the paper's Fig. 2, Fig. 4 and Fig. 5)
# ---------------------------------------------------------------------------
def _slope(xs, ys):
    xs, ys = np.asarray(xs, float), np.asarray(ys, float)
    ok = np.isfinite(ys)
    if ok.sum() < 2:
        return None
    return float(np.polyfit(xs[ok], ys[ok], 1)[0])


def run_levels_workload(args):
    """m_l and V_l of the coupled corrections P_l - P_{l-1} against the level
    (Fig. 2): total communicability (v = 1, beta = 1) of Newman-Watts
    small-world networks (k = 2, p = 0.1) of three sizes, FP64 walks, a fixed
    number of walks per row at every level (one mlmc_mlmcl launch each).
    Reported per level: the mean correction per row (1^T m_l / n) and the
    per-row variance V_l, with least-squares slopes of their log2 over the
    finer levels (the paper's analysis: both -2)."""
    import torch
    import mlmc_inputs as I
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    stream = torch.cuda.current_stream()
    out = {"metric": "MLMC level statistics m_l, V_l vs level (TC of small-world networks)",
           "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "Newman-Watts small world k=2 p=0.1, beta=1, v=1, FP64 walk",
                      "levels": list(range(0, args.max_level + 1))}, "networks": {}}
    for n, reps in ((10 ** 4, 8192), (10 ** 5, 1024), (10 ** 6, 128)):
        a = I.small_world(n, 2, 0.1, seed=20190429)
        sched = M.schedule_default(precision=M.FP64)
        plan = M.Plan.from_csr(a, 1.0, sched, rel_tol=1e-3, stream=stream.cuda_stream)
        dv = torch.ones(n, dtype=torch.float64, device="cuda")
        sums = torch.zeros(n, dtype=torch.float64, device="cuda")
        tot = torch.zeros(5, dtype=torch.float64, device="cuda")
        rows = []
        for lvl in range(0, args.max_level + 1):
            sums.zero_()
            tot.zero_()
            t0 = time.perf_counter()
            plan.mlmcl(lvl, lvl > 0, 0, reps, dv, 77 + lvl, sums, tot)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            sv = sums.cpu().numpy()
            t = tot.cpu().numpy()
            mean = float(sv.sum() / (n * reps))
            var = float((t[0] - float((sv * sv).sum()) / reps) / (reps - 1) / n)
            rows.append({"level": lvl, "m_l": mean, "V_l": var, "walks": int(t[2]),
                         "jumps": int(t[1]), "seconds": sec})
        fine = [r for r in rows if r["level"] >= 3]
        lv = [r["level"] for r in fine]
        out["networks"][f"n={n}"] = {
            "n": n, "nnz": a.nnz, "max_degree": int(np.diff(a.row_ptr).max()),
            "walks_per_row": reps, "levels": rows,
            "slope_log2_abs_m_l": _slope(lv, [np.log2(abs(r["m_l"])) if r["m_l"] else np.nan for r in fine]),
            "slope_log2_V_l": _slope(lv, [np.log2(r["V_l"]) if r["V_l"] > 0 else np.nan for r in fine])}
        log(f"n={n}: slopes m_l {out['networks'][f'n={n}']['slope_log2_abs_m_l']}, "
            f"V_l {out['networks'][f'n={n}']['slope_log2_V_l']}")
        plan.close()
    print(json.dumps(out), flush=True)


def run_complexity_workload(args):
    """Time to tolerance of MLMC and of single-level Monte Carlo (Fig. 5) and
    the MLMC time against the initial level l0 (Fig. 4), on total and single
    node communicability (beta = 1, v = 1) of a Newman-Watts small-world
    network with n = 1e6, FP32 walks.  The single-level run uses the finest
    level the MLMC run reached at the same tolerance (the same splitting-bias
    budget).  Besides GPU seconds, the cost is given in the paper's units
    (Eq. 14: sum over levels of M_l (N_l + jumps)), where the interval loop
    makes a fine level expensive; the event-driven walk's cost per walk does
    not grow with the level."""
    import torch
    import mlmc_inputs as I
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    stream = torch.cuda.current_stream()
    n = 10 ** 6
    a = I.small_world(n, 2, 0.1, seed=20190429)
    dv = torch.ones(n, dtype=torch.float64, device="cuda")
    node = 0

    def solve(target, tol, l0=-1, levels=3, max_levels=12, seed=5):
        sched = M.schedule_default(precision=M.FP32_KAHAN, num_levels=levels, max_levels=max_levels,
                                   time_budget_s=60.0)
        if l0 >= 0:
            sched.l0 = l0
        with M.Plan.from_csr(a, 1.0, sched, rel_tol=tol, stream=stream.cuda_stream) as plan:
            best = None
            for rep in range(3):  # first solve warms up; keep the fastest of the others
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if target == "entry":
                    val = plan.expmv_entry(node, dv, seed=seed + rep, allow_not_converged=True)
                else:
                    val = plan.expmv_sum(dv, seed=seed + rep, allow_not_converged=True)
                sec = time.perf_counter() - t0
                lv, est = plan.stats()
                rows = 1 if target == "entry" else n
                walks = sum(l["walks_per_row"] for l in lv) * rows
                paper_cost = sum(l["walks_per_row"] * rows * (2 ** l["level"]) + l["jumps"] for l in lv)
                rec = {"seconds": sec, "value": val, "est_rel_err": est, "levels": [l["level"] for l in lv],
                       "walks": walks, "paper_cost_units": paper_cost,
                       "events": sum(l["walks_per_row"] * rows + l["jumps"] for l in lv)}
                if rep > 0 and (best is None or sec < best["seconds"]):
                    best = rec
            return best

    tols = [1e-2, 5e-3, 2.5e-3, 1.25e-3, 6.25e-4]
    fig5 = {}
    for target in ("entry", "sum"):
        res = []
        for tol in tols:
            ml = solve(target, tol)
            finest = max(ml["levels"])
            mc = solve(target, tol, l0=finest, levels=1, max_levels=1)
            res.append({"tol": tol, "mlmc": ml, "mc_single_level": dict(mc, level=finest)})
            log(f"{target} tol {tol:g}: MLMC {ml['seconds']:.4f} s (levels {ml['levels']}), "
                f"MC at level {finest} {mc['seconds']:.4f} s")
        lt = np.log10(tols)
        fig5[target] = {
            "runs": res,
            "slope_log10_seconds": {"mlmc": _slope(lt, [np.log10(r["mlmc"]["seconds"]) for r in res]),
                                    "mc": _slope(lt, [np.log10(r["mc_single_level"]["seconds"]) for r in res])},
            "slope_log10_paper_cost": {
                "mlmc": _slope(lt, [np.log10(r["mlmc"]["paper_cost_units"]) for r in res]),
                "mc": _slope(lt, [np.log10(r["mc_single_level"]["paper_cost_units"]) for r in res])},
            "slope_log10_events": {
                "mlmc": _slope(lt, [np.log10(r["mlmc"]["events"]) for r in res]),
                "mc": _slope(lt, [np.log10(r["mc_single_level"]["events"]) for r in res])}}
    fig4 = []
    for l0 in range(0, 8):
        r = solve("sum", 6.25e-4, l0=l0)
        fig4.append(dict(r, l0=l0))
        log(f"l0 sweep: l0={l0} {r['seconds']:.4f} s, levels {r['levels']}")
    tb_l0 = None
    with M.Plan.from_csr(a, 1.0, M.schedule_default(precision=M.FP32_KAHAN), rel_tol=1e-3,
                         stream=stream.cuda_stream) as plan:
        tb_l0 = plan.info()["l0"]
    out = {"metric": "MLMC vs single-level MC time to tolerance; MLMC time vs l0",
           "n_gpus": 1, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "Newman-Watts small world n=1e6 k=2 p=0.1, beta=1, v=1",
                      "nnz": a.nnz, "max_degree": int(np.diff(a.row_ptr).max()), "entry_node": node,
                      "l0_eq16": tb_l0},
           "fig5_time_vs_tol": fig5, "fig4_time_vs_l0": fig4}
    print(json.dumps(out), flush=True)



def run_source_workload(args):
    """The inhomogeneous problem du/dt = A u + F, u(0) = v (Sec. 5, Algorithm
    3): the convection-diffusion operator of the precision workload on a 64^3
    grid, v the Gaussian bump, F = 1 (a uniform load), t ||A||_inf = 8, FP32
    walks, tolerance --tol.  The same plan solves it without the source
    (exp(tA)v) and with it (mlmc_plan_set_source); both against the FP64
    judge (Taylor, the integral from the sparse augmented matrix)."""
    import torch
    import mlmc_inputs as I
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    stream = torch.cuda.current_stream()
    a = I.convdiff_3d(64)
    t = 8.0 / float(abs(a.scipy()).sum(axis=1).max())
    g_ = 64
    h = 8.0 / (g_ + 1)
    xs = -4.0 + h * np.arange(1, g_ + 1)
    X, Y, Z = np.meshgrid(xs, xs, xs, indexing="ij")
    v = np.exp(-(X ** 2 + Y ** 2 + Z ** 2)).ravel()
    f = np.ones(a.n)
    ref_h = _fp64_judge(a, t, v)
    ref_s = _fp64_judge(a, t, v, f)
    dv = torch.from_numpy(v).cuda()
    dx = torch.zeros(a.n, dtype=torch.float64, device="cuda")
    sched = M.schedule_default(precision=M.FP32_KAHAN, num_levels=3, max_levels=10,
                               time_budget_s=args.step_budget)
    res = {}
    with M.Plan.from_csr(a, t, sched, rel_tol=args.tol, stream=stream.cuda_stream) as plan:
        for name, src, ref in (("homogeneous", None, ref_h), ("with_source", f, ref_s)):
            plan.set_source(src)
            _timed_solve(plan, dv, dx, 20)  # warm-up (loads this kernel variant)
            sec, est, conv, events = _timed_solve(plan, dv, dx, 21)
            x = dx.cpu().numpy()
            lv, _ = plan.stats()
            res[name] = {"seconds": sec, "est_rel_err": est, "converged": conv,
                         "walk_steps_per_s": events / sec, "levels": [l["level"] for l in lv],
                         "rel_err_vs_fp64": float(np.linalg.norm(x - ref) / np.linalg.norm(ref))}
            log(f"{name}: {sec:.3f} s, est {est:.3g}, err {res[name]['rel_err_vs_fp64']:.3g}")
        l0 = plan.info()["l0"]
    out = {"metric": "inhomogeneous solve (Algorithm 3 source term): time to tolerance",
           "n_gpus": 1, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "convection-diffusion 64^3, v = Gaussian bump, F = 1, t||A||=8",
                      "n": a.n, "nnz": a.nnz, "t": t, "tol": args.tol, "l0": l0},
           **res, "value": res["with_source"]["seconds"], "unit": "s", "higher_is_better": False}
    print(json.dumps(out), flush=True)


def run_forward_workload(args):
    """Forward mode (Eq. 5: walks on A^T from starts drawn ~ |v|) against
    backward mode (walks from every row) for the full vector x = exp(tA)v on
    the convection-diffusion workload (nonsymmetric; v the Gaussian bump,
    concentrated near the centre), FP32 walks, tolerance --tol, both against
    the FP64 Taylor judge."""
    import torch
    import mlmc_inputs as I
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    stream = torch.cuda.current_stream()
    w = I.workload_c4()
    ref = _fp64_judge(w.a, w.t, w.v)
    nref = np.linalg.norm(ref)
    dv = torch.from_numpy(w.v).cuda()
    dx = torch.zeros(w.a.n, dtype=torch.float64, device="cuda")
    res = {}
    for name, mode in (("backward", M.BACKWARD), ("forward", M.FORWARD)):
        sched = M.schedule_default(precision=M.FP32_KAHAN, num_levels=4, max_levels=10, mode=mode,
                                   time_budget_s=args.step_budget)
        with M.Plan.from_csr(w.a, w.t, sched, rel_tol=args.tol, stream=stream.cuda_stream) as plan:
            _timed_solve(plan, dv, dx, 40)  # warm-up
            sec, est, conv, _ = _timed_solve(plan, dv, dx, 41)
            lv, _ = plan.stats()
            walks = sum(l["walks_per_row"] for l in lv) * (1 if mode == M.FORWARD else w.a.n)
            events = walks + sum(l["jumps"] for l in lv)
        x = dx.cpu().numpy()
        res[name] = {"seconds": sec, "est_rel_err": est, "converged": conv, "walks": walks,
                     "walk_steps_per_s": events / sec,
                     "rel_err_vs_fp64_taylor": float(np.linalg.norm(x - ref) / nref)}
        log(f"{name}: {sec:.3f} s, {walks:.3g} walks, est {est:.3g}, "
            f"err {res[name]['rel_err_vs_fp64_taylor']:.3g}")
    out = {"metric": "full vector exp(tA)v: forward vs backward mode, time to tolerance",
           "n_gpus": 1, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "n": w.a.n, "nnz": w.a.nnz, "t": w.t, "tol": args.tol},
           **res, "value": res["backward"]["seconds"] / res["forward"]["seconds"],
           "unit": "x (backward time / forward time)", "higher_is_better": True}
    print(json.dumps(out), flush=True)


def run_c1_workload(args):
    """The FP64 walk on the small 2D Laplacian (32 x 32 grid scaled by 1/h^2,
    t ||A||_inf = 4, v uniform, 3 levels, tolerance 1e-2): time to the
    tolerance per solve, walk-steps/s and the error against dense FP64
    scaling-and-squaring (scipy.linalg.expm), over --steps solves with new
    seeds after --warmup untimed ones."""
    import scipy.linalg
    import torch
    import mlmc_inputs as I
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc as M
    stream = torch.cuda.current_stream()
    w = I.workload_c1()
    ref = scipy.linalg.expm(w.t * w.a.scipy().toarray()) @ w.v
    nref = np.linalg.norm(ref)
    dv = torch.from_numpy(w.v).cuda()
    dx = torch.zeros(w.a.n, dtype=torch.float64, device="cuda")
    sched = M.schedule_default(precision=M.FP64, num_levels=w.num_levels, max_levels=10,
                               time_budget_s=args.step_budget)
    runs = []
    with M.Plan.from_csr(w.a, w.t, sched, rel_tol=w.tol, stream=stream.cuda_stream) as plan:
        for k in range(args.warmup):
            _timed_solve(plan, dv, dx, 100 + k)
        for k in range(args.steps):
            sec, est, conv, events = _timed_solve(plan, dv, dx, 1000 + k)
            x = dx.cpu().numpy()
            levels, _ = plan.stats()
            runs.append({"seconds": sec, "est_rel_err": est, "converged": conv,
                         "rel_err_vs_fp64_expm": float(np.linalg.norm(x - ref) / nref),
                         "walk_steps_per_s": events / sec, "levels": len(levels),
                         "walks_per_row": [lv["walks_per_row"] for lv in levels]})
            log(f"c1 solve {k}: {sec * 1e3:.2f} ms, est {est:.3g}, "
                f"err {runs[-1]['rel_err_vs_fp64_expm']:.3g}")
        l0 = plan.info()["l0"]
    errs = [r["rel_err_vs_fp64_expm"] for r in runs]
    out = {"metric": "time to rel. RMS tolerance 1e-2, FP64 walk",
           "value": statistics.median(r["seconds"] for r in runs), "unit": "s",
           "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "n": w.a.n, "nnz": w.a.nnz, "t": w.t, "tol": w.tol,
                      "l0": l0, "levels": w.num_levels},
           "walk_steps_per_s": statistics.median(r["walk_steps_per_s"] for r in runs),
           "all_converged": all(r["converged"] for r in runs),
           "rel_err_vs_fp64_expm": {"median": statistics.median(errs), "max": max(errs)},
           "runs": runs}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--dist-backend", choices=["nccl", "gloo"], default="nccl",
                    help="N > 1: the process group's backend (gloo: a host-side check of the "
                         "sharded path; ranks may share a GPU)")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--step-budget", type=float, default=60.0,
                    help="controller wall-clock budget of one solve (s); the plain solve of the "
                         "default workload runs to it")
    ap.add_argument("--plain-budget", type=float, default=8.0,
                    help="budget of the plain (untilted) comparison solve of the default workload")
    ap.add_argument("--mlp-steps", type=int, default=150,
                    help="Adam steps per round of the learned proposal's training")
    ap.add_argument("--mlp-batch", type=int, default=16384,
                    help="rows per training step (128 per CTA of the fused training kernel)")
    ap.add_argument("--rounds", type=int, default=2,
                    help="pilot-train-install rounds of the learned proposal (mlmc_learn_tilt)")
    ap.add_argument("--time-pieces", type=int, default=1, choices=[0, 1],
                    help="1: laws that change with time (4 and 8 pieces of the scaled time) are "
                         "candidates of the learned proposal too")
    ap.add_argument("--pilot", type=int, default=64,
                    help="first-round pilot walks per row of the learned proposal")
    ap.add_argument("--workload", choices=["tc", "batch", "learned", "precision", "kernel",
                                           "levels", "complexity", "source", "forward", "c1"],
                    default="tc",
                    help="tc: the metric's workload (default); batch: batched vs plain; "
                         "learned: learned proposal vs plain; precision: FP32 vs FP64 walk; "
                         "kernel: the walk kernel alone; levels: m_l and V_l vs level; "
                         "complexity: MLMC vs single-level MC and the l0 sweep; "
                         "source: the inhomogeneous problem (Algorithm 3); "
                         "forward: forward vs backward mode; c1: the FP64 walk on the small 2D "
                         "Laplacian")
    ap.add_argument("--max-level", type=int, default=10, help="--workload levels: finest level")
    ap.add_argument("--kernel-reps", type=int, default=4096,
                    help="walks per row of one launch in --workload kernel")
    ap.add_argument("--kernel-matrix", choices=["ba", "lap3d", "c4", "c5"], default="ba",
                    help="--workload kernel: ba = the metric's graph (short walks), "
                         "lap3d = 64^3 Laplacian at t = 1 (long walks), c4 = convection-diffusion "
                         "128^3, c5 = BA n = 1e6 m = 8 (tables larger than L2)")
    ap.add_argument("--kernel-tilt", action="store_true",
                    help="--workload kernel: time the walk with the learned tilted proposal "
                         "(the default workload's solve)")
    ap.add_argument("--kernel-precision", choices=["fp32", "fp64"], default="fp32",
                    help="--workload kernel: walk precision (fp64: the all-FP64 walk)")
    ap.add_argument("--l2-persist", type=int, default=1, choices=[0, 1],
                    help="--workload kernel: L2 access-policy window over the tables")
    ap.add_argument("--walks-per-lane", type=int, default=0,
                    help="--workload kernel: walks per lane of one work item (0 = library default)")
    ap.add_argument("--block", type=int, default=0,
                    help="--workload kernel: threads per block (0 = library default)")
    ap.add_argument("--tol", type=float, default=1e-2, help="tolerance of --workload batch")
    ap.add_argument("--batch-nmax", type=float, default=1e6,
                    help="--workload batch: largest instance size (1e6: the batching workload; "
                         "smaller: many small problems)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.workload == "batch":
        run_batch_workload(args)
    elif args.workload == "learned":
        run_learned_workload(args)
    elif args.workload == "precision":
        run_precision_workload(args)
    elif args.workload == "kernel":
        run_kernel_workload(args)
    elif args.workload == "levels":
        run_levels_workload(args)
    elif args.workload == "complexity":
        run_complexity_workload(args)
    elif args.workload == "source":
        run_source_workload(args)
    elif args.workload == "forward":
        run_forward_workload(args)
    elif args.workload == "c1":
        run_c1_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
