"""Benchmark: SSN solves to ||R(w)|| <= 1e-6 per second on GB300 (features + Algorithm 2 per step).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload NAME] [--precision fp64|mixed]

A step is one pass of the whole hot path on one synthetic problem: feature assembly (kernel
embeddings, Gram matrices, Cholesky) followed by Algorithm 2 until the natural residual is at
most 1e-6.  Under torchrun every rank solves its own independently seeded problem of the same
shape (weak scaling, no collective on the data path).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_14087_gb300 import workloads  # noqa: E402

METRIC = "SSN solves/s to ||R||<=1e-6 (time-to-residual = ms_per_step), FP64 vs mixed"
WORKLOADS = {
    # The timed shapes (d, n, l) in the Sec. 5 parameter regime (sigma^2 = 0.005, lambda1 = 1/l,
    # lambda2 = 1/sqrt(n), unit-cube filling points).  Step k of rank r solves the problem drawn
    # with seed 100 * (r + 1) + k: Algorithm 2's iteration count varies strongly with rounding
    # (the trajectories of two correct runs separate near the solution), so the metric is taken
    # over a set of problems of the same shape rather than one draw.
    "paper_d5_n1000_l300": dict(d=5, n=1000, l=300),
    "paper_d2_n100_l50": dict(d=2, n=100, l=50),
    "paper_d10_n2000_l1024": dict(d=10, n=2000, l=1024),
    "paper_d64_n4000_l2048": dict(d=64, n=4000, l=2048),
}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12     # SMs x FP64 FMA/clk x 2 flops x max clock
# kernel class whose launches are timed live inside the timed region for the roofline: the
# dominant O(l^3) product of each form (events around every other class's launches would only
# perturb the latency-bound step; the per-class breakdown comes from one extra untimed step)
ROOF_CLASS = {"mixed": "gemm_oz", "fp64": "gemm_f64"}
PROFILE_EVERY = 8   # events around one launch in 8 of that class (less perturbation of the step)
# DRAM bytes (read + write) of one k_oz_gemm launch of this workload's shape (300 x 300 x 300,
# six slices) from ncu captures of the current kernel; the algorithmic bytes of that launch (the
# sliced operands) are 2 x 300 x 6 x 320 x 2 = 2.30 MB.  Empty: the kernel gained its
# programmatic-launch wait/trigger after the last capture (2.34 MB,
# profiles/oz_gemm_emulated_fp64_l300_l1024_l2048.md), which is reported beside the null
# "traffic" as traffic_last_capture.
ROOF_TRAFFIC = {}
ROOF_TRAFFIC_LAST = {("gemm_oz", "paper_d5_n1000_l300"): {
    "bytes": 2340096.0,
    "note": "ncu dram__bytes_read+write of one 300x300x300 six-slice launch, taken before the "
            "kernel's griddepcontrol wait/trigger was added"}}


def seed_of(rank: int, step: int) -> int:
    """Seed of the problem solved in `step` by `rank` (step < 0: warm-up problems); every rank
    solves problems of its own (weak scaling: no problem is shared or split across ranks)."""
    return 100 * (rank + 1) + step if step >= 0 else 10_000 + 100 * rank - step


def make_problem(name: str, rank: int, step: int = 0):
    """Problem solved in `step` by `rank` (step < 0: warm-up problems)."""
    cfg = WORKLOADS[name]
    return workloads.paper_regime(seed=seed_of(rank, step), d=cfg["d"], n=cfg["n"], l=cfg["l"])


def job_totals(count_local: float, ms_local: float, world: int, device="cpu"):
    """Whole-job aggregate over the ranks of the default process group: (units summed over ranks,
    time = max over ranks in ms, rate = units / max time in s).  This reduction and the barriers
    around the timed region are the only cross-rank traffic."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    c = torch.tensor([float(count_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c)
    ms, units = float(t.item()), float(c.item())
    return units, ms, units / (ms / 1e3) if ms > 0 else 0.0


def config_of(name: str) -> dict:
    return dict(WORKLOADS[name])


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_solve(p):
    from oracle import kot_oracle as ko
    t = time.perf_counter()
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    r = ko.ssn_solve(F, p.tol)
    return time.perf_counter() - t, r


def run_reference(args, rank, world):
    """The oracle (plain FP64 NumPy/LAPACK) timed on the host cores: rank 0 only."""
    if rank != 0:
        return
    oracle_solve(make_problem(args.workload, 0, -1))
    times, iters, conv = [], [], 0
    for k in range(args.steps):
        t, r = oracle_solve(make_problem(args.workload, 0, k))
        times.append(t)
        iters.append(r.iters)
        conv += int(r.converged)
    total = sum(times)
    cores = len(os.sched_getaffinity(0))
    val = conv / total
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, **config_of(args.workload), "tol": 1e-6,
                   "oracle_iters": iters, "converged": conv},
        "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full solves (features + Algorithm 2 to 1e-6, one "
                                   f"problem per step) of {args.workload}, NumPy/LAPACK with "
                                   "default BLAS threads"},
        "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper_d5_n1000_l300", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-other", action="store_true", help="do not time the other precision")
    ap.add_argument("--skip-e2e", action="store_true", help="do not time the host-buffer path")
    ap.add_argument("--profile", default="roofline", choices=["roofline", "all", "none"],
                    help="kernel classes timed with CUDA events inside the timed region")
    ap.add_argument("--method", default="ssn", choices=["ssn", "eg", "batch"],
                    help="ssn: Algorithm 2 (the headline); eg: the pure extragradient method of "
                         "App. F, a fixed number of steps per problem; batch: kot_batch_solve "
                         "over an uneven batch (d 2..20, n 200..2000, l 32..512)")
    ap.add_argument("--batch", type=int, default=32, help="problems per batch (--method batch)")
    ap.add_argument("--autotune", action="store_true",
                    help="run kot_autotune for l first (untimed); off by default: its standalone "
                         "choices measured no better than the occupancy rule inside the solve")
    ap.add_argument("--max-iter", type=int, default=200,
                    help="outer-iteration cap of Algorithm 2 (lower it to time iterations at large l)")
    ap.add_argument("--workers", type=int, default=8, help="concurrent solves (--method batch)")
    ap.add_argument("--eg-steps", type=int, default=200, help="EG steps per problem (--method eg)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2310_14087_gb300 import kot

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(dev))
    if args.method == "eg":
        return eg_bench(args, world, rank, local_rank, dev)
    if args.method == "batch":
        return batch_bench(args, world, rank, local_rank, dev)
    p = make_problem(args.workload, rank, 0)
    tuned = None
    if args.autotune:
        # untimed: pick the emulated product's split counts and the Jacobi CTA count for this l
        tuned = dict(zip(("splits_3_slices", "splits_6_slices", "jacobi_ctas", "tile_n_3_slices",
                          "tile_n_6_slices"),
                         kot.Context(device=local_rank).autotune(p.l)))
    probs = [make_problem(args.workload, rank, k) for k in range(args.steps)]
    dprobs = [kot.DeviceProblem.from_problem(q, dev) for q in probs]
    warm = [kot.DeviceProblem.from_problem(make_problem(args.workload, rank, -1 - k), dev)
            for k in range(args.warmup)]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2
    peaks = load_peaks()

    def timed(prec):
        """W warm-up steps, then K timed steps (CUDA events on the library's stream, L2 flushed
        before each step outside the events); returns ms, per-class stats, launches, iters."""
        ctx = kot.Context(device=local_rank, stream=stream.cuda_stream, precision=prec,
                          max_iter=args.max_iter)
        g = torch.zeros(p.l, dtype=torch.float64, device=dev)

        def step(dp):
            ctx.build_features(dp.X, dp.Y, dp.Xf, dp.Yf, dp.sigma, dp.lambda1, dp.lambda2)
            return ctx.ssn_solve(dp.tol, g, allow_no_convergence=True)

        for dp in warm:
            step(dp)
        pname = "mixed" if prec == kot.MIXED else "fp64"
        all_mask = (1 << len(kot.KERNEL_CLASSES)) - 1
        mask = {"roofline": 1 << kot.KERNEL_CLASSES.index(ROOF_CLASS[pname]), "all": all_mask,
                "none": 0}[args.profile]
        ctx.profile_every(PROFILE_EVERY if args.profile == "roofline" else 1)
        ctx.profile(mask)
        launches0 = kot.launch_count()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        iters, conv = [], []
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                ev[k][0].record(stream)
            res = step(dprobs[k])
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
            iters.append(res.iters)
            conv.append(res.status == kot.OK)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        launches = kot.launch_count() - launches0
        ms = sum(a.elapsed_time(b) for a, b in ev)
        stats = {name: ctx.profile_read(i) for i, name in enumerate(kot.KERNEL_CLASSES)}
        # per-class breakdown: one more step (untimed) with every class under events
        ctx.profile_every(1)
        ctx.profile(all_mask)
        step(dprobs[0])
        torch.cuda.synchronize()
        breakdown = {name: ctx.profile_read(i) for i, name in enumerate(kot.KERNEL_CLASSES)}
        ctx.profile(0)
        return ms, (stats, breakdown), launches, iters, conv

    main_prec = kot.MIXED if args.precision == "mixed" else kot.FP64
    other_prec = kot.FP64 if main_prec == kot.MIXED else kot.MIXED
    with ClockSampler(local_rank) as clocks:
        ms_local, stats, launches, iters, conv = timed(main_prec)
    conv_all, ms_max, _ = job_totals(sum(conv), ms_local, world, dev)
    if not args.skip_other:
        o_ms_local, _, _, o_iters, o_conv = timed(other_prec)
        _, o_ms_max, o_value = job_totals(sum(o_conv), o_ms_local, world, dev)

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.skip_e2e:
        e2e = end_to_end(args, p, main_prec, world, dev, local_rank)
    if rank == 0:
        report(args, probs, world, ms_max, ms_local, stats, launches, iters, conv, clocks, peaks,
               None if args.skip_other else (other_prec, o_value, o_ms_max, o_iters, o_conv), e2e,
               conv_all, tuned)
    if world > 1:
        dist.destroy_process_group()


def eg_bench(args, world, rank, local_rank, dev):
    """Pure extragradient (App. F, Fig. 6): --eg-steps steps per problem after the features;
    reports EG steps per second and the residual reached, beside the SSN time to 1e-6."""
    import torch
    import torch.distributed as dist
    from paper_2310_14087_gb300 import kot
    prec = kot.MIXED if args.precision == "mixed" else kot.FP64
    stream = torch.cuda.Stream(device=dev)
    ctx = kot.Context(device=local_rank, stream=stream.cuda_stream, precision=prec,
                      max_iter=args.eg_steps)
    probs = [kot.DeviceProblem.from_problem(make_problem(args.workload, rank, k), dev)
             for k in range(args.steps)]
    warm = [kot.DeviceProblem.from_problem(make_problem(args.workload, rank, -1 - k), dev)
            for k in range(args.warmup)]
    l = WORKLOADS[args.workload]["l"]
    g = torch.zeros(l, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(dp):
        ctx.build_features(dp.X, dp.Y, dp.Xf, dp.Yf, dp.sigma, dp.lambda1, dp.lambda2)
        return ctx.eg_solve(1e-30, g, allow_no_convergence=True)

    for dp in warm:
        step(dp)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms, resid = 0.0, []
    for dp in probs:
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        r = step(dp)
        with torch.cuda.stream(stream):
            b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
        resid.append(r.residual)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        total = args.steps * args.eg_steps * world
        print(json.dumps({
            "metric": "pure extragradient steps/s (App. F), features included", "method": "eg",
            "value": total / (float(t.item()) / 1e3), "unit": "EG steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(t.item()) / args.steps,
            "higher_is_better": True, "scaling": "weak", "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, **config_of(args.workload), "precision": args.precision,
                       "eg_steps_per_problem": args.eg_steps, "eg_step_size": "1/L",
                       "residual_after_steps": resid}}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batch_bench(args, world, rank, local_rank, dev):
    """Uneven batch through kot_batch_solve (largest problems first, --workers concurrent
    solves with their own streams): each step solves one seeded batch to 1e-6.  Timed on the
    host between device synchronisations (the workers' streams belong to the library)."""
    import torch
    import torch.distributed as dist
    from paper_2310_14087_gb300 import kot
    prec = kot.MIXED if args.precision == "mixed" else kot.FP64
    ctx = kot.Context(device=local_rank, precision=prec, batch_workers=args.workers)

    def make(k):
        probs = workloads.paper_regime_batch(count=args.batch, base_seed=50_000 + 10_000 * rank + 1000 * k)
        return probs, [kot.DeviceProblem.from_problem(p, dev) for p in probs]

    warm = [make(-1 - k) for k in range(args.warmup)]
    steps = [make(k) for k in range(args.steps)]

    def solve(item):
        probs, dps = item
        gs = [torch.zeros(p.l, dtype=torch.float64, device=dev) for p in probs]
        return ctx.batch_solve(dps, gs)

    for w in warm:
        solve(w)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    results = [solve(st) for st in steps]
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    conv = sum(int(r.status == kot.OK) for res in results for r in res)
    iters = [r.iters for res in results for r in res]
    t = torch.tensor([secs], dtype=torch.float64, device=dev)
    c = torch.tensor([float(conv)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c)
    if rank == 0:
        print(json.dumps({
            "metric": "SSN solves/s to ||R||<=1e-6 over uneven batches (converged solves / wall s)",
            "method": "batch", "value": float(c.item()) / float(t.item()), "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(t.item()) / args.steps, "higher_is_better": True,
            "scaling": "weak", "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper_regime_batch", "batch": args.batch, "workers": args.workers,
                       "precision": args.precision, "d": "2..20", "n": "200..2000", "l": "32..512",
                       "converged": conv, "problems": args.batch * args.steps * world,
                       "mean_iters": float(np.mean(iters)), "timing": "host wall between device syncs"}}),
              flush=True)
    if world > 1:
        dist.destroy_process_group()


def end_to_end(args, p, main_prec, world, dev, local_rank):
    """The same problems through the C ABI with HOST buffers: the library copies each step's
    inputs in and gamma out inside the timed region."""
    import torch
    import torch.distributed as dist
    from paper_2310_14087_gb300 import kot
    rank = int(os.environ.get("RANK", "0"))
    hctx = kot.Context(device=local_rank, host_pointers=1, precision=main_prec)
    hp = [make_problem(args.workload, rank, k) for k in range(args.steps)]
    host = [tuple(np.ascontiguousarray(a, dtype=np.float64) for a in (q.X, q.Y, q.Xf, q.Yf)) for q in hp]
    hg = np.zeros(p.l)
    w = make_problem(args.workload, rank, -1)
    hctx.build_features(*(np.ascontiguousarray(a, dtype=np.float64) for a in (w.X, w.Y, w.Xf, w.Yf)),
                        w.sigma, w.lambda1, w.lambda2)
    hctx.ssn_solve(w.tol, hg, allow_no_convergence=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv = 0
    for q, (hX, hY, hXf, hYf) in zip(hp, host):
        hctx.build_features(hX, hY, hXf, hYf, q.sigma, q.lambda1, q.lambda2)
        r = hctx.ssn_solve(q.tol, hg, allow_no_convergence=True)
        conv += int(r.status == kot.OK)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    c = torch.tensor([float(conv)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c)
    e2e_value = float(c.item()) / float(t.item())
    h2d = 8 * sum(a.size for a in host[0])
    d2h = 8 * p.l
    return {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def report(args, probs, world, ms_max, ms_local, stats, launches, iters, conv, clocks, peaks, other,
           e2e, conv_all, tuned=None):
    from paper_2310_14087_gb300 import kot
    value = conv_all / (ms_max / 1e3)          # converged solves per second, all ranks
    stats, breakdown = stats
    # the dominant O(l^3) product of the form, timed live with CUDA events in the timed region
    dom = ROOF_CLASS[args.precision]
    s = stats[dom]
    per_launch_ms = s.ms / max(1, s.launches)
    if s.launches == 0:
        dom = None                         # nothing was timed (--profile none)
    if dom == "gemm_oz":
        # executed BF16 tensor work (slice-pair products) against the sustained BF16 peak
        bound, unit = "tensor", "TFLOP/s"
        peak = peaks.get("bf16_tflops_sustained", 1713.0)
        peak_src = "bf16_tflops_sustained of MEASURED_PEAKS.json (kernel timed inside a long step)"
    elif dom is not None:
        bound, unit = "alu", "TFLOP/s"
        peak, peak_src = FP64_PEAK_TFLOPS, "FP64 FMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz"
    roofline = None
    if dom is not None:
        achieved = (s.flops / s.launches) / (per_launch_ms * 1e-3) / 1e12
        traffic = ROOF_TRAFFIC.get((dom, args.workload))
        roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak,
                    "unit": unit, "frac": achieved / peak, "traffic": traffic,
                    "traffic_note": None if traffic is None else
                    "ncu dram__bytes_read+write of one 300x300x300 six-slice launch (bytes)",
                    "traffic_last_capture": ROOF_TRAFFIC_LAST.get((dom, args.workload)),
                    "launches_timed": s.launches, "timed_one_in": PROFILE_EVERY if args.profile == "roofline" else 1,
                    "avg_launch_us": per_launch_ms * 1e3,
                    "share_of_step": s.ms * (PROFILE_EVERY if args.profile == "roofline" else 1) / ms_local,
                    "peak_source": peak_src}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, **config_of(args.workload), "tol": 1e-6,
                   "precision": args.precision, "iters_per_solve": iters,
                   "converged": sum(conv), "ms_per_iteration": ms_local / max(1, sum(iters)),
                   "problems": "one seeded problem per step (seed 100 (rank+1) + step)",
                   "autotuned": tuned,
                   "l2": "flushed before every step (256 MB write, untimed)"},
        "other_precision": None if other is None else {
            "precision": "fp64" if other[0] == kot.FP64 else "mixed", "value": other[1],
            "ms_per_step": other[2] / args.steps, "iters_per_solve": other[3],
            "converged": sum(other[4]), "ms_per_iteration": other[2] / max(1, sum(other[3]))},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "roofline": roofline,
        "kernels_one_untimed_step": {k: {"launches": v.launches, "ms": round(v.ms, 3)}
                                     for k, v in breakdown.items() if v.launches},
    }
    if not args.no_cpu_baseline and world == 1:
        tcpu, r = oracle_solve(probs[0])
        line["cpu_baseline"] = {
            "value": (1.0 if r.converged else 0.0) / tcpu, "unit": "solves/s",
            "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "ms_per_iteration": 1e3 * tcpu / max(1, r.iters),
            "sample": f"1 full solve of {args.workload} (the step-0 problem: features + "
                      f"Algorithm 2, {r.iters} iterations, converged={r.converged}), "
                      "NumPy/LAPACK FP64, default BLAS threads"}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
