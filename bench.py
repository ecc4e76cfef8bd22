"""Benchmark: SSN solves to ||R(w)|| <= 1e-6 per second on GB300 (features + Algorithm 2 per step).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload NAME] [--precision fp64|mixed] [--method ssn|eg|batch|product|features]

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
# DRAM bytes (read + write) per launch of the dominant kernel, from an ncu capture of the
# current kernel on a standalone product of the workload's size (bench.py --method product;
# profiles/ names the command).  The solve's launches of that kernel mix shapes (l x l x l
# products and the |alpha-bar|- or |alpha|-row products of CG), so the figure is that of the
# l x l x l six-slice launch; None until a capture of the current kernel exists.
# (gemm_oz, 300^3, six slices): 2344704 and 2340352 bytes read, 0 written, in the two captured
# launches (profiles/oz_gemm_emulated_fp64_l300_l1024_l2048.md); algorithmic 2.30 MB of slices.
# DRAM bytes per launch of the dominant kernel from an ncu capture (see profiles/), keyed by class,
# workload and slices; None where the kernel changed since the counters were taken
ROOF_TRAFFIC = {("gemm_oz", "paper_d5_n1000_l300", 6): 2341803.0}   # k_oz_gemm<128>


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


def oracle_solve(p, with_features=False):
    from oracle import kot_oracle as ko
    t = time.perf_counter()
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    r = ko.ssn_solve(F, p.tol)
    t = time.perf_counter() - t
    return (t, r, F) if with_features else (t, r)


ONE_CORE_ENV = {"OPENBLAS_NUM_THREADS": "1", "OMP_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                "GOTO_NUM_THREADS": "1"}


def oracle_one_core(workload: str, step: int = 0):
    """The oracle's solve of one problem timed in a child process whose BLAS uses one thread
    (the thread count is fixed when NumPy loads its BLAS, so it takes a fresh interpreter)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "t, r = bench.oracle_solve(bench.make_problem(%r, 0, %d)); "
            "print(json.dumps({'s': t, 'iters': r.iters, 'converged': bool(r.converged)}))"
            % (ROOT, workload, step))
    env = dict(os.environ, **ONE_CORE_ENV)
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=600)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:   # the baseline is reported, never required
        return {"error": str(e)[:200]}


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
                   "oracle_iters": iters, "converged": conv,
                   "one_core": one_core_line(args.workload)},
        "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full solves (features + Algorithm 2 to 1e-6, one "
                                   f"problem per step) of {args.workload}, NumPy/LAPACK with "
                                   "default BLAS threads"},
        "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def one_core_line(workload):
    r = oracle_one_core(workload)
    if "s" not in r:
        return r
    return {"value": (1.0 if r["converged"] else 0.0) / r["s"], "unit": "solves/s", "cores": 1,
            "iters": r["iters"], "sample": f"the step-0 problem of {workload}, BLAS on one thread"}


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
    ap.add_argument("--method", default="ssn", choices=["ssn", "eg", "batch", "product", "features", "eig",
                                                        "bootstrap"],
                    help="ssn: Algorithm 2 (the headline); eg: the pure extragradient method of "
                         "App. F, a fixed number of steps per problem; batch: kot_batch_solve "
                         "over an uneven batch (d 2..20, n 200..2000, l 32..512); product: one "
                         "FP64-accurate l x l x l product per step (kot_dense_product, the "
                         "solve's dominant kernel alone, for ncu); features: the feature "
                         "assembly alone (kot_build_features); eig: cold symmetric "
                         "eigendecompositions (kot_eig_sym) per size bucket, --sizes; bootstrap: "
                         "--batch resamples sharing the filling points (kot_bootstrap_solve) against "
                         "as many separate feature builds and solves")
    ap.add_argument("--batch", type=int, default=32, help="problems per batch (--method batch)")
    ap.add_argument("--autotune", action="store_true",
                    help="run kot_autotune for l first (untimed); off by default: its standalone "
                         "timings favour more splits than the default, which measured best inside "
                         "the solve (8 splits, 128-wide tiles at l = 300)")
    ap.add_argument("--max-iter", type=int, default=200,
                    help="outer-iteration cap of Algorithm 2 (lower it to time iterations at large l)")
    ap.add_argument("--workers", type=int, default=8, help="concurrent solves (--method batch)")
    ap.add_argument("--eg-steps", type=int, default=200, help="EG steps per problem (--method eg)")
    ap.add_argument("--slices", type=int, default=6, help="slices of the emulated product (--method product)")
    ap.add_argument("--sizes", default="64,160,300,512,1024,2048", help="sizes l (--method eig)")
    ap.add_argument("--gram-fp32", action="store_true", help="Gram matrices in FP32 (--method features)")
    ap.add_argument("--no-large-l", action="store_true",
                    help="skip the fixed-iteration lines at C3's and C5's shapes (--method ssn)")
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
    if args.method == "product":
        return product_bench(args, world, rank, local_rank, dev)
    if args.method == "features":
        return features_bench(args, world, rank, local_rank, dev)
    if args.method == "eig":
        return eig_bench(args, world, rank, local_rank, dev)
    if args.method == "bootstrap":
        return bootstrap_bench(args, world, rank, local_rank, dev)
    p = make_problem(args.workload, rank, 0)
    tuned = None
    if args.autotune:
        # untimed: pick the emulated product's split counts and the Jacobi CTA count for this l
        tuned = dict(zip(("splits_3_slices", "splits_6_slices", "jacobi_ctas", "tile_n_3_slices",
                          "tile_n_6_slices", "jacobi_threads"),
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

    # ---- untimed: the step-0 problem once more in each form, kept for the errors vs the oracle
    finals = {}
    for prec in ([main_prec] + ([] if args.skip_other else [other_prec])):
        c = kot.Context(device=local_rank, precision=prec, max_iter=args.max_iter)
        dp = dprobs[0]
        c.build_features(dp.X, dp.Y, dp.Xf, dp.Yf, dp.sigma, dp.lambda1, dp.lambda2)
        g0 = torch.zeros(p.l, dtype=torch.float64, device=dev)
        X0 = torch.zeros(p.l, p.l, dtype=torch.float64, device=dev)
        r0 = c.ssn_solve(dp.tol, g0, X0, allow_no_convergence=True)
        finals["mixed" if prec == kot.MIXED else "fp64"] = (g0.cpu().numpy(), X0.cpu().numpy(), r0)
        c.close()

    # ---- untimed by the step events: fixed-iteration solves at the large-l shapes
    large = None
    if not args.no_large_l and world == 1 and args.workload == "paper_d5_n1000_l300":
        large = large_l_lines(main_prec, dev, local_rank)

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.skip_e2e:
        e2e = end_to_end(args, p, main_prec, world, dev, local_rank)
    if rank == 0:
        report(args, probs, world, ms_max, ms_local, stats, launches, iters, conv, clocks, peaks,
               None if args.skip_other else (other_prec, o_value, o_ms_max, o_iters, o_conv), e2e,
               conv_all, tuned, finals, large)
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


def product_bench(args, world, rank, local_rank, dev):
    """One FP64-accurate l x l x l product per step through kot_dense_product (C = A B^T): the
    solve's dominant kernel class on its own, at the workload's l, with the L2 flushed between
    steps.  --precision mixed: emulated on the tensor cores with --slices slices; fp64: the FP64
    stream-K GEMM.  This is also the command the ncu captures of that kernel run."""
    import torch
    from paper_2310_14087_gb300 import kot
    l = WORKLOADS[args.workload]["l"]
    prec = kot.MIXED if args.precision == "mixed" else kot.FP64
    pieces = -args.slices if prec == kot.MIXED else 0
    stream = torch.cuda.Stream(device=dev)
    ctx = kot.Context(device=local_rank, stream=stream.cuda_stream, precision=prec)
    gen = torch.Generator(device=dev).manual_seed(1234 + rank)
    A = torch.randn(l, l, dtype=torch.float64, device=dev, generator=gen)
    B = torch.randn(l, l, dtype=torch.float64, device=dev, generator=gen)
    Cm = torch.zeros(l, l, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    cls = "gemm_oz" if prec == kot.MIXED else "gemm_f64"
    for _ in range(args.warmup):
        ctx.dense_product(l, l, l, 1.0, A, l, 0, B, l, 0, 0.0, Cm, l, pieces)
    ctx.profile_every(1)
    ctx.profile(1 << kot.KERNEL_CLASSES.index(cls) | 1 << kot.KERNEL_CLASSES.index("oz_aux"))
    torch.cuda.synchronize()
    ms = 0.0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        ctx.dense_product(l, l, l, 1.0, A, l, 0, B, l, 0, 0.0, Cm, l, pieces)
        with torch.cuda.stream(stream):
            b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    st = ctx.profile_read(kot.KERNEL_CLASSES.index(cls))
    aux = ctx.profile_read(kot.KERNEL_CLASSES.index("oz_aux"))
    ctx.profile(0)
    ref = A @ B.T
    err = float((Cm - ref).abs().max() / ref.abs().max())
    peaks = load_peaks()
    kms = st.ms / max(1, st.launches)
    if prec == kot.MIXED:
        peak, src = peaks.get("bf16_tflops", 1934.6), "bf16_tflops (burst) of MEASURED_PEAKS.json: kernel timed alone"
    else:
        peak, src = FP64_PEAK_TFLOPS, "FP64 FMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz"
    achieved = st.flops / max(1, st.launches) / (kms * 1e-3) / 1e12
    traffic = ROOF_TRAFFIC.get((cls, args.workload, args.slices if prec == kot.MIXED else 0))
    if rank == 0:
        print(json.dumps({
            "metric": "FP64-accurate l x l x l products/s (kot_dense_product)", "method": "product",
            "value": args.steps / (ms / 1e3), "unit": "products/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "l": l, "precision": args.precision,
                       "slices": args.slices if prec == kot.MIXED else None,
                       "rel_max_error_vs_torch_fp64": err, "l2": "flushed before every step"},
            "roofline": {"kernel": cls, "bound": "tensor" if prec == kot.MIXED else "alu",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "count": "method: 2 l^3 per FP64-accurate product",
                         "executed_tflops": st.exec_flops / max(1, st.launches) / (kms * 1e-3) / 1e12,
                         "traffic": traffic, "kernel_us": kms * 1e3,
                         "aux_us_per_product": aux.ms * 1e3 / max(1, args.steps), "peak_source": src}}),
              flush=True)


def features_bench(args, world, rank, local_rank, dev):
    """Feature assembly alone (kot_build_features: kernel embeddings, q2 pair sums, Gram matrices,
    Cholesky) per step on the workload's shape, each kernel class timed with CUDA events."""
    import torch
    from paper_2310_14087_gb300 import kot
    stream = torch.cuda.Stream(device=dev)
    ctx = kot.Context(device=local_rank, stream=stream.cuda_stream, gram_fp32=int(args.gram_fp32))
    probs = [kot.DeviceProblem.from_problem(make_problem(args.workload, rank, k), dev)
             for k in range(args.steps)]
    warm = kot.DeviceProblem.from_problem(make_problem(args.workload, rank, -1), dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    build = lambda dp: ctx.build_features(dp.X, dp.Y, dp.Xf, dp.Yf, dp.sigma, dp.lambda1, dp.lambda2)
    for _ in range(args.warmup):
        build(warm)
    names = ["embed", "pair_sums", "gram", "cholesky", "gemm_f64"]
    ctx.profile_every(1)
    ctx.profile(sum(1 << kot.KERNEL_CLASSES.index(n) for n in names))
    torch.cuda.synchronize()
    ms = 0.0
    for k, dp in enumerate(probs):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        build(dp)
        with torch.cuda.stream(stream):
            b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    stats = {n: ctx.profile_read(kot.KERNEL_CLASSES.index(n)) for n in names}
    ctx.profile(0)
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    per = {}
    for n, st in stats.items():
        if st.launches:
            per[n] = {"launches": st.launches, "ms": st.ms, "GB/s": st.bytes / (st.ms * 1e-3) / 1e9,
                      "frac_hbm": st.bytes / (st.ms * 1e-3) / 1e9 / hbm,
                      "fp64_tflops": st.flops / (st.ms * 1e-3) / 1e12,
                      "frac_fp64": st.flops / (st.ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
    if rank == 0:
        print(json.dumps({
            "metric": "feature assemblies/s (kot_build_features)", "method": "features",
            "value": args.steps / (ms / 1e3), "unit": "assemblies/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, **config_of(args.workload),
                       "gram": "fp32" if args.gram_fp32 else "fp64", "l2": "flushed before every step"},
            "classes": per, "hbm_peak_gbs": hbm, "fp64_peak_tflops": FP64_PEAK_TFLOPS}), flush=True)


def eig_bench(args, world, rank, local_rank, dev):
    """Cold symmetric eigendecompositions (no warm basis) per size l, of clustered spectra and of
    separated ones; the FP64-accurate decomposition behind Eq. (4.4)."""
    import torch
    from paper_2310_14087_gb300 import kot
    stream = torch.cuda.Stream(device=dev)
    prec = kot.MIXED if args.precision == "mixed" else kot.FP64
    ctx = kot.Context(device=local_rank, stream=stream.cuda_stream, precision=prec)
    out, out_sep = {}, {}
    for l, spectrum in [(int(x), s) for s in ("clustered", "separated") for x in args.sizes.split(",")]:
        if spectrum == "separated" and l > 512:
            continue
        gen = workloads.clustered_symmetric if spectrum == "clustered" else workloads.separated_symmetric
        Z = torch.as_tensor(gen(l, seed=l), device=dev)
        P = torch.zeros(l, l, dtype=torch.float64, device=dev)
        sig = torch.zeros(l, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            ctx.eig_sym(l, Z, None, P, sig)
        torch.cuda.synchronize()
        ms, sweeps = [], []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
            info = ctx.eig_sym(l, Z, None, P, sig)
            with torch.cuda.stream(stream):
                b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            sweeps.append(info)
        Zh = Z.cpu().numpy()
        Ph, sh = P.cpu().numpy(), sig.cpu().numpy()
        ref = np.linalg.eigvalsh(Zh)
        (out if spectrum == "clustered" else out_sep)[l] = {
            "ms_cold": statistics.median(ms), "sweeps": sweeps[0][0], "refine_steps": sweeps[0][1],
            "rel_err_eigenvalues": float(np.abs(sh - ref).max() / np.abs(ref).max()),
            "orthogonality": float(np.abs(Ph.T @ Ph - np.eye(l)).max())}
    if rank == 0:
        print(json.dumps({"metric": "cold symmetric eigendecomposition time per size (kot_eig_sym)",
                          "method": "eig", "unit": "ms", "higher_is_better": False, "n_gpus": 1,
                          "steps": args.steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
                          "config": {"spectrum": "clustered_symmetric (half in 6 clusters of width 1e-9)",
                                     "precision": args.precision},
                          "sizes": out,
                          "separated": {"spectrum": "separated_symmetric (gaps about 2/l)", "sizes": out_sep}}),
              flush=True)


def bootstrap_bench(args, world, rank, local_rank, dev):
    """--batch bootstrap resamples of one problem that share its filling points: one
    kot_build_features plus kot_bootstrap_solve (Q, K and R built once), against a feature build
    and solve per resample.  Both to ||R|| <= 1e-6 (or --max-iter iterations)."""
    import torch
    from paper_2310_14087_gb300 import kot
    prec = kot.MIXED if args.precision == "mixed" else kot.FP64
    stream = torch.cuda.Stream(device=dev)
    ctx = kot.Context(device=local_rank, stream=stream.cuda_stream, precision=prec, max_iter=args.max_iter)
    p = make_problem(args.workload, rank, 0)
    B = args.batch
    Xs, Ys = workloads.bootstrap_resamples(p, B, seed=7 + rank)
    dp = kot.DeviceProblem.from_problem(p, dev)
    tX, tY = (torch.as_tensor(a, device=dev) for a in (Xs, Ys))
    G = torch.zeros(B, p.l, dtype=torch.float64, device=dev)

    def shared():
        ctx.build_features(dp.X, dp.Y, dp.Xf, dp.Yf, dp.sigma, dp.lambda1, dp.lambda2)
        return ctx.bootstrap_solve(tX, tY, p.tol, G)

    def separate():
        res = []
        for b in range(B):
            ctx.build_features(tX[b], tY[b], dp.Xf, dp.Yf, dp.sigma, dp.lambda1, dp.lambda2)
            res.append(ctx.ssn_solve(p.tol, G[b], allow_no_convergence=True))
        return res

    def timed(f):
        f()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        res = f()
        with torch.cuda.stream(stream):
            b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), res

    ms_sh, res_sh = timed(shared)
    ms_sep, res_sep = timed(separate)
    its = [r.iters for r in res_sh]
    if rank == 0:
        print(json.dumps({
            "metric": "bootstrap solves/s with shared filling points (kot_bootstrap_solve)",
            "method": "bootstrap", "value": B / (ms_sh / 1e3), "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, **config_of(args.workload), "resamples": B,
                       "precision": args.precision, "max_iter": args.max_iter, "iters": its,
                       "converged": sum(int(r.status == kot.OK) for r in res_sh)},
            "ms_shared": ms_sh, "ms_separate": ms_sep, "separate_value": B / (ms_sep / 1e3),
            "same_iterations": its == [r.iters for r in res_sep]}), flush=True)


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


def errors_vs_oracle(F, ref, finals):
    """Distance of each form's result from the oracle's solve of the same problem to the same
    tolerance: relative error of f(gamma) and of gamma (max norm over max |gamma|), and ||R|| as
    the oracle evaluates it at the returned iterate."""
    from oracle import kot_oracle as ko
    out = {}
    for name, (g, X, r) in finals.items():
        out[name] = {"rel_err_objective": abs(r.objective - ref.objective) / abs(ref.objective),
                     "rel_err_gamma": float(np.abs(g - ref.gamma).max() / np.abs(ref.gamma).max()),
                     "residual_reported": r.residual, "residual_by_oracle": ko.residual(F, g, X).norm,
                     "iters": r.iters, "oracle_iters": ref.iters}
    return out


# Fixed-iteration lines (one warm-up solve first): the large-l shapes in the Sec. 5 regime, where
# Algorithm 2 does not reach 1e-6 within 200 iterations, and BASELINE's literal C2 inputs
# (Wishart Gaussians, sigma = the median distance, lambda2 = 1/n), where it stalls near 1e-2.
LARGE_L = [("paper_d10_n2000_l1024", 12, None), ("paper_d64_n4000_l2048", 5, None),
           ("literal_c2_wishart_d5_n1000_l300", 30, lambda: workloads.wishart_pair(seed=1))]


def large_l_lines(prec, dev, local_rank):
    """Per-iteration time of Algorithm 2 at C3's (l = 1024) and C5's (l = 2048) shapes over a fixed
    number of iterations, with the feature assembly timed separately (CUDA events)."""
    import torch
    from paper_2310_14087_gb300 import kot
    out = {}
    stream = torch.cuda.Stream(device=dev)
    for name, k, gen in LARGE_L:
        ctx = kot.Context(device=local_rank, stream=stream.cuda_stream, precision=prec, max_iter=k)
        p = gen() if gen else make_problem(name, 0, 0)
        dp = kot.DeviceProblem.from_problem(p, dev)
        g = torch.zeros(p.l, dtype=torch.float64, device=dev)
        build = lambda: ctx.build_features(dp.X, dp.Y, dp.Xf, dp.Yf, dp.sigma, dp.lambda1, dp.lambda2)
        build()
        ctx.ssn_solve(p.tol, g, allow_no_convergence=True)          # warm-up (allocations)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
        build()
        with torch.cuda.stream(stream):
            ev[1].record(stream)
        r = ctx.ssn_solve(p.tol, g, allow_no_convergence=True)
        with torch.cuda.stream(stream):
            ev[2].record(stream)
        ev[2].synchronize()
        solve_ms = ev[1].elapsed_time(ev[2])
        out[name] = {"d": p.d, "n": p.n, "l": p.l, "iterations": r.iters, "residual_after": r.residual,
                     "features_ms": ev[0].elapsed_time(ev[1]), "solve_ms": solve_ms,
                     "ms_per_iteration": solve_ms / max(1, r.iters), "eig_calls": r.eig_calls,
                     "jacobi_sweeps": r.eig_sweeps}
        ctx.close()
    return out


def report(args, probs, world, ms_max, ms_local, stats, launches, iters, conv, clocks, peaks, other,
           e2e, conv_all, tuned=None, finals=None, large=None):
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
        # the method's work (2MNK per FP64-accurate product) against the sustained BF16 peak;
        # the executed BF16 slice-pair work is reported beside it
        bound, unit = "tensor", "TFLOP/s"
        peak = peaks.get("bf16_tflops_sustained", 1713.0)
        peak_src = "bf16_tflops_sustained of MEASURED_PEAKS.json (kernel timed inside a long step)"
    elif dom is not None:
        bound, unit = "alu", "TFLOP/s"
        peak, peak_src = FP64_PEAK_TFLOPS, "FP64 FMA: 152 SMs x 2/clk x 2 flop x 2.07 GHz"
    roofline = None
    if dom is not None:
        achieved = (s.flops / s.launches) / (per_launch_ms * 1e-3) / 1e12
        executed = (s.exec_flops / s.launches) / (per_launch_ms * 1e-3) / 1e12
        traffic = ROOF_TRAFFIC.get((dom, args.workload, 6 if dom == "gemm_oz" else 0))
        roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak,
                    "unit": unit, "frac": achieved / peak, "traffic": traffic,
                    "count": "method: 2MNK flops per FP64-accurate product",
                    "executed_tflops": executed, "executed_frac": executed / peak,
                    "traffic_note": "ncu dram__bytes_read+write per launch of the standalone l x l x l "
                                    "six-slice product (bench.py --method product)" if traffic else
                                    "no capture of the current kernel: bench.py --method product under ncu",
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
    if large:
        line["large_l"] = {"what": "fixed-iteration solves, one problem each after one warm-up solve: "
                                   "C3's and C5's shapes in the Sec. 5 regime (1e-6 is not reached "
                                   "there in 200 iterations) and BASELINE's literal C2 inputs "
                                   "(Algorithm 2 stalls near 1e-2 there)", "precision": args.precision,
                           **large}
    mv = breakdown.get("schur_matvec")
    if mv is not None and mv.launches:
        mpk = peaks.get("bf16_tflops_sustained", 1713.0) if args.precision == "mixed" else FP64_PEAK_TFLOPS
        line["matvec"] = {
            "what": "one Schur-operator application of CG (Algorithm 1), one untimed step",
            "launches": mv.launches, "us_per_matvec": 1e3 * mv.ms / mv.launches,
            "fmv_tflops": mv.flops / (mv.ms * 1e-3) / 1e12,
            "exec_tflops": mv.exec_flops / (mv.ms * 1e-3) / 1e12,
            "frac_fmv": mv.flops / (mv.ms * 1e-3) / 1e12 / mpk, "peak": mpk,
            "count": "F_mv = (4/3) l^3 + 8 min(|alpha|,|alpha-bar|) l^2 + 2 l^2 (algorithmic); executed: "
                     "the eigenbasis form, 4 min(|alpha|,|alpha-bar|) l^2 + 2 l^2"}
    gr = breakdown.get("gram")
    if gr is not None and gr.launches:
        hbm = peaks.get("hbm_gbs", 6800.0)
        gbs = gr.bytes / (gr.ms * 1e-3) / 1e9
        line["gram"] = {"what": "Gram matrices Q and K (k_gram), one untimed step", "ms": gr.ms,
                        "GB/s": gbs, "frac_hbm": gbs / hbm, "hbm_peak": hbm,
                        "fp64_tflops": gr.flops / (gr.ms * 1e-3) / 1e12,
                        "frac_fp64": gr.flops / (gr.ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
    if not args.no_cpu_baseline and world == 1:
        tcpu, r, F = oracle_solve(probs[0], with_features=True)
        if finals:
            line["errors_vs_oracle"] = errors_vs_oracle(F, r, finals)
        line["cpu_baseline"] = {
            "value": (1.0 if r.converged else 0.0) / tcpu, "unit": "solves/s",
            "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "ms_per_iteration": 1e3 * tcpu / max(1, r.iters),
            "sample": f"1 full solve of {args.workload} (the step-0 problem: features + "
                      f"Algorithm 2, {r.iters} iterations, converged={r.converged}), "
                      "NumPy/LAPACK FP64, default BLAS threads"}
        line["cpu_baseline"]["one_core"] = one_core_line(args.workload)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
