"""The multi-rank path of bench.py on CPU (gloo, world size 2).

Under torchrun every rank solves problems of its own (disjoint seeds: weak scaling, nothing shared
or split across ranks), and the job's numbers are the units summed over ranks divided by the
slowest rank's time; the reduction in bench.job_totals is the only cross-rank traffic.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from oracle import kot_oracle as ko
        seeds = [bench.seed_of(rank, k) for k in range(4)] + [bench.seed_of(rank, -1 - k) for k in range(3)]
        all_seeds = [None] * world
        dist.all_gather_object(all_seeds, seeds)
        # each rank solves its own (tiny) problem; one converged unit per rank plus rank extra
        p = bench.workloads.paper_regime(seed=seeds[0], d=2, n=30, l=8)
        F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
        r = ko.ssn_solve(F, 1e-3, ko.Options(max_iter=50))
        units = (1.0 if r.iters >= 0 else 0.0) + rank
        totals = bench.job_totals(units, 10.0 * (rank + 1), world)
        if rank == 0:
            q.put((all_seeds, totals))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_problems_and_aggregate_the_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    try:
        all_seeds, (units, ms, rate) = q.get(timeout=300)
    finally:
        for pr in procs:
            pr.join(timeout=120)
    assert all(pr.exitcode == 0 for pr in procs)
    assert set(all_seeds[0]).isdisjoint(all_seeds[1])
    assert units == 3.0                       # 1 + (1 + 1): summed over the ranks
    assert ms == 20.0                         # the slowest rank's time
    assert rate == pytest.approx(3.0 / 0.020)


def test_single_rank_totals_are_local():
    import bench
    assert bench.job_totals(5, 250.0, 1) == (5.0, 250.0, 20.0)


def test_errors_vs_oracle_reports_distances():
    # the bench line's distances of each form's result from the oracle's solve of the same
    # problem: relative objective and gamma errors, and R(w) as the oracle evaluates it
    import types
    import bench
    from oracle import kot_oracle as ko
    from paper_2310_14087_gb300 import workloads as wl
    p = wl.paper_regime(seed=2, d=2, n=100, l=50)
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    ref = ko.ssn_solve(F, p.tol)
    g = ref.gamma * (1 + 1e-7)
    r = types.SimpleNamespace(objective=ko.objective(F, g), residual=ref.residual, iters=ref.iters)
    out = bench.errors_vs_oracle(F, ref, {"fp64": (g, ref.X, r)})["fp64"]
    assert out["rel_err_gamma"] == pytest.approx(1e-7, rel=1e-6)
    assert out["rel_err_objective"] == pytest.approx(abs(r.objective - ref.objective) / abs(ref.objective))
    assert out["residual_by_oracle"] == pytest.approx(ko.residual(F, g, ref.X).norm)
    assert out["iters"] == out["oracle_iters"] == ref.iters
