"""CPU checks of bench.py's multi-rank path: the job's time is the maximum
over the ranks of a process group (two gloo ranks on this host), and the
reference arm runs on rank 0 only."""
import contextlib
import io
import json
import os
import socket
import sys
import tempfile
import types


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out_dir):
    import torch.distributed as dist
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(values[rank], world)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"rank": rank, "max": got}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    values = [3.25, 7.5]
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), values, d), nprocs=2, join=True)
        got = [json.load(open(os.path.join(d, f"rank{r}.json")))["max"] for r in range(2)]
    assert got == [max(values)] * 2


def test_max_over_ranks_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5


def _reference_args(gpus):
    return types.SimpleNamespace(n=16, p=2, tol=1e-8, steps=1, warmup=0, gpus=gpus,
                                 ref_budget=60.0, workers=2)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(_reference_args(2))
    assert buf.getvalue() == ""          # the other ranks exit without work or output
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(_reference_args(2))
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert isinstance(line["cpu_baseline"]["cpu_model"], str) and line["cpu_baseline"]["cpu_model"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_arm_counts_only_the_solves_it_ran(monkeypatch):
    """A step of the reference arm is one full oracle solve; with a budget of
    zero seconds it stops after the first timed solve and says so."""
    import bench
    monkeypatch.setenv("RANK", "0")
    args = _reference_args(1)
    args.steps, args.ref_budget, args.workers = 5, 0.0, 1
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip())
    assert line["steps"] == 1 and line["steps_requested"] == 5
    assert line["iterations"] > 0 and line["ms_per_step"] == 1e3 * line["value"]


def test_oracle_leg_reports_solution_differences():
    """The oracle leg solves the workload itself: fed its own tol solution as
    the 'GPU' FP64 solution, the same-tolerance difference is exactly 0 and the
    difference from the converged (1e-13) solution is the algebraic error of
    a 1e-8 solve (small, but not 0)."""
    import numpy as np
    import bench
    o = bench.OracleRun(12, 2, workers=1)
    res, _, _ = o.solve(1e-8)
    cpu, vs = bench.oracle_baseline(12, 2, 1e-8, {"fp64": res.x, "tf32": res.x + 1e-9}, workers=1)
    assert cpu["kind"] == "oracle" and cpu["iterations"] == res.iters and cpu["value"] > 0
    assert vs["fp64"]["vs_oracle_same_tol"]["max_rel"] == 0.0
    assert 0.0 < vs["fp64"]["vs_converged"]["max_rel"] < 1e-6
    assert vs["tf32"]["vs_converged"]["max_rel"] > 0.0
    assert vs["oracle_iterations_at_tol"] == res.iters
    assert np.isfinite(vs["fp64"]["vs_converged"]["l2_rel"])


def test_batch_timeline_summary():
    """bench.batch_timeline: per group its members' iterations, passes, first
    start and last end; passes and their summed time by the unfinished
    members at each pass's start; groups listed latest end first."""
    import numpy as np
    import bench

    class FakeBatch:
        def groups(self):
            return 2, [0, 1, 0]

        def pass_log(self, g):
            if g == 0:
                return {"start_us": np.array([0.0, 100.0, 250.0]),
                        "dur_us": np.array([100.0, 150.0, 50.0]), "active": np.array([2, 2, 1])}
            return {"start_us": np.array([10.0]), "dur_us": np.array([500.0]),
                    "active": np.array([1])}

    infos = [types.SimpleNamespace(iterations=i) for i in (3, 1, 2)]
    t = bench.batch_timeline(FakeBatch(), infos)
    assert t["groups"] == 2
    first, second = t["latest_groups"]
    assert first["group"] == 1 and first["end_ms"] == 0.51 and first["iterations"] == [1]
    assert second["group"] == 0 and second["iterations"] == [3, 2] and second["passes"] == 3
    assert second["end_ms"] == 0.3 and second["start_ms"] == 0.0
    assert t["latest_start_ms"] == 0.01
    assert t["passes_by_unfinished_members"]["1"] == {"passes": 2, "ms": 0.55}
    assert t["passes_by_unfinished_members"]["2-4"] == {"passes": 2, "ms": 0.25}


def test_stencil_dram_summary_is_current():
    """The committed DRAM summary of the stencil kernel was taken on the
    current kernel sources, so the bench reports its traffic (1.072 x the
    compulsory bytes at n = 128, p = 3) instead of null."""
    import bench
    assert bench.stencil_traffic(3, 128) == 5.96e9
    assert bench.stencil_traffic(3, 96) is None        # no summary for that size
