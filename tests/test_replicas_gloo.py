"""The host side of the benchmark.  The multi-rank path (replicas only: one independent run per
rank, no data-path collective) on CPU with two gloo ranks: the whole-job time
is the slowest rank's, the particle-steps are summed over the ranks, every rank
draws its own seed, and only rank 0 prints the reference (oracle) arm's line,
which carries the keys the benchmark's contract asks for."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.aggregate(10.0 + 3.0 * rank, 1000 * (rank + 1), "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(7, rank))
        with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
            json.dump({"ms": ms, "units": units, "seeds": seeds}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms"] == 13.0                 # the slowest rank
        assert r["units"] == 3000.0            # all ranks' particle-steps
        assert len(set(r["seeds"])) == world   # independent replicas


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(4.5, 123, "cpu") == (4.5, 123)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    bench.reference_arm(bench.args())
    assert capsys.readouterr().out == ""


def test_reference_arm_line(tmp_path):
    # the oracle arm of the benchmark: one JSON line with the contract's keys
    import json as _json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600,
                       env={**os.environ, "RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = _json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "particle-steps/s"
    for k in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config"):
        assert k in d, k
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
