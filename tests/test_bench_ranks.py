"""The benchmark's multi-rank host logic, as world-size-2 `gloo` process
groups on the CPU.  The product is replicated per GPU (nothing is sharded);
what N > 1 adds is rank discovery from the torchrun environment, the
max-over-ranks step time every rank agrees on, the whole-job rate (units of
all ranks over the slowest rank's time), and the reference arm that runs on
rank 0 only.  The reference arm's JSON line is checked too: it runs the CPU
oracle and needs no GPU."""
import os
import socket
import sys

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, root, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, root)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, local = bench.dist_env()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, w)     # rank 1 is the slow one
        rate = bench.job_rate(1000, w, ms)
        dist.barrier()
        q.put((r, w, local, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, root, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got) and [g[2] for g in got] == [0, 1]
    for _, _, _, ms, rate in got:
        assert ms == 15.0                         # the slowest rank's time, seen by both
        assert rate == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_needs_no_process_group(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(900, 1, 300.0) == pytest.approx(3000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    # under torchrun every rank but 0 exits without work and prints nothing
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(workload="tiny", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line():
    # the reference arm (the CPU oracle, timed on the host) runs without a GPU
    # and prints one JSON line with the keys the benchmark contract names
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "jw_hh_n100_m2000",
                          "--steps", "1", "--warmup", "0"], cwd=root, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "products/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "jw_hh_n100_m2000"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
