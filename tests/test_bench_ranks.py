"""Host logic of bench.py with several ranks, on CPU (gloo, world size 2).

On a multi-GPU node every rank runs an independent replica of the workload
(the step has no exchange between replicas), so the only cross-rank logic is
the timing reduction (the slowest rank's time, received by every rank), the
whole-job throughput over all replicas, and rank 0 alone printing; the
reference arm runs on rank 0 only.
"""
import json
import os
import socket
import sys
import types

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, device="cpu")
        out_q.put((rank, ms, bench.job_mlups(1000, world, 10, ms)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world, times = 2, [3.0, 5.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, mlups in res:
        assert ms == 5.0  # every rank holds the slowest rank's time
        # 1000 nodes per replica x 2 replicas x 10 steps in 5 ms
        assert mlups == pytest.approx(1000 * 2 * 10 / 5e-3 / 1e6)


def test_single_process_timing_unchanged():
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.job_mlups(16777216, 1, 1000, 280.0) == pytest.approx(16777216 * 1000 / 0.28 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = types.SimpleNamespace(nx=8, ny=6, nz=4, steps=1, warmup=0)
    bench.run_reference(args)  # returns before touching the oracle
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    args = types.SimpleNamespace(nx=8, ny=6, nz=4, steps=2, warmup=1)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
