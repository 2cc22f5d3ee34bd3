"""The multi-rank logic of bench.py on the CPU: world-size-2 gloo process groups stand in for the NCCL
ranks of a multi-GPU run (each rank advances its own replica; the job's time is the slowest rank's).

- max_over_ranks gives every rank the element-wise maximum of the ranks' timings.
- The whole-job value counts every rank's node updates over that time.
- Under torchrun, ranks other than 0 of the reference arm exit without work or output."""

import multiprocessing as mp
import socket

import pytest

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, timings, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        out.put((rank, bench.max_over_ranks(timings[rank], ws, "cpu")))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_time_reaches_every_rank():
    ws, port = 2, _free_port()
    timings = [[0.010, 2.5], [0.013, 2.1]]  # (device seconds, wall seconds) per rank
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, timings, out)) for r in range(ws)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == [0.013, 2.5]


def test_single_rank_keeps_its_own_times():
    assert bench.max_over_ranks([0.5, 1.5], 1, "cpu") == [0.5, 1.5]


def test_whole_job_value_counts_every_replica():
    # two ranks, 256^2 nodes each, 200 steps in 0.013 s (the slower rank)
    v = bench.aggregate_mlups(2, 65536, 200, 0.013)
    assert v == pytest.approx(2 * 65536 * 200 / 0.013 / 1e6)
    assert bench.aggregate_mlups(1, 65536, 200, 0.013) == pytest.approx(v / 2)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = bench.parse(["--impl", "reference", "--steps", "3", "--warmup", "3"])
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
