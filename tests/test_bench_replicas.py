"""The replica path of the benchmark on CPU: two gloo ranks on 127.0.0.1 (one process per
rank, as torchrun starts them).  Every GPU of a multi-GPU run solves its own problem (no
data-path collective), so the only cross-rank steps are the barrier and the maximum of the
per-step times that rank 0 reports."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, values, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        dist.barrier()
        out.put((rank, bench._max_over_ranks(values[rank], ws, "cpu")))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_step():
    ws, values = 2, [1.25, 3.5]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, values, out)) for r in range(ws)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 3.5, 1: 3.5}


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench._max_over_ranks(2.0, 1) == 2.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload, steps, warmup, cpu_budget = "sphere-ka4-ct-L4", 1, 0, 1.0

    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
