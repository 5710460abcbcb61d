"""The bench's multi-rank path on CPU (gloo, world size 2): replicas report the max step
time over ranks and the whole-job throughput; the reference arm does no work off rank 0."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms_local = [0.030, 0.045][rank]
    ms = bench.max_over_ranks(torch, ms_local, w, "cpu")
    out[rank] = (r, w, local, ms, bench.whole_job_value(w, 36864, 3, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_and_sum_replicas():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][:3] == (0, 2, 0) and out[1][:3] == (1, 2, 1)
    for r in (0, 1):
        assert out[r][3] == pytest.approx(0.045)
        assert out[r][4] == pytest.approx(2 * 36864 * 3 / 0.045e-3)


def test_reference_arm_idle_off_rank_zero(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
