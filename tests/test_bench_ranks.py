"""The multi-rank logic of bench.py on CPU: two gloo ranks with different
local times agree on the max-over-ranks time and on the whole-job value
(the ranks split one batch, so the value is its updates over the max time)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [12.0, 15.5][rank]
        ms, value = bench.job_time_and_value(local_ms, 2e9, world, bench.torch_reduce_max("cpu"))
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_max_time_and_sum_the_work():
    port = _free_port()
    with tmp.Manager() as man:
        out = man.dict()
        tmp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 15.5
    assert value == pytest.approx(2 * 1e9 / 15.5e-3)


def test_single_rank_needs_no_collective():
    ms, value = bench.job_time_and_value(10.0, 5e8, 1)
    assert ms == 10.0 and value == pytest.approx(5e10)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), dict(steps=3, warmup=3, gpus=2))()
    bench.reference_arm(args, {"workload": "x"})
    assert capsys.readouterr().out == ""
