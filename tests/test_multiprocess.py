"""The multi-rank path of the benchmark on CPU: two gloo ranks on 127.0.0.1.

The method's per-sensor work shares nothing between ranks (replicas, weak scaling), so
the only cross-rank steps are the barrier around the timed region, the maximum of the
ranks' step times, and rank 0 alone printing (and, for the oracle arm, doing) the work.
"""
import contextlib
import io
import os
import socket
import sys
import types

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(3.0 + 2.0 * rank, torch.device("cpu"))   # ranks: 3 ms and 5 ms
        value = bench.job_throughput(1000.0, world, ms * 1e-3)
        # the oracle arm: only rank 0 works and prints
        args = types.SimpleNamespace(impl="reference", gpus=world, steps=1, warmup=0, workload="driving")
        out = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(out):
                bench.run_reference(args)
        results[rank] = (ms, value, out.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_only_rank_zero_reports():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), results), nprocs=2, join=True, start_method="spawn")
        res = dict(results)
    assert set(res) == {0, 1}
    for rank in (0, 1):
        ms, value, printed = res[rank]
        assert ms == 5.0                        # both ranks see the slower rank's time
        assert value == pytest.approx(2 * 1000.0 / 5e-3)   # the job's rays over that time
    assert res[1][2] == ""                      # rank 1 of the oracle arm exits without work


def test_single_process_passes_values_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.5, torch.device("cpu")) == 4.5
    assert bench.job_throughput(12_476_160, 1, 7.3e-3) == pytest.approx(12_476_160 / 7.3e-3)
