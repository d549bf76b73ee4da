"""The N>1 form of bench.py, on CPU: one gloo process per rank (world size 2).

The path does not exchange data between GPUs (each rank quantizes its own
images: replicas only), so what N>1 adds is host logic: disjoint per-rank
workloads, the max-over-ranks time and the summed units, and the reference
arm printing on rank 0 alone.  These run here without a GPU.
"""
import io
import os
import socket
import contextlib

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        total, e2e, units = bench.combine_ranks(10.0 + rank, 30.0 - 5 * rank, 1000 * (rank + 1),
                                                "cpu")
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            if rank != 0:
                bench.run_reference(type("A", (), dict(steps=1, warmup=3))())
        out[rank] = (total, e2e, units, bench.dist_env(), buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_summed_units():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        total, e2e, units, env, printed = res[rank]
        assert total == 11.0            # the slower rank's device time
        assert e2e == 30.0              # the slower rank's end-to-end time
        assert units == 3000.0          # both ranks' units
        assert env == (world, rank, rank)
        assert printed == ""            # the reference arm prints on rank 0 only


def test_single_process_combine_is_identity():
    assert bench.combine_ranks(2.5, 4.0, 7, "cpu") == (2.5, 4.0, 7.0)


def test_rank_workloads_are_disjoint():
    seeds = {r: [bench.image_seed(r, s) for s in range(8)] for r in range(4)}
    flat = [x for v in seeds.values() for x in v]
    assert len(set(flat)) == len(flat)
    a, b = bench.workload(0), bench.workload(1)
    assert len(a) == len(b) == 8
    assert all(x.shape == (bench.H, bench.W, 3) for x in a + b)
    assert not any(np.array_equal(x, y) for x, y in zip(a, b))
