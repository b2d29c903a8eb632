"""The multi-GPU path of bench.py exercised as two gloo ranks on the CPU:
every rank is a replica with its own seeded data, the slowest rank's time
is taken (max over ranks), and the whole-job throughput counts the bytes of
all ranks.  No data-path collective exists; only the timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import synth_signals as ss


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, l = bench.dist_env()
    # per-rank replica data and a per-rank "time"
    x = ss.uniform_complex(bench.rank_seed(r), 2, 16, np.float32)
    my_ms = 10.0 + 5.0 * r
    mx = bench.max_over_ranks(my_ms, w, "cpu")
    val = bench.aggregate_gbs(1e9, 3, mx, w)
    q.put((r, w, l, float(x[0, 0].real), mx, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, w0, l0, x0, m0, v0), (r1, w1, l1, x1, m1, v1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert x0 != x1                       # replicas see different seeded data
    assert m0 == m1 == 15.0               # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 1e9 * 3 / 0.015 / 1e9)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.aggregate_gbs(2e9, 2, 1000.0, 1) == pytest.approx(4.0)
