"""The multi-GPU path is replicas only (independent query batches, no
data-path collective): each rank evaluates its own seeded batch, the job's
step time is the slowest rank's, and the job's rate counts every rank's
queries.  Exercised here with two gloo ranks on the CPU, through the same
helpers bench.py uses; the oracle arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, local = bench._dist()
        step_ms = [3.0, 5.0][rank]                      # rank 1 is the slower replica
        ms = bench._max_over_ranks(step_ms)
        rate = bench._job_rate(1000, w, ms)
        seed = bench._rank_seed(1000, r)
        # the oracle arm: rank 0 alone does the work and prints
        import argparse
        args = argparse.Namespace(config="C0", steps=1, warmup=0, cpu_budget=0.1)
        import io
        import contextlib
        buf = io.StringIO()
        if r != 0:
            with contextlib.redirect_stdout(buf):
                bench.run_reference(args)
        q.put((r, w, local, ms, rate, seed, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get() for _ in range(2))
    (r0, w0, l0, ms0, rate0, seed0, out0), (r1, w1, l1, ms1, rate1, seed1, out1) = got
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert ms0 == ms1 == 5.0                      # max over ranks
    assert rate0 == rate1 == pytest.approx(2 * 1000 / 5e-3)
    assert seed0 != seed1                         # independent batches
    assert out1 == ""                             # non-zero ranks print nothing


def test_single_process_helpers():
    import bench
    assert bench._max_over_ranks(2.5) == 2.5
    assert bench._job_rate(65536, 1, 0.5) == pytest.approx(65536 / 5e-4)
    assert bench._rank_seed(1000, 0) == 1017 and bench._rank_seed(1000, 2) == 3017
