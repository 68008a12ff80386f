"""The multi-rank host logic of bench.py on two gloo ranks (CPU): each rank gets
its own disorder sample, the timing is the slowest rank's, and the value counts
every rank's spin updates."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    try:
        _run(rank, world, port, out)
    except BaseException as e:          # report instead of leaving the parent waiting
        out.put((rank, "error", repr(e), None))
        raise


def _run(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import bench
    from paper_1204_6192_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (world, rank, rank)
    wl = bench.shard_samples(inputs.workload("L8_plain"), rank)
    checksum = float(np.abs(wl.samples[0].J).sum())
    sums = [None] * world
    dist.all_gather_object(sums, checksum)
    ms = bench.max_over_ranks(10.0 + rank, torch, torch.device("cpu"))
    value = bench.whole_job_value(ms, updates_per_rank=1_000_000, world=world)
    out.put((rank, sums, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in procs), key=lambda r: r[0])
    assert all(r[1] != "error" for r in res), res
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, sums0, ms0, v0), (r1, sums1, ms1, v1) = res
    assert (r0, r1) == (0, 1)
    assert sums0 == sums1 and sums0[0] != sums0[1]       # distinct disorder per rank
    assert ms0 == ms1 == 11.0                             # the slower rank's time
    assert v0 == v1 == pytest.approx(11.0 * 1e6 / 2_000_000)
