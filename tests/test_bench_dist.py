"""Host logic of bench.py's multi-GPU (replica) path, run as two gloo ranks on the CPU.

On a GPU machine the driver launches ``bench.py --gpus N`` under torchrun, one rank per GPU,
each rank working on its own slice: the timed region is the maximum over ranks and the
reported value counts the units of all ranks.  Here two CPU processes check that
reduction, the whole-job rate, and that the reference arm prints only on rank 0.
"""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    step_ms = 100.0 + 25.0 * rank  # rank 1 is the slow one
    m = bench.reduce_max(step_ms, "cpu")
    rate = bench.whole_job_rate(w, 50, m)
    out = io.StringIO()
    rc = 0
    if rank == 1:  # rank 0 would run the CPU oracle for real
        with contextlib.redirect_stdout(out):
            rc = bench.run_reference(types.SimpleNamespace(steps=1, warmup=0, gpus=world))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, r, w, local, m, rate, rc, out.getvalue()))


def test_replica_timing_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, local, m, rate, rc, printed in res:
        assert (r, w, local) == (rank, world, rank)
        assert m == pytest.approx(125.0)  # the max over ranks, seen by every rank
        assert rate == pytest.approx(world * 50 / 0.125)  # units of all ranks / slowest rank's time
    assert res[1][6] == 0 and res[1][7] == ""  # the reference arm: rank 1 exits 0 without output


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(3.5, "cpu") == 3.5
    assert bench.whole_job_rate(1, 10, 20.0) == pytest.approx(500.0)
