"""The N > 1 path of bench.py (replicas, no data-path collective) with two gloo ranks on
the CPU: the barrier, the max-over-ranks timing, the whole-job rate and the reference
arm running on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_init()
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    local_ms = 100.0 + 50.0 * rank  # the slower rank decides the timed region
    tmax = bench.allreduce_max(local_ms, w)
    rate = bench.whole_job_rate(16, 5, w, tmax)

    class Args:
        workload = "q1_poisson_64x64"
        steps = 1
        warmup = 0
    ref = bench.run_reference(Args, r, w) if r != 0 else None  # rank 0 alone runs the oracle
    out.put((rank, tmax, rate, ref))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_replica_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, rate, ref in res:
        assert tmax == 150.0                       # max over ranks
        assert rate == pytest.approx(16 * 5 * 2 / 0.150)
        assert ref is None                         # non-zero ranks exit without work
