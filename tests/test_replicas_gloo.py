"""Multi-GPU is replicas only (no data exchange in the path): the benchmark's
N > 1 logic is the replica seeds, the max over ranks of the timed region and
the whole-job rate.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank                       # rank 1 is the slower one
    got = bench.max_over_ranks(ms, dist, "cpu")
    out.put((rank, got, [bench.replica_seed(rank, k) for k in range(3)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_distinct_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    seeds = [set(r[2]) for r in res]
    assert not (seeds[0] & seeds[1])
    # whole-job rate: all replicas' solves over the slowest time
    assert bench.whole_job_rate(2, 3, 1, 150.0) == pytest.approx(2 * 3 / 0.150)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(12.5, None) == 12.5
