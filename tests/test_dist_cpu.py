"""Multi-process host logic on the CPU (gloo ranks): the benchmark's
max-over-ranks timing and whole-job throughput (replicas, no data-path
collective), and the single-graph counting shard's reduction (each rank
counts the butterflies anchored in its own priority-rank range -- here with
the CPU oracle standing in for the GPU library -- and one all-reduce sums the
parts into the supports)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    dist.barrier()
    t = bench.max_over_ranks(local_ms, dist, device="cpu")
    out[rank] = (t, bench.job_throughput(world, 1000, 10, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0
    # 2 ranks x 1000 units x 10 steps in 0.15 s
    assert abs(out[0][1] - 2 * 1000 * 10 / 0.15) < 1e-6


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 2_000_000, 5, 1000.0) == 10_000_000.0


def _shard_rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import oracle
    from paper_2001_06111_gb300 import shard, synth
    g = synth.chunglu(300, 200, 3000, 2.1, 2.4, seed=77)
    n = g.nU + g.nL
    bounds = np.linspace(0, n, world + 1).astype(int)

    def count_part(p, P):
        return oracle.support_anchored(g.edges, g.nU, g.nL, int(bounds[p]), int(bounds[p + 1]))

    sup = shard.count_support_sharded(g.edges, g.nU, g.nL, count_part=count_part)
    out[rank] = sup.tolist()
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_counting_shard_sums_to_supports():
    import numpy as np

    import oracle
    from paper_2001_06111_gb300 import synth
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_shard_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    g = synth.chunglu(300, 200, 3000, 2.1, 2.4, seed=77)
    want = oracle.support(g.edges, g.nU, g.nL).tolist()
    assert out[0] == want and out[1] == want
    assert int(np.asarray(want).sum()) > 0
