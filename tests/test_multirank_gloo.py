"""The bench's multi-rank path on the CPU: one replica per rank, a barrier, the
step time as the maximum over ranks and the landscape mean as the mean over
ranks (gloo, world size 2, rendezvous on 127.0.0.1)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        dist.barrier()
        step_ms = 100.0 + 50.0 * rank          # rank 1 is the slower replica
        mean_tflops = 600.0 + 10.0 * rank
        q.put((r, w, bench.max_over_ranks(step_ms, dist), bench.mean_over_ranks(mean_tflops, dist)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_step_time_and_mean():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 150.0 for o in out)            # max over ranks
    assert all(o[3] == 605.0 for o in out)            # mean over ranks


def test_single_process_helpers_are_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5 and bench.mean_over_ranks(2.0) == 2.0
