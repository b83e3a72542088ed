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


def _shard_worker(rank, world, port, q, bad_header):
    import numpy as np
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        U = 1 << 60
        rs = np.random.default_rng(0)                       # the same table and order on every rank
        full = rs.integers(1000, 10 ** 7, size=(5, 64)).astype(np.int64)
        full[1, ::7] = U                                    # pruned on every rank
        order = rs.permutation(full.size)
        order = order[full.ravel()[order] != U]             # the library shards the pruned order
        local = full.copy().ravel()
        for p, item in enumerate(order):
            if p % world != rank:
                local[item] = 0                             # another shard times it
        hdr = bench.device_header("NVIDIA GB300" if not (bad_header and rank == 1) else "other GPU", 152,
                                  (4, 4, 4), list(range(5)), "rg test")
        try:
            merged = bench.merge_t0_shards(local.reshape(full.shape), hdr, dist)
            q.put((rank, "ok", bool(np.array_equal(merged, full))))
        except RuntimeError as e:
            q.put((rank, "error", str(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("bad_header", [False, True])
def test_sharded_sweep_merge_over_two_gloo_ranks(bad_header):
    """The exchange step of the sharded autotune sweep on two CPU ranks: every entry comes back from the
    rank that timed it, pruned entries stay pruned, and ranks that report different devices are refused."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q, bad_header)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    if bad_header:
        assert all(o[1] == "error" and "headers differ" in o[2] for o in out)
    else:
        assert all(o[1] == "ok" and o[2] for o in out)
