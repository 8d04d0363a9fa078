"""The N > 1 host logic of bench.py on CPU: two gloo ranks run the replica
aggregation (max over ranks of the timed region, whole-job rate) the way the
GPU ranks do under NCCL.  No GPU is involved."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    dist.barrier()
    local_ms = 1000.0 * (rank + 1)                # rank 1 is the slow one
    total_ms, value = bench.job_throughput(local_ms, w, units_per_step=5.0e9, steps=3, device="cpu")
    q.put((r, w, local, total_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [0, 1]
    for _, _, _, total_ms, value in out:
        assert total_ms == pytest.approx(2000.0)  # max over ranks
        assert value == pytest.approx(2 * 5.0e9 * 3 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    total_ms, value = bench.job_throughput(500.0, 1, units_per_step=1.0e9, steps=2)
    assert total_ms == 500.0 and value == pytest.approx(4.0e9)
