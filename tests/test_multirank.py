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


def _shard_rank(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    import kald_inputs as ki
    from oracle import anharmonic as an
    from oracle import phonons as ph
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = ki.small_binary(mesh=(3, 3, 3), sigma=0.1)
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    nq = nu.shape[0]
    per = -(-nq // world)                          # contiguous q ranges
    mine = list(range(rank * per, min(nq, (rank + 1) * per)))
    g = an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz, w.n_sigma, q_list=mine)
    buf = torch.zeros(per, nu.shape[1], dtype=torch.float64)
    buf[:len(mine)] = torch.from_numpy(g)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    full = torch.cat(parts)[:nq].numpy()
    if rank == 0:
        ref = an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz, w.n_sigma)
        q.put(float(np.max(np.abs(full - ref))))
    dist.barrier()
    dist.destroy_process_group()


def test_q_sharded_linewidths_gather_to_the_single_rank_result():
    """The multi-GPU split of the hot path (independent q items, contiguous q
    ranges per rank, one all-gather of gamma), emulated by two gloo ranks that
    each run the oracle on their shard: the gathered gamma equals the
    single-rank result exactly."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    diff = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert diff == 0.0
