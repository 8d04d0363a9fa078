"""The N > 1 host logic of bench.py on CPU: two gloo ranks run the timing
aggregation (max over ranks of the timed region, whole-job rate) and the
q-sharded split (bench.shard_plan lists of inversion classes {q, -q},
bench.gather_q_sharded all-gather) the way the GPU ranks do under NCCL, with
the oracle standing in for kald_linewidths_qlist on each rank's q-points.  No
GPU is involved."""

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
    total_ms, value = bench.job_throughput(local_ms, w, units_per_step=2 * 5.0e9, steps=3, device="cpu")
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
    import bench
    nq, nb = nu.shape
    plan = bench.shard_plan(w.mesh, 1, world, rank)
    assert plan["kind"] == "qlist"
    mine = plan["q"]
    g = an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz, w.n_sigma, q_list=mine)
    full = bench.gather_q_sharded(torch.from_numpy(np.ravel(g)), plan, nb, nq, world)
    full = full.numpy().reshape(nq, nb)
    if rank == 0:
        ref = an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz, w.n_sigma)
        q.put(float(np.max(np.abs(full - ref))))
    dist.barrier()
    dist.destroy_process_group()


def test_q_sharded_linewidths_gather_to_the_single_rank_result():
    """The multi-GPU split of the hot path (independent q items, runs of
    inversion classes {q, -q} per rank from bench.shard_plan, one all-gather of
    gamma by bench.gather_q_sharded), emulated by two gloo ranks that each run
    the oracle on their q-points: the gathered gamma equals the single-rank
    result exactly."""
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


def test_shard_plan_covers_every_unit_once():
    """Every q-point is in exactly one rank's list, each list is closed under
    q -> -q, and the ranks' inversion classes differ in number by at most one
    (ceil split)."""
    import bench
    for mesh in ((1, 1, 1), (2, 1, 1), (7, 1, 1), (3, 3, 3), (4, 4, 4), (8, 8, 8), (3, 4, 5)):
        nq = mesh[0] * mesh[1] * mesh[2]
        cls = bench.inversion_classes(mesh)
        assert sorted(q for c in cls for q in c) == list(range(nq))
        for world in (1, 2, 3, 4, 8):
            plans = [bench.shard_plan(mesh, 1, world, r) for r in range(world)]
            if world == 1:
                assert plans[0]["kind"] == "whole"
                continue
            if nq == 1:
                assert all(p["kind"] == "replica" for p in plans)
                continue
            qs = sorted(q for p in plans for q in p["q"])
            assert qs == list(range(nq))
            for p in plans:
                mine = set(p["q"])
                for c in cls:
                    assert mine.issuperset(c) or not mine.intersection(c)
    # the inverse of a mesh point, by its coordinates
    assert bench.inversion_classes((4, 1, 1)) == [[0], [1, 3], [2]]
    plans = [bench.shard_plan((1, 1, 1), 24, 8, r) for r in range(8)]
    assert sorted(x for p in plans for x in p["idx"]) == list(range(24))
