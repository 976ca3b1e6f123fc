"""The multi-GPU path is independent replicas (particles never interact across ranks): what bench.py
does across ranks is host logic, tested here with two gloo ranks on the CPU -- every rank's replica
uses its own Philox seeds and a disjoint id range, and the job's time is the slowest rank's while its
particle-steps are the sum over ranks."""
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


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2511_08929_gb300 import inputs as I
        import dataclasses
        wl = dataclasses.replace(I.BATCHED_96, n_min=50, n_max=400, n_inst=6)
        insts, seeds, off = bench.replica_plan(wl, rank)
        ids = np.concatenate([wl.beam(k, x)["id"] + off for k, x in enumerate(insts)])
        gathered_ids = [None] * world
        gathered_seeds = [None] * world
        dist.all_gather_object(gathered_ids, ids.tolist())
        dist.all_gather_object(gathered_seeds, seeds)
        ms = 10.0 + 5.0 * rank
        psteps = 1000.0 * (rank + 1)
        tmax, total = bench.reduce_over_ranks(ms, psteps, dist, "cpu")
        out.put((rank, tmax, total, gathered_ids, gathered_seeds))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_are_independent_and_timed_as_one_job():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, total, ids, seeds in res:
        assert tmax == 15.0 and total == 3000.0
        assert not set(ids[0]) & set(ids[1])  # disjoint particle ids
        assert not set(seeds[0]) & set(seeds[1])  # distinct Philox seeds per instance
        assert len(ids[0]) == len(ids[1]) > 0
