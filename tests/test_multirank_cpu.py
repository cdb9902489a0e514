"""Multi-rank sharding on CPU (gloo, world size 2): independent jobs are split across ranks with
no collective on the data path; only the end-of-run statistics are gathered."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1410_2817_gb300 import inputs
from paper_1410_2817_gb300.serve import Scheduler, shard_jobs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jobs = inputs.serving_trace(njobs=80, seed=1, side2d=(16, 64), side3d=(8, 16), steps=(2, 6))
    mine = shard_jobs(jobs, rank, world)
    # each rank admits and retires its own jobs (host-side scheduler, nothing shared)
    sch = Scheduler(budget_bytes=1 << 40, bytes_of=lambda j: j.workload.nnodes * 16)
    for j in mine:
        sch.submit(j)
    sch.admit(0.0)
    for st in list(sch.active.values()):
        sch.finish(st, 1.0)
    local = {"rank": rank, "ids": sorted(j.job_id for j in mine),
             "node_steps": sum(j.workload.nnodes * j.workload.steps for j in mine), "done": len(sch.done)}
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    if rank == 0:
        q.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_shard_jobs_without_overlap():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=100)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids0, ids1 = set(gathered[0]["ids"]), set(gathered[1]["ids"])
    assert not (ids0 & ids1)
    assert sorted(ids0 | ids1) == list(range(80))
    assert gathered[0]["done"] == len(ids0) and gathered[1]["done"] == len(ids1)
    a, b = gathered[0]["node_steps"], gathered[1]["node_steps"]
    assert abs(a - b) <= 0.5 * max(a, b)
