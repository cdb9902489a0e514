"""Host-side logic of the server: admission under a budget and a slot limit, FIFO order, release,
rejection of jobs larger than the budget, and sharding of jobs across ranks (no GPU)."""
import numpy as np

from paper_1410_2817_gb300 import inputs
from paper_1410_2817_gb300.serve import Scheduler, percentiles, shard_jobs


def _jobs(n=40, seed=7):
    return inputs.serving_trace(njobs=n, seed=seed, side2d=(16, 64), side3d=(8, 16), steps=(2, 5))


def test_admission_respects_budget_and_order():
    jobs = _jobs()
    size = {j.job_id: 1000 + 10 * j.job_id for j in jobs}
    sch = Scheduler(budget_bytes=5000, max_active=3, bytes_of=lambda j: size[j.job_id])
    for j in jobs:
        sch.submit(j)
    admitted = sch.admit(0.0)
    assert [s.job.job_id for s in admitted] == [0, 1, 2]  # slot limit 3, FIFO
    assert sch.used == sum(size[i] for i in (0, 1, 2)) <= 5000
    assert sch.admit(0.1) == []  # full
    sch.finish(sch.active[1], 0.2)
    nxt = sch.admit(0.2)
    assert [s.job.job_id for s in nxt] == [3]
    done = 0
    t = 0.3
    while not sch.idle():
        for st in list(sch.active.values()):
            sch.finish(st, t)
            done += 1
        sch.admit(t)
        t += 0.1
        assert sch.used <= 5000 and len(sch.active) <= 3
    assert len(sch.done) == len(jobs)
    assert sch.peak_active == 3


def test_oversized_job_is_rejected_not_blocking():
    jobs = _jobs(5)
    sch = Scheduler(budget_bytes=100, bytes_of=lambda j: 500 if j.job_id == 1 else 50)
    for j in jobs:
        sch.submit(j)
    assert sch.done[1].rejected
    got = [s.job.job_id for s in sch.admit(0.0)]
    assert got == [0, 2]  # budget 100 holds two 50-byte jobs; the oversized job left the queue


def test_percentiles():
    p = percentiles(list(range(1, 101)))
    assert abs(p["p50"] - 50.5) < 1e-9 and abs(p["p99"] - 99.01) < 1e-9


def test_shard_jobs_partition_and_balance():
    jobs = _jobs(60)
    parts = [shard_jobs(jobs, r, 3) for r in range(3)]
    ids = sorted(j.job_id for p in parts for j in p)
    assert ids == sorted(j.job_id for j in jobs)
    loads = [sum(j.workload.nnodes * j.workload.steps for j in p) for p in parts]
    assert max(loads) - min(loads) <= max(j.workload.nnodes * j.workload.steps for j in jobs)
    assert shard_jobs(jobs, 0, 1) == list(jobs)


def test_trace_statistics():
    jobs = inputs.serving_trace(njobs=2000, seed=1)
    arr = np.array([j.arrival_s for j in jobs])
    assert abs(len(jobs) / arr[-1] - 200.0) < 20.0  # Poisson stream, mean 200 jobs/s
    frac3d = np.mean([j.workload.dim == 3 for j in jobs])
    assert 0.25 < frac3d < 0.35
    assert all(1 <= j.workload.nfields <= 4 and 10 <= j.workload.steps <= 200 for j in jobs)
