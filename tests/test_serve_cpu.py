"""Host-side logic of the server: admission under a budget and a slot limit, FIFO and
shortest-work-first order, release, rejection of jobs larger than the budget, sharding of jobs
across ranks, and which jobs share a batch lane (no GPU)."""
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


def test_sjf_admits_least_work_first_under_the_cap():
    jobs = _jobs(12)
    work = {j.job_id: float((7 * j.job_id) % 12) for j in jobs}  # a permutation of 0..11
    sch = Scheduler(budget_bytes=10 ** 9, max_active=4, bytes_of=lambda j: 100, policy="sjf",
                    work_of=lambda j: work[j.job_id])
    for j in jobs:
        sch.submit(j)
    first = [s.job.job_id for s in sch.admit(0.0)]
    assert sorted(work[i] for i in first) == [0.0, 1.0, 2.0, 3.0] and len(sch.active) == 4
    order = list(first)
    t = 0.1
    while not sch.idle():
        st = min(sch.active.values(), key=lambda s: s.job.job_id)
        sch.finish(st, t)
        order += [s.job.job_id for s in sch.admit(t)]
        assert len(sch.active) <= 4
        t += 0.1
    assert [work[i] for i in order] == sorted(work.values())  # admitted in increasing work


def test_sjf_waits_for_memory_instead_of_skipping():
    jobs = _jobs(3)
    size = {0: 80, 1: 60, 2: 10}
    work = {0: 3.0, 1: 1.0, 2: 2.0}
    sch = Scheduler(budget_bytes=100, max_active=8, bytes_of=lambda j: size[j.job_id], policy="sjf",
                    work_of=lambda j: work[j.job_id])
    for j in jobs:
        sch.submit(j)
    assert [s.job.job_id for s in sch.admit(0.0)] == [1, 2]  # 60 + 10; job 0 (80) must wait
    assert [s.job.job_id for s in sch.admit(0.1)] == []
    sch.finish(sch.active[1], 0.2)
    assert [s.job.job_id for s in sch.admit(0.2)] == [0]


def test_unknown_policy_rejected():
    import pytest
    with pytest.raises(ValueError):
        Scheduler(budget_bytes=1, policy="lifo", bytes_of=lambda j: 1)


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


def test_lanes_group_batchable_jobs_and_isolate_the_rest():
    """2-D FP32 jobs with a given velocity and at most 4 fields share a lane per field count and
    spline family; FP64, 3-D, wide, carried-velocity (Burgers) and shallow-water jobs get lanes of
    their own.  The memory a job is charged grows with the shallow-water registers."""
    import types

    from paper_1410_2817_gb300 import build, sl
    from paper_1410_2817_gb300.serve import GpuExecutor, JobState
    build.build()
    ex = types.SimpleNamespace(sl=sl, dtype_code=GpuExecutor.dtype_code, tile_config=0)

    def key(wl, dtype="f32", jid=1):
        return GpuExecutor._lane_key(ex, JobState(job=inputs.Job(jid, 0.0, wl, dtype), nbytes=0))

    cubic = inputs.workload_swirl(64)
    quintic = inputs.workload_swirl(64)
    quintic.max_order = 2
    wide = inputs.workload_swirl(64)
    wide.nfields, wide.fields = 5, np.zeros((5, 64, 64))
    assert key(cubic) == ("batch", 3, False) and key(quintic) == ("batch", 3, True)
    assert key(cubic, "f64", 7) == ("job", 7)
    assert key(wide, jid=8) == ("job", 8)
    assert key(inputs.workload_deform3d(16, steps=2), jid=9) == ("job", 9)
    assert key(inputs.workload_burgers(64), jid=10) == ("job", 10)
    assert key(inputs.workload_kelvin(64), jid=11) == ("job", 11)
    plain = inputs.workload_swirl(64)
    kelvin = inputs.workload_kelvin(64)
    b_plain = GpuExecutor.bytes_of(ex, inputs.Job(1, 0.0, plain, "f32"))
    b_kelvin = GpuExecutor.bytes_of(ex, inputs.Job(2, 0.0, kelvin, "f32"))
    # the shallow-water workspace holds 13 more planes; the swirl's holds sin and cos of pi x at its
    # node coordinates (two values per coordinate of each axis), which the shallow-water one lacks
    assert b_kelvin >= b_plain - 2 * (64 + 64) * 4 + 13 * 64 * 64 * 4
