"""Continuous-batching server on the GPU: jobs arriving while others run are admitted as memory
frees up, every active job advances each iteration (2-D FP32 jobs batched, 3-D and FP64 jobs on
concurrent streams), and each job's result is the same alone and in the mix, bit for bit."""
import numpy as np
import pytest
import torch

from paper_1410_2817_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1410_2817_gb300 import build, serve as srv, sl
    build.build()
    sl.lib()
    return srv


def _trace():
    jobs = inputs.serving_trace(njobs=16, seed=4, rate_hz=120.0, frac_3d=0.3, frac_f64=0.25, side2d=(24, 96),
                                side3d=(10, 18), steps=(3, 7))
    return jobs


def _fields_of(job):
    wl = job.workload
    return inputs.job_fields_device(wl.dim, wl.n[0], wl.nfields, seed=1000 + job.job_id)


@pytest.mark.parametrize("policy,max_active", [("fifo", 4096), ("sjf", 4)])
def test_mix_equals_alone(serve, policy, max_active):
    jobs = _trace()
    kinds = {(j.workload.dim, j.dtype) for j in jobs}
    assert (2, "f32") in kinds and (3, "f32") in kinds and any(d == "f64" for _, d in kinds)
    mix = serve.serve_trace(jobs, _fields_of, budget_bytes=8 << 30, keep_results=True, policy=policy,
                            max_active=max_active)
    assert mix["completed"] == len(jobs) and mix["rejected"] == 0
    assert mix["peak_active"] >= 2  # arrivals overlapped with running jobs
    for job in jobs:
        alone_job = inputs.Job(job.job_id, 0.0, job.workload, job.dtype)
        alone = serve.serve_trace([alone_job], _fields_of, budget_bytes=8 << 30, keep_results=True)
        a, b = mix["results"][job.job_id], alone["results"][job.job_id]
        # a job runs the same kernels on the same inputs in the mix and alone: bit for bit
        assert np.array_equal(a, b), (job.job_id, job.workload.dim, job.dtype, float(np.abs(a - b).max()))
    assert mix["latency_s"]["p50"] is not None and mix["latency_s"]["p99"] >= mix["latency_s"]["p50"]


def test_budget_limits_resident_jobs(serve):
    jobs = _trace()[:8]
    ex = serve.GpuExecutor()
    sizes = [ex.bytes_of(j) for j in jobs]
    budget = 2 * max(sizes)
    out = serve.serve_trace(jobs, _fields_of, budget_bytes=budget, executor=ex)
    ex.close()
    assert out["completed"] == len(jobs)
    assert out["peak_bytes"] <= budget


def test_oversized_job_rejected(serve):
    jobs = _trace()[:4]
    ex = serve.GpuExecutor()
    big = max(jobs, key=ex.bytes_of)
    budget = sorted(ex.bytes_of(j) for j in jobs)[-2]  # everything but the largest fits
    out = serve.serve_trace(jobs, _fields_of, budget_bytes=budget, executor=ex)
    ex.close()
    assert out["rejected"] == sum(1 for j in jobs if ex.bytes_of(j) > budget) >= 1
    assert out["completed"] == len(jobs) - out["rejected"]
    del big


def test_served_job_accuracy(serve):
    from oracle import oracle
    jobs = [j for j in inputs.serving_trace(njobs=40, seed=9, side2d=(40, 64), side3d=(10, 12), steps=(3, 4))
            if j.workload.dim == 2 and j.dtype == "f32"][:2]
    out = serve.serve_trace(jobs, _fields_of, budget_bytes=4 << 30, keep_results=True)
    for j in jobs:
        wl = j.workload
        h0 = _fields_of(j).cpu().numpy()
        og = oracle.OracleGrid(dim=2, n=wl.n, nfields=wl.nfields, velocity=wl.velocity,
                               velocity_params=wl.velocity_params)
        ref, _ = oracle.step(og, h0, 0.0, wl.dt, wl.steps)
        got = out["results"][j.job_id].astype(np.float64)
        l1 = np.abs(got[0] - ref[0]).sum() / np.abs(ref[0]).sum()
        assert l1 <= 1e-5, l1


def test_other_job_kinds_in_the_mix(serve):
    """Quintic, Burgers (carried velocity) and shallow-water jobs served beside ordinary ones: the
    quintic jobs share a batch lane of their own, the Burgers and shallow-water jobs run in their
    own lanes, and every result equals the job run alone."""
    base = _trace()[:6]
    z2 = inputs.workload_swirl(64, steps=4)
    z2.max_order = 2
    extra = [z2, inputs.workload_burgers(64, steps=5), inputs.workload_kelvin(64)]
    extra[2].steps = 4
    jobs = list(base)
    for q, wl in enumerate(extra):
        jobs.append(inputs.Job(100 + q, 0.01 * q, wl, "f32"))

    def fields_of(job):
        wl = job.workload
        if job.job_id >= 100:
            return torch.tensor(wl.fields, dtype=torch.float32, device="cuda")
        return _fields_of(job)

    mix = serve.serve_trace(jobs, fields_of, budget_bytes=8 << 30, keep_results=True)
    assert mix["completed"] == len(jobs) and mix["rejected"] == 0
    for job in jobs:
        alone = serve.serve_trace([inputs.Job(job.job_id, 0.0, job.workload, job.dtype)], fields_of,
                                  budget_bytes=8 << 30, keep_results=True)
        a, b = mix["results"][job.job_id], alone["results"][job.job_id]
        assert np.array_equal(a, b), (job.job_id, job.workload.name, float(np.abs(a - b).max()))
