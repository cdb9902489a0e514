"""Continuous-batching server for advection jobs (FSL steps of arXiv:1410.2817 on many grids).

Jobs arrive over time (2-D or 3-D grids of different sizes, field counts, step counts and
precisions).  The server keeps every admitted job's grid and fields resident in device memory and
advances ALL active jobs by one step per iteration:

* 2-D FP32 jobs with a given velocity, the same field count and the same spline family (cubic /
  linear, or quintic) form one batch (sl_batch_step: one persistent launch over a work-list of
  tiles of all those grids), rebuilt only when its membership changes;
* 3-D, FP64, carried-velocity (Burgers) and shallow-water jobs are stepped with sl_step, each on
  its own stream, so their kernels run concurrently with the batches.

Each of these lanes is relaunched as soon as its previous step has finished (an event per lane,
polled by the host loop): slow FP64 jobs never hold back the FP32 batches.  Arrived jobs are
admitted in arrival order while the device-memory budget and the slot limit allow (a job's bytes:
its grid workspace plus its field and scratch planes) -- or, with policy "sjf", shortest
estimated device work first under a cap on concurrent jobs --, join their lane at its next step,
and are read back and released when done.  A job's result does not depend on what it is batched with:
every tile of a batch runs the same code as the job alone.

`Scheduler` holds the queue/admission/budget logic (no GPU); `GpuExecutor` runs jobs through the C
ABI; `serve_trace` drives a trace in real time and reports latency percentiles and throughput.
`shard_jobs` splits a trace across ranks (independent jobs: no collective on the data path).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np


# ------------------------------------------------------------------------------------------------
# admission and bookkeeping (no GPU)
# ------------------------------------------------------------------------------------------------
@dataclass
class JobState:
    job: object                      # inputs.Job
    nbytes: int
    steps_done: int = 0
    admitted_s: Optional[float] = None
    finished_s: Optional[float] = None
    rejected: bool = False
    handle: object = None            # executor's per-job resources


class Scheduler:
    """Admission under a byte budget and a slot limit.  policy "fifo": in arrival order; "sjf":
    the queued job with the least estimated device work first (`work_of`, ties by arrival), which
    under overload lets short jobs finish instead of every job sharing the device until the end.
    Either way a job that does not fit the budget waits for memory (it is never skipped)."""

    def __init__(self, budget_bytes: int, max_active: int = 4096, bytes_of: Callable[[object], int] = None,
                 policy: str = "fifo", work_of: Callable[[object], float] = None):
        if policy not in ("fifo", "sjf"):
            raise ValueError(f"unknown policy {policy!r}")
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.bytes_of = bytes_of
        self.policy = policy
        self.work_of = work_of or (lambda job: float(job.workload.nnodes * job.workload.steps))
        self.queue: collections.deque = collections.deque()
        self.active: Dict[int, JobState] = {}
        self.done: Dict[int, JobState] = {}
        self.used = 0
        self.peak_used = 0
        self.peak_active = 0

    def submit(self, job) -> JobState:
        st = JobState(job, int(self.bytes_of(job)))
        if st.nbytes > self.budget:
            st.rejected = True
            self.done[job.job_id] = st
        else:
            self.queue.append(st)
        return st

    def _next(self) -> Optional[JobState]:
        if not self.queue:
            return None
        if self.policy == "fifo":
            return self.queue[0]
        return min(self.queue, key=lambda st: (self.work_of(st.job), st.job.arrival_s, st.job.job_id))

    def admit(self, now: float) -> List[JobState]:
        out = []
        while len(self.active) < self.max_active:
            st = self._next()
            if st is None or self.used + st.nbytes > self.budget:
                break
            self.queue.remove(st)
            st.admitted_s = now
            self.active[st.job.job_id] = st
            self.used += st.nbytes
            out.append(st)
        self.peak_used = max(self.peak_used, self.used)
        self.peak_active = max(self.peak_active, len(self.active))
        return out

    def finish(self, st: JobState, now: float):
        st.finished_s = now
        del self.active[st.job.job_id]
        self.used -= st.nbytes
        self.done[st.job.job_id] = st

    def idle(self) -> bool:
        return not self.queue and not self.active


def shard_jobs(jobs: Sequence, rank: int, world: int) -> List:
    """Jobs of one rank: greedy balance of node-steps (largest first), deterministic."""
    if world <= 1:
        return list(jobs)
    load = [0.0] * world
    owner = {}
    for job in sorted(jobs, key=lambda j: (-j.workload.nnodes * j.workload.steps, j.job_id)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[job.job_id] = r
        load[r] += job.workload.nnodes * job.workload.steps
    return [j for j in jobs if owner[j.job_id] == rank]


def percentiles(values: Sequence[float], ps=(50, 99)) -> Dict[str, float]:
    if not values:
        return {f"p{p}": None for p in ps}
    v = np.asarray(values, dtype=np.float64)
    return {f"p{p}": float(np.percentile(v, p)) for p in ps}


# ------------------------------------------------------------------------------------------------
# GPU execution through the C ABI: asynchronous lanes
# ------------------------------------------------------------------------------------------------
class Lane:
    """A unit of work the server relaunches as soon as its previous step has finished: the batch
    of all 2-D FP32 jobs with one field count, or a single other job.  Each lane owns a stream."""

    def __init__(self, key, stream):
        self.key = key
        self.stream = stream
        self.members: List[JobState] = []
        self.running: List[JobState] = []
        self.chunk = 0  # steps of the launch in flight
        self.event = None
        self.batch = None
        self.batch_ids = None


class GpuExecutor:
    """Runs admitted jobs; lanes progress independently (no iteration-wide barrier).  A lane
    advances its jobs by up to `max_chunk` steps per launch (never past a member's last step):
    fewer host round trips, at the price of a new job waiting up to one chunk to join a batch."""

    def __init__(self, tile_config: int = 0, max_chunk: int = 8):
        import torch

        from . import sl
        self.torch, self.sl = torch, sl
        self.tile_config = tile_config
        self.max_chunk = max(1, int(max_chunk))
        self.lanes: Dict[object, Lane] = {}
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
        self.prio_fp64, self.prio_fp32 = lo, hi  # lowest and highest priority the device offers

    @staticmethod
    def dtype_code(sl, job):
        return sl.SL_F64 if job.dtype == "f64" else sl.SL_F32

    def bytes_of(self, job) -> int:
        sl = self.sl
        wl = job.workload
        d = sl.make_desc(wl.dim, list(wl.n)[: wl.dim], wl.nfields, self.dtype_code(sl, job), velocity=wl.velocity,
                         velocity_params=list(wl.velocity_params), tile_config=self.tile_config)
        tsize = 8 if job.dtype == "f64" else 4
        return sl.sl_grid_workspace_bytes(d) + 2 * wl.nfields * wl.nnodes * tsize

    def work_of(self, job) -> float:
        """Relative device time of a job: node-steps, weighted by the measured cost of an FP64
        node-step against an FP32 one (~25x in 2-D, ~30x in 3-D on GB300) and of a 3-D FP32
        node-step against a 2-D one (~1.6x)."""
        wl = job.workload
        w = float(wl.nnodes * wl.steps)
        if wl.dim == 3:
            w *= 1.6
        if job.dtype == "f64":
            w *= 25.0 if wl.dim == 2 else 30.0
        return w

    def _lane_key(self, st: JobState):
        """2-D FP32 jobs with a given velocity and at most 4 fields share a batch lane per field
        count and spline family (cubic / linear, or quintic); the others run in their own lane."""
        wl = st.job.workload
        if (self.dtype_code(self.sl, st.job) == self.sl.SL_F32 and wl.dim == 2 and wl.nfields <= 4
                and wl.velocity not in ("carried", "nlsw")):
            return ("batch", wl.nfields, wl.max_order == 2)
        return ("job", st.job.job_id)

    def start(self, st: JobState, fields):
        """Create the job's grid and resident planes and put it in its lane; `fields` is a host
        array or a CUDA tensor."""
        torch, sl = self.torch, self.sl
        job, wl = st.job, st.job.workload
        code = self.dtype_code(sl, job)
        td = torch.float64 if code == sl.SL_F64 else torch.float32
        key = self._lane_key(st)
        lane = self.lanes.get(key)
        if lane is None:
            # FP32 lanes run at high stream priority: when SMs free up the block scheduler serves
            # them first, so the slow FP64 lanes use the leftover capacity instead of holding the
            # FP32 work back
            prio = self.prio_fp64 if code == sl.SL_F64 else self.prio_fp32
            lane = self.lanes[key] = Lane(key, torch.cuda.Stream(priority=prio))
        g = sl.grid_for(wl, code, tile_config=self.tile_config)
        if isinstance(fields, torch.Tensor):
            f = fields.to(device="cuda", dtype=td).contiguous()
        else:
            f = torch.from_numpy(np.ascontiguousarray(fields)).to(td).pin_memory().to("cuda", non_blocking=True)
        lane.stream.wait_stream(torch.cuda.current_stream())  # the upload precedes the lane's work
        st.handle = {"grid": g, "fields": f, "scratch": torch.empty_like(f), "t": wl.t0, "lane": lane}
        lane.members.append(st)

    def poll(self) -> List[JobState]:
        """Retire the steps that finished; returns the jobs that completed all their steps."""
        done = []
        for lane in list(self.lanes.values()):
            if lane.event is None or not lane.event.query():
                continue
            lane.event = None
            for st in lane.running:
                st.steps_done += lane.chunk
                st.handle["t"] += lane.chunk * st.job.workload.dt
            lane.running = []
            for st in list(lane.members):
                if st.steps_done >= st.job.workload.steps:
                    lane.members.remove(st)
                    done.append(st)
        return done

    def launch_ready(self) -> int:
        """Launch the next step of every idle lane that has jobs; returns how many lanes started."""
        torch, sl = self.torch, self.sl
        started = 0
        for key, lane in list(self.lanes.items()):
            if lane.event is not None:
                continue
            if not lane.members:
                if lane.batch is not None:
                    lane.batch.close()
                    lane.batch, lane.batch_ids = None, None
                continue
            chunk = min([self.max_chunk] + [m.job.workload.steps - m.steps_done for m in lane.members])
            with torch.cuda.stream(lane.stream):
                if key[0] == "batch":
                    ids = tuple(st.job.job_id for st in lane.members)
                    if ids != lane.batch_ids:
                        if lane.batch is not None:
                            lane.batch.close()
                        ms = lane.members
                        lane.batch = sl.Batch([m.handle["grid"] for m in ms], [m.handle["fields"] for m in ms],
                                              [m.handle["scratch"] for m in ms], [m.handle["t"] for m in ms],
                                              [m.job.workload.dt for m in ms], tile_config=self.tile_config)
                        lane.batch_ids = ids
                    lane.batch.step(chunk, use_graph=False, stream=lane.stream)
                else:
                    st = lane.members[0]
                    h = st.handle
                    h["grid"].step(h["fields"], h["scratch"], h["t"], st.job.workload.dt, chunk, stream=lane.stream)
                lane.chunk = chunk
                lane.running = list(lane.members)
                lane.event = torch.cuda.Event()
                lane.event.record(lane.stream)
            started += 1
        return started

    def finish(self, st: JobState) -> np.ndarray:
        h = st.handle
        lane = h["lane"]
        with self.torch.cuda.stream(lane.stream):
            out = h["fields"].cpu().numpy()
        h["grid"].close()
        if lane.key[0] == "job":
            self.lanes.pop(lane.key, None)
        st.handle = None
        return out

    def close(self):
        self.torch.cuda.synchronize()
        for lane in self.lanes.values():
            if lane.batch is not None:
                lane.batch.close()
        self.lanes = {}


def serve_trace(jobs: Sequence, fields_of: Callable[[object], np.ndarray], budget_bytes: int,
                max_active: int = 4096, executor: Optional[GpuExecutor] = None, keep_results: bool = False,
                poll_sleep_s: float = 5e-5, policy: str = "fifo") -> Dict:
    """Serve a trace of inputs.Job in real time (arrival times in seconds from the start).  Returns
    latency percentiles (finish - arrival), throughput, and optionally each job's final fields."""
    ex = executor or GpuExecutor()
    sched = Scheduler(budget_bytes, max_active, ex.bytes_of, policy=policy, work_of=ex.work_of)
    pending = collections.deque(sorted(jobs, key=lambda j: j.arrival_s))
    results = {}
    t_start = time.perf_counter()
    lane_steps = 0
    while pending or not sched.idle():
        now = time.perf_counter() - t_start
        while pending and pending[0].arrival_s <= now:
            sched.submit(pending.popleft())
        for st in ex.poll():
            out = ex.finish(st)
            if keep_results:
                results[st.job.job_id] = out
            sched.finish(st, time.perf_counter() - t_start)
        for st in sched.admit(time.perf_counter() - t_start):
            ex.start(st, fields_of(st.job))
        started = ex.launch_ready()
        lane_steps += started
        if not started:
            time.sleep(poll_sleep_s)
    makespan = time.perf_counter() - t_start
    if executor is None:
        ex.close()
    done = [st for st in sched.done.values() if not st.rejected]
    lat = [st.finished_s - st.job.arrival_s for st in done]
    total = sum(st.job.workload.nnodes * st.job.workload.steps for st in done)
    offered = sum(j.workload.nnodes * j.workload.steps for j in jobs)
    last_arrival = max((j.arrival_s for j in jobs), default=0.0)
    by_kind = collections.defaultdict(list)
    work_kind = collections.defaultdict(float)
    offered_kind = collections.defaultdict(float)
    for st in done:
        kind = f"{st.job.workload.dim}d_{st.job.dtype}"
        by_kind[kind].append(st.finished_s - st.job.arrival_s)
        work_kind[kind] += st.job.workload.nnodes * st.job.workload.steps
    for j in jobs:
        offered_kind[f"{j.workload.dim}d_{j.dtype}"] += j.workload.nnodes * j.workload.steps
    return {
        "jobs": len(jobs), "completed": len(done), "rejected": sum(1 for s in sched.done.values() if s.rejected),
        "latency_s": percentiles(lat), "mean_latency_s": float(np.mean(lat)) if lat else None,
        "latency_by_kind_s": {k: percentiles(v) for k, v in sorted(by_kind.items())},
        "makespan_s": makespan, "lane_steps": lane_steps, "node_steps": total,
        "achieved_node_updates_per_s": total / makespan if makespan > 0 else None,
        "offered_node_updates_per_s": offered / last_arrival if last_arrival > 0 else None,
        # per job kind: node-updates offered per second of arrivals, and completed per second of
        # the whole run (the kinds share the device, so these add up to the totals above)
        "node_updates_per_s_by_kind": {
            k: {"offered": offered_kind[k] / last_arrival if last_arrival > 0 else None,
                "achieved": work_kind[k] / makespan if makespan > 0 else None}
            for k in sorted(offered_kind)},
        "peak_active": sched.peak_active, "peak_bytes": sched.peak_used, "budget_bytes": budget_bytes,
        "policy": policy, "max_active": max_active,
        "results": results if keep_results else None,
    }
