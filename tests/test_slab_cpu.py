"""One grid split into slabs of rows across CPU ranks (gloo, world size 2), stepped by the oracle.

Each rank owns a slab of rows and, every step, receives from its neighbours (periodic ring) a halo
of H = ceil(max |D_y|) + m_max + 2 rows of every field: the element holding a target's departure
point lies within ceil(max |D_y|) + 1 rows of it, the Z-spline stencil reaches m_max + 1 rows
further, and the jump flags of those nodes need one more row (Sec. 2.2, 2.3).  The displacement
comes from the analytic velocity, so it needs no exchange; max |D_y| is one all-reduce (MAX).  The
rank builds a full-size plane that holds only its own rows and its halos -- NaN everywhere else,
so that any value read beyond the halo would poison its targets -- and remaps it with the oracle.
Its own rows must equal the single-domain oracle's bit for bit, every step.  The discrete moments
(Sec. 3.1) of the whole field are one all-reduce (SUM) of the ranks' partial sums.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1410_2817_gb300 import inputs

NX, NY, NF, STEPS = 48, 64, 3, 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _grid(oracle):
    wl = inputs.workload_swirl(64, steps=STEPS)
    return wl, oracle.OracleGrid(dim=2, n=(NX, NY), nfields=NF, velocity=wl.velocity,
                                 velocity_params=list(wl.velocity_params))


def _fields():
    return np.stack([inputs.swirl_fields(64)[f][:NY, :NX] for f in range(NF)])


def _exchange(rank, world, own, y0, y1, H):
    """Halo rows from the ring neighbours: rows [y0 - H, y0) come from the rank below, rows
    [y1, y1 + H) from the rank above (periodic)."""
    below, above = (rank - 1) % world, (rank + 1) % world
    send_up = torch.from_numpy(np.ascontiguousarray(own[:, -H:, :]))    # my top rows: the halo below the rank above
    send_down = torch.from_numpy(np.ascontiguousarray(own[:, :H, :]))   # my bottom rows: the halo above the rank below
    recv_below = torch.empty_like(send_up)
    recv_above = torch.empty_like(send_down)
    reqs = [dist.isend(send_up, above, tag=1), dist.isend(send_down, below, tag=2),
            dist.irecv(recv_below, below, tag=1), dist.irecv(recv_above, above, tag=2)]
    for r in reqs:
        r.wait()
    return recv_below.numpy(), recv_above.numpy()


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle
    wl, og = _grid(oracle)
    rows = NY // world
    y0, y1 = rank * rows, (rank + 1) * rows
    own = _fields()[:, y0:y1, :].copy()
    t, halos = wl.t0, []
    for k in range(STEPS):
        D = oracle.advect(og, t, wl.dt)  # analytic: any rank evaluates it where it needs it
        dmax = torch.tensor([float(np.abs(D[y0:y1, :, 1]).max())], dtype=torch.float64)
        dist.all_reduce(dmax, op=dist.ReduceOp.MAX)
        H = int(math.ceil(dmax.item())) + og.max_order + 2
        halos.append(H)
        lo, hi = _exchange(rank, world, own, y0, y1, H)
        full = np.full((NF, NY, NX), np.nan)
        full[:, y0:y1, :] = own
        full[:, [(y0 - H + i) % NY for i in range(H)], :] = lo
        full[:, [(y1 + i) % NY for i in range(H)], :] = hi
        out = oracle.remap_values(og, D, oracle.flags(og, full), full)
        own = out[:, y0:y1, :].copy()
        t = t + wl.dt
    # moments of the whole first field: partial sums of the own rows, one all-reduce
    part = np.zeros((NY, NX))
    part[y0:y1] = own[0]
    m = torch.from_numpy(oracle.moments(og, part, 4))
    dist.all_reduce(m, op=dist.ReduceOp.SUM)
    gathered = [None] * world
    dist.all_gather_object(gathered, {"rank": rank, "rows": (y0, y1), "own": own, "halos": halos})
    if rank == 0:
        q.put((gathered, m.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_slabs_with_exchanged_halos_equal_one_domain(oracle_mod):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, m = q.get(timeout=170)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl, og = _grid(oracle_mod)
    ref, nfail = oracle_mod.step(og, _fields(), wl.t0, wl.dt, STEPS)
    assert nfail == 0
    for g in gathered:
        y0, y1 = g["rows"]
        assert np.isfinite(g["own"]).all(), "a value beyond the halo reached a target"
        assert np.array_equal(g["own"], ref[:, y0:y1, :]), g["rank"]
        assert min(g["halos"]) >= 3 and max(g["halos"]) < NY // 2
    m_ref = oracle_mod.moments(og, ref[0], 4)
    assert np.allclose(m, m_ref, rtol=1e-13, atol=1e-13 * abs(m_ref[0]))


def test_halo_rule_covers_the_smallest_working_halo(oracle_mod):
    """The check has teeth: the smallest halo that reproduces the single domain is found by
    trying widths from 0 up, one row fewer lets NaN or a wrong flag reach a target, and the rule's
    width is at least the smallest one (the rule bounds the worst case)."""
    wl, og = _grid(oracle_mod)
    h = _fields()
    y0, y1 = 0, NY // 2
    for k, t in enumerate((wl.t0, wl.t0 + 3 * wl.dt)):
        D = oracle_mod.advect(og, t, wl.dt)
        ref = oracle_mod.remap_values(og, D, oracle_mod.flags(og, h), h)[:, y0:y1, :]

        def works(H):
            full = np.full_like(h, np.nan)
            keep = [(y0 - H + i) % NY for i in range(H)] + list(range(y0, y1)) + [(y1 + i) % NY for i in range(H)]
            full[:, keep, :] = h[:, keep, :]
            out = oracle_mod.remap_values(og, D, oracle_mod.flags(og, full), full)[:, y0:y1, :]
            return bool(np.isfinite(out).all() and np.array_equal(out, ref))

        h_min = next(H for H in range(NY // 2) if works(H))
        rule = int(math.ceil(float(np.abs(D[:, :, 1]).max()))) + og.max_order + 2
        assert h_min >= 2 and not works(h_min - 1)
        assert rule >= h_min, (k, rule, h_min)
