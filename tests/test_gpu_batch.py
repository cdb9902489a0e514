"""Batched grids (sl_batch_*): a persistent launch per step over a work-list of (grid, tile) items.

Each grid advanced in a batch must give what it gives when stepped alone with sl_step (same tiled
FP32 code per tile; the first step's trajectories come from a different launch, so equality is to
FP32 rounding), a captured CUDA graph must replay exactly what the direct launches compute, and
the FP32 results must stay within the FP32 path's accuracy of the FP64 oracle.
"""
import math

import numpy as np
import pytest
import torch

from paper_1410_2817_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1410_2817_gb300 import build, sl as slmod
    build.build()
    slmod.lib()
    return slmod


def _small_batch(count, seed, side_lo=24, side_hi=96, steps=4):
    wls = inputs.batched_grids(count=count, seed=seed, steps=steps, side_lo=side_lo, side_hi=side_hi)
    return wls


def _make(sl, wls, tile_config=0, velocity_override=None):
    grids, fields, scratch = [], [], []
    for wl in wls:
        g = sl.grid_for(wl, sl.SL_F32, tile_config=tile_config)
        grids.append(g)
        fields.append(torch.tensor(wl.fields, dtype=torch.float32, device=DEV))
        scratch.append(torch.empty_like(fields[-1]))
    return grids, fields, scratch


def _alone(sl, wl, nsteps, t0, tile_config=0, diag=None):
    g = sl.grid_for(wl, sl.SL_F32, tile_config=tile_config)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    g.step(f, torch.empty_like(f), t0, wl.dt, nsteps)
    torch.cuda.synchronize()
    if diag is not None:
        diag.update(g.diagnostics())
    return f.cpu().numpy()


def _fails(d):
    return d["fail_locate"] + d["fail_newton"] + d["fail_fold"]


def _same(a, b):
    """A grid in a batch runs the single-grid tile body on the same inputs: bit for bit."""
    return np.array_equal(a, b)


@pytest.mark.parametrize("tile_config", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("nsteps", [3, 4])
def test_batch_matches_grids_alone(sl, tile_config, nsteps):
    wls = _small_batch(9, seed=3)
    grids, fields, scratch = _make(sl, wls, tile_config)
    t0 = [0.0] * len(wls)
    b = sl.Batch(grids, fields, scratch, t0, [wl.dt for wl in wls], tile_config=tile_config)
    b.step(nsteps)
    torch.cuda.synchronize()
    for q, wl in enumerate(wls):
        dref = {}
        ref = _alone(sl, wl, nsteps, 0.0, tile_config, dref)
        got = fields[q].cpu().numpy()
        assert _same(got, ref), (q, wl.n, float(np.abs(got - ref).max()))
        d = grids[q].diagnostics()
        assert d["targets"] == nsteps * wl.nnodes
        # the random flows at CFL 4 fold some elements of the small grids (strain x dt > 1): the
        # batch meets exactly the failures the grid meets alone
        assert _fails(d) == _fails(dref), (_fails(d), _fails(dref))
    info = b.info()
    assert info["launches"] == nsteps + 2
    assert math.isclose(info["t_first"], nsteps * wls[0].dt)


@pytest.mark.parametrize("tile_config", [1, 3])
def test_quintic_batch_matches_grids_alone(sl, tile_config):
    """Grids with the quintic Z-spline run in one batch on the quintic tile body (32 x 32 tiles
    whatever the tile configuration) and give what each grid gives alone."""
    wls = _small_batch(7, seed=13)
    for wl in wls:
        wl.max_order = 2
    grids, fields, scratch = _make(sl, wls, tile_config)
    b = sl.Batch(grids, fields, scratch, [0.0] * len(wls), [wl.dt for wl in wls], tile_config=tile_config)
    b.step(3)
    torch.cuda.synchronize()
    for q, wl in enumerate(wls):
        dref = {}
        ref = _alone(sl, wl, 3, 0.0, tile_config, dref)
        got = fields[q].cpu().numpy()
        assert _same(got, ref), (q, wl.n, float(np.abs(got - ref).max()))
        d = grids[q].diagnostics()
        assert d["order_hist"][2] > 0
        assert _fails(d) == _fails(dref)
    assert b.info()["launches"] == 3 + 2


def test_batch_rejects_mixed_orders(sl):
    a = sl.Grid(2, (40, 40), 2, sl.SL_F32, max_order=1)
    c = sl.Grid(2, (40, 40), 2, sl.SL_F32, max_order=2)
    assert sl.sl_batch_workspace_bytes([a, c]) == 0
    f = [torch.zeros((2, 40, 40), device=DEV) for _ in range(2)]
    s = [torch.zeros_like(x) for x in f]
    with pytest.raises(sl.SLError) as ei:
        sl.Batch([a, c], f, s, [0.0, 0.0], [0.01, 0.01])
    assert ei.value.status == sl.SL_ERR_UNSUPPORTED


def test_graph_replay_equals_direct_launches(sl):
    wls = _small_batch(7, seed=5)
    res = {}
    for use_graph in (False, True):
        grids, fields, scratch = _make(sl, wls)
        stream = torch.cuda.Stream()
        b = sl.Batch(grids, fields, scratch, [0.0] * len(wls), [wl.dt for wl in wls])
        with torch.cuda.stream(stream):
            for _ in range(3):  # three calls: the graph is captured once and replayed twice
                b.step(5, use_graph=use_graph, stream=stream)
        stream.synchronize()
        res[use_graph] = [f.cpu().numpy() for f in fields]
    for a, c in zip(res[False], res[True]):
        assert np.array_equal(a, c)


def test_time_dependent_velocity_in_a_batch(sl):
    """The swirl's cos(pi t / T) factor is evaluated per step on the device from each grid's time."""
    wls = [inputs.workload_swirl(n, steps=3) for n in (64, 96, 80)]
    for wl in wls:
        wl.fields = wl.fields[:2]
        wl.nfields = 2
    grids, fields, scratch = _make(sl, wls)
    t0 = [0.3, 1.1, 2.0]
    b = sl.Batch(grids, fields, scratch, t0, [wl.dt for wl in wls])
    b.step(3)
    b.step(2)  # continues from the device-side times
    torch.cuda.synchronize()
    for q, wl in enumerate(wls):
        ref = _alone(sl, wl, 5, t0[q])
        got = fields[q].cpu().numpy()
        assert _same(got, ref), (q, float(np.abs(got - ref).max()))


def test_batch_accuracy_against_oracle(sl):
    """Against the FP64 oracle.  One batch step, target by target, with the displacement each grid
    integrated on the GPU: every value is the oracle's interpolation in the oracle's element and
    order (within 2e-6, or a face or limiter tie), and exactly the targets where the oracle's
    search fails (the random flows at CFL 4 fold elements of the smaller grids) keep their
    values.  Three steps with each side's own trajectories: the smooth Gaussian within 1e-5 in
    relative L1 and its moments m_0..m_2 within 1e-6 of its L1 mass."""
    from oracle import oracle
    from tests import tiecheck
    wls = _small_batch(4, seed=11, side_lo=48, side_hi=64, steps=3)
    grids, fields, scratch = _make(sl, wls)
    b = sl.Batch(grids, fields, scratch, [0.0] * 4, [wl.dt for wl in wls])
    b.step(1)
    torch.cuda.synchronize()
    for q, wl in enumerate(wls):
        og = oracle.OracleGrid(dim=2, n=wl.n, nfields=2, velocity=wl.velocity, velocity_params=wl.velocity_params,
                               start=oracle.START_BACKWARD)
        D32 = grids[q].get_displacement().cpu().numpy()[..., :2]
        h32 = np.asarray(wl.fields, dtype=np.float32)
        counts = tiecheck.f32_remap_targets(oracle, og, D32, h32, fields[q].double().cpu().numpy(), 2e-6)
        d = grids[q].diagnostics()
        assert _fails(d) == counts["oracle_failed"], (q, _fails(d), counts)
    b.step(2)
    torch.cuda.synchronize()
    for q, wl in enumerate(wls):
        og = oracle.OracleGrid(dim=2, n=wl.n, nfields=2, velocity=wl.velocity, velocity_params=wl.velocity_params)
        ref, _ = oracle.step(og, wl.fields, 0.0, wl.dt, 3)
        got = fields[q].double().cpu().numpy()
        l1 = np.abs(got[0] - ref[0]).sum() / np.abs(ref[0]).sum()  # the smooth Gaussian
        assert l1 <= 1e-5, (q, l1)
        mr, mg = oracle.moments(og, ref[0], 2), oracle.moments(og, got[0], 2)
        mass = float(np.abs(ref[0]).sum())
        assert np.max(np.abs(mg - mr)) <= 1e-6 * mass, (q, mg, mr)


def test_batch_rejects_ineligible_grids(sl):
    g64 = sl.Grid(2, (32, 32), 2, sl.SL_F64)
    assert sl.sl_batch_workspace_bytes([g64]) == 0
    g3d = sl.Grid(3, (16, 16, 16), 2, sl.SL_F32)
    assert sl.sl_batch_workspace_bytes([g3d]) == 0
    # the tile bodies invert in FP32: a grid that asks for FP64 inversion of every target is not batched
    gn = sl.Grid(2, (32, 32), 2, sl.SL_F32, newton_mode=sl.SL_NEWTON_F64)
    assert sl.sl_batch_workspace_bytes([gn]) == 0
    a = sl.Grid(2, (32, 32), 2, sl.SL_F32)
    c = sl.Grid(2, (32, 32), 3, sl.SL_F32)
    f = [torch.zeros((2, 32, 32), device=DEV), torch.zeros((3, 32, 32), device=DEV)]
    s = [torch.zeros_like(x) for x in f]
    with pytest.raises(sl.SLError) as ei:
        sl.Batch([a, c], f, s, [0.0, 0.0], [0.1, 0.1])
    assert ei.value.status == sl.SL_ERR_UNSUPPORTED


def test_autotuner_picks_a_valid_configuration(sl):
    from paper_1410_2817_gb300 import autotune
    wls = _small_batch(6, seed=13, side_lo=64, side_hi=160)
    r = autotune.tune_batch(wls, steps_per_trial=2, repeats=2)
    assert r["best"] in autotune.CONFIGS and set(r["ms_per_call"]) == set(autotune.CONFIGS)
    assert all(v > 0 for v in r["ms_per_call"].values())
    rg = autotune.tune_grid(inputs.workload_swirl(256, steps=2), repeats=2)
    assert rg["best"] in autotune.CONFIGS
