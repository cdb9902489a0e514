"""The carried velocity on the CUDA path (Sec. 3.2, Burgers): the velocity components are
transported fields and every node moves with the value it carries.  FP64 trajectories and steps
match the oracle within 1e-12; the FP32 tiled path (a trajectory launch plus the tiled remap per
step) matches the plain FP32 path and the oracle to FP32 accuracy."""
import numpy as np
import pytest
import torch

from paper_1410_2817_gb300 import inputs
from tests import tiecheck

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


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("dim,params", [(2, []), (2, [2, 0]), (3, []), (3, [1, 2, 0])])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_advect_carried_parity(sl, orc, dim, params, dtype):
    n = (40, 24) if dim == 2 else (12, 10, 8)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(21)
    h = rng.uniform(-1.0, 1.0, size=(3,) + shape)
    dt = 0.011
    og = orc.OracleGrid(dim=dim, n=n, nfields=3, velocity="carried", velocity_params=params)
    ref = orc.advect_carried(og, h, dt)
    sd, td = (sl.SL_F64, torch.float64) if dtype == "f64" else (sl.SL_F32, torch.float32)
    g = sl.Grid(dim, n, 3, sd, velocity="carried", velocity_params=params)
    g.advect_carried(torch.tensor(h, dtype=td, device=DEV), dt)
    got = g.get_displacement().double().cpu().numpy()[..., :dim]
    tol = 1e-12 if dtype == "f64" else 2e-7
    assert np.max(np.abs(got - ref)) <= tol * max(1.0, float(np.abs(ref).max()))


def test_carried_entry_points_check_the_kind(sl):
    g = sl.Grid(2, (32, 32), 2, sl.SL_F32, velocity="carried", velocity_params=[])
    with pytest.raises(sl.SLError) as ei:
        g.advect(0.0, 0.01)
    assert ei.value.status == sl.SL_ERR_ARG
    ga = sl.Grid(2, (32, 32), 2, sl.SL_F32, velocity="uniform", velocity_params=[0.1, 0.2])
    with pytest.raises(sl.SLError) as ei:
        ga.advect_carried(torch.zeros((2, 32, 32), device=DEV), 0.01)
    assert ei.value.status == sl.SL_ERR_ARG
    assert sl.sl_batch_workspace_bytes([g]) == 0


def _smooth3d(n, seed):
    """Three smooth periodic velocity components (amplitude <= 0.6 of a cell per step at dt) and a
    tracer with a jump."""
    rng = np.random.default_rng(seed)
    x, y, z = inputs.node_coords(n)
    out = []
    for _ in range(3):
        k = rng.integers(1, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        out.append(0.5 * np.sin(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + ph))
    out.append((x > 0.5).astype(np.float64))
    return np.stack(out)


@pytest.mark.parametrize("case", ["burgers128", "burgers_ragged", "carried3d"])
def test_step_parity_f64(sl, orc, case):
    if case == "carried3d":
        n, nsteps = (16, 12, 10), 3
        h = _smooth3d(n, 22)
        dt = 0.6 / 16
        kw = dict(dim=3, n=n, nfields=4)
    else:
        wl = inputs.workload_burgers(128)
        n, nsteps, h, dt = wl.n, 8, wl.fields, wl.dt
        if case == "burgers_ragged":
            n = (100, 72)
            h = inputs.burgers_fields(n)
            dt = 0.5 / 100
        kw = dict(dim=2, n=n, nfields=2)
    og = orc.OracleGrid(velocity="carried", velocity_params=[], start=orc.START_PAPER, **kw)
    g = sl.Grid(kw["dim"], n, kw["nfields"], sl.SL_F64, velocity="carried", velocity_params=[],
                walk_start=sl.SL_START_PAPER)
    # every step within 1e-12 of the oracle's from the same fields (both sides take the velocity
    # from those fields) but for face ties; one call of nsteps = the chained steps bit for bit
    _, beyond, ties = tiecheck.f64_run_ties(orc, og, g, h, 0.1, dt, nsteps, velocity_from_fields=True)
    assert beyond == ties
    d = g.diagnostics()
    assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0


@pytest.mark.parametrize("tile_config", [1, 5])
def test_burgers_f32_tiled_matches_plain(sl, tile_config):
    """Tiled FP32 steps (configuration 1: the remap launch also writes the next step's D from the
    remapped velocity; configuration 5: a trajectory launch and the remap).  From the same
    fields, two steps give the plain FP32 kernels' values up to FP32 rounding (a limiter decision
    at the shock may flip a rare node); checked at several times as the shock forms.  Over many
    steps the velocity feeds back into the trajectories, so the two runs drift apart at the shock
    by more than rounding, but stay within FP32 accuracy in L1."""
    wl = inputs.workload_burgers(256)
    gt = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_AUTO, tile_config=tile_config)
    gg = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_GENERIC, tile_config=tile_config)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    t = 0.0
    for _ in range(4):
        ft, fg = f.clone(), f.clone()
        l0 = gt.diagnostics()["kernel_launches"]
        gt.step(ft, torch.empty_like(ft), t, wl.dt, 2)
        # configuration 1: the first D from the fields, then one remap launch per step that also
        # writes the next D; the pipelined configuration 5: a trajectory launch and a remap per step
        assert gt.diagnostics()["kernel_launches"] - l0 == (1 + 2 if tile_config == 1 else 2 * 2)
        gg.step(fg, torch.empty_like(fg), t, wl.dt, 2)
        torch.cuda.synchronize()
        diff = (ft - fg).abs()
        assert float((diff > 2e-5).float().mean()) <= 1e-3 and float(diff.max()) <= 0.1, float(diff.max())
        gg.step(f, torch.empty_like(f), t, wl.dt, 20)  # advance to the next checkpoint
        t += 20 * wl.dt
    for g in (gt, gg):
        d = g.diagnostics()
        assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0
    # 40 steps each from the initial condition
    ft = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    fg = ft.clone()
    gt.step(ft, torch.empty_like(ft), 0.0, wl.dt, 40)
    gg.step(fg, torch.empty_like(fg), 0.0, wl.dt, 40)
    torch.cuda.synchronize()
    for q in range(2):
        l1 = float((ft[q] - fg[q]).abs().sum() / fg[q].abs().sum())
        assert l1 <= 1e-4, (q, l1)


def test_burgers_f32_against_oracle(sl, orc):
    """FP32 Burgers to t = 0.1 on 128^2 (26 steps) against the FP64 oracle: L1 error of each
    velocity component at FP32 level; the shock front (the ring where the speed drops) sits in the
    same place."""
    wl = inputs.workload_burgers(128)
    nsteps = 26
    og = orc.OracleGrid(dim=2, n=wl.n, nfields=2, velocity="carried", velocity_params=[],
                        start=orc.START_BACKWARD)
    ref, _ = orc.step(og, wl.fields, 0.0, wl.dt, nsteps)
    g = sl.grid_for(wl, sl.SL_F32)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    g.step(f, torch.empty_like(f), 0.0, wl.dt, nsteps)
    torch.cuda.synchronize()
    got = f.double().cpu().numpy()
    for q in range(2):
        l1 = np.abs(got[q] - ref[q]).sum() / np.abs(ref[q]).sum()
        assert l1 <= 1e-4, (q, l1)
    # radial speed profile along the x axis through the centre: same maximum position
    s_ref = np.hypot(ref[0], ref[1])[64, 64:]
    s_got = np.hypot(got[0], got[1])[64, 64:]
    assert int(np.argmax(s_ref)) == int(np.argmax(s_got))


def test_burgers_quintic_fused_matches_plain(sl):
    """Burgers with the quintic Z-spline: the quintic tile kernel writes the next step's D from its
    own remapped velocity as the cubic one does (one launch per step after the first), and two
    steps from the same fields give the plain FP32 kernels' values."""
    wl = inputs.workload_burgers(192)
    wl.max_order = 2
    gt = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_AUTO)
    gg = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_GENERIC)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    gg.step(f, torch.empty_like(f), 0.0, wl.dt, 30)  # let the shock form
    t = 30 * wl.dt
    ft, fg = f.clone(), f.clone()
    l0 = gt.diagnostics()["kernel_launches"]
    gt.step(ft, torch.empty_like(ft), t, wl.dt, 2)
    assert gt.diagnostics()["kernel_launches"] - l0 == 1 + 2
    gg.step(fg, torch.empty_like(fg), t, wl.dt, 2)
    torch.cuda.synchronize()
    diff = (ft - fg).abs()
    assert float((diff > 2e-5).float().mean()) <= 1e-3 and float(diff.max()) <= 0.1, float(diff.max())
    assert gt.diagnostics()["order_hist"][2] > 0
