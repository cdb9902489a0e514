"""Trajectory integrators on the CUDA path (Sec. 2, eq. (vel)): Williamson's low-storage
third-order Runge-Kutta scheme and trajectory sub-steps (several integrator steps of dt / k per
remap), against the oracle.  FP64 displacements agree within 1e-12; the FP32 kernels (plain,
tiled 2-D with the next step fused in, blocked 3-D, batches) agree with the plain FP32 path and
with the oracle to FP32 accuracy."""
import math

import numpy as np
import pytest
import torch

from paper_1410_2817_gb300 import inputs
from tests import tiecheck

pytestmark = pytest.mark.gpu

DEV = "cuda"

SCHEMES = [("wrk3", 1), ("wrk3", 3), ("rk4", 4)]


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


def _og(orc, dim, n, nf, kind, params, integrator, substeps, threshold=0.25):
    return orc.OracleGrid(dim=dim, n=n, nfields=nf, velocity=kind, velocity_params=list(params), threshold=threshold,
                          integrator=integrator, substeps=substeps)


@pytest.mark.parametrize("integrator,substeps", SCHEMES)
@pytest.mark.parametrize("kind,dim,n,params,t,dt", [
    ("solid_body", 2, (64, 48), [2 * math.pi, 0.5, 0.5], 0.0, 1 / 64),
    ("swirl2d", 2, (96, 80), [5.0], 0.37, 5 / 96),
    ("deform3d", 3, (14, 12, 10), [3.0], 0.8, 0.03),
    ("fourier2d", 2, (40, 40), inputs.fourier2d_params(np.random.default_rng(1)), 0.0, 0.002),
])
def test_advect_parity_f64(sl, orc, integrator, substeps, kind, dim, n, params, t, dt):
    og = _og(orc, dim, n, 1, kind, params, integrator, substeps)
    ref = orc.advect(og, t, dt)
    g = sl.Grid(dim, n, 1, sl.SL_F64, velocity=kind, velocity_params=list(params), integrator=integrator,
                trajectory_substeps=substeps)
    g.advect(t, dt)
    got = g.get_displacement().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, float(np.abs(ref).max()))


@pytest.mark.parametrize("integrator,substeps", SCHEMES)
@pytest.mark.parametrize("kind,dim,n,params,t,dt", [
    ("swirl2d", 2, (128, 96), [5.0], 0.37, 5 / 128),
    ("deform3d", 3, (16, 12, 10), [3.0], 0.8, 0.03),
])
def test_advect_f32_accuracy(sl, orc, integrator, substeps, kind, dim, n, params, t, dt):
    og = _og(orc, dim, n, 1, kind, params, integrator, substeps)
    ref = orc.advect(og, t, dt)
    g = sl.Grid(dim, n, 1, sl.SL_F32, velocity=kind, velocity_params=list(params), integrator=integrator,
                trajectory_substeps=substeps)
    g.advect(t, dt)
    got = g.get_displacement().double().cpu().numpy()[..., :dim]
    # k sub-steps accumulate k roundings of the FP32 position
    assert np.max(np.abs(got - ref)) <= 2e-6 * substeps * float(np.abs(ref).max())
    assert np.all(got[ref == 0.0] == 0.0)


@pytest.mark.parametrize("integrator,substeps", SCHEMES)
@pytest.mark.parametrize("name,nsteps", [("swirl128", 6), ("deform3d16", 3)])
def test_step_parity_f64(sl, orc, integrator, substeps, name, nsteps):
    wl = inputs.workload_swirl(128, steps=nsteps) if name == "swirl128" else inputs.workload_deform3d(16, steps=nsteps)
    og = orc.OracleGrid(dim=wl.dim, n=wl.n, nfields=wl.nfields, velocity=wl.velocity,
                        velocity_params=list(wl.velocity_params), max_order=wl.max_order, threshold=wl.threshold,
                        start=orc.START_PAPER, integrator=integrator, substeps=substeps)
    g = sl.grid_for(wl, sl.SL_F64, walk_start=sl.SL_START_PAPER, integrator=integrator,
                    trajectory_substeps=substeps)
    # every step within 1e-12 of the oracle's from the same fields but for face ties; one call of
    # nsteps = the chained steps bit for bit
    _, beyond, ties = tiecheck.f64_run_ties(orc, og, g, wl.fields, wl.t0, wl.dt, nsteps)
    assert beyond == ties


@pytest.mark.parametrize("integrator,substeps", SCHEMES)
@pytest.mark.parametrize("tile_config", [1, 5])
def test_fused_tiled_step_matches_plain_f32(sl, integrator, substeps, tile_config):
    """The tiled 2-D step integrates the next step's trajectories (all sub-steps) in the remap
    launch: still one launch per step, and the plain FP32 path's values."""
    wl = inputs.workload_swirl(192, steps=5)
    kw = dict(integrator=integrator, trajectory_substeps=substeps)
    gt = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_AUTO, tile_config=tile_config, **kw)
    gg = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_GENERIC, **kw)
    ft = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    fg = ft.clone()
    l0 = gt.diagnostics()["kernel_launches"]
    gt.step(ft, torch.empty_like(ft), 0.25, wl.dt, 4)
    assert gt.diagnostics()["kernel_launches"] - l0 == 1 + 4  # one advect, then one launch per step
    gg.step(fg, torch.empty_like(fg), 0.25, wl.dt, 4)
    torch.cuda.synchronize()
    diff = (ft - fg).abs()
    assert float((diff > 2e-6).float().mean()) <= 1e-4 and float(diff.max()) <= 1e-3, float(diff.max())
    # the displacement left for the step after the call is sl_advect_nodes' at that time
    d_fused = gt.get_displacement()
    gg.advect(0.25 + 4 * wl.dt, wl.dt)
    d_plain = gg.get_displacement()
    assert float((d_fused - d_plain).abs().max()) <= 1e-6 * float(d_plain.abs().max())


@pytest.mark.parametrize("integrator,substeps", [("wrk3", 2), ("rk4", 3)])
def test_fused_blocked3d_step_matches_plain_f32(sl, integrator, substeps):
    wl = inputs.workload_deform3d(24, steps=3)
    kw = dict(integrator=integrator, trajectory_substeps=substeps)
    out = {}
    for name, kern in (("tiled", sl.SL_KERNEL_TILED), ("generic", sl.SL_KERNEL_GENERIC)):
        g = sl.grid_for(wl, sl.SL_F32, kernel=kern, **kw)
        f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
        g.step(f, torch.empty_like(f), wl.t0, wl.dt, 3)
        torch.cuda.synchronize()
        out[name] = f.double().cpu().numpy()
    diff = np.abs(out["tiled"] - out["generic"])
    scale = max(1.0, float(np.abs(out["generic"]).max()))
    assert float((diff > 4e-6 * scale).mean()) <= 1e-4 and float(diff.max()) <= 1e-3 * scale, float(diff.max())


def test_fp32_wrk3_step_accuracy_against_oracle(sl, orc):
    """FP32 steps with the paper's integrator track the FP64 oracle (same integrator) to FP32
    accuracy in L1 over a few steps of the swirl."""
    wl = inputs.workload_swirl(128, steps=4)
    og = orc.OracleGrid(dim=2, n=wl.n, nfields=wl.nfields, velocity=wl.velocity,
                        velocity_params=list(wl.velocity_params), max_order=wl.max_order, threshold=wl.threshold,
                        start=orc.START_BACKWARD, integrator="wrk3", substeps=2)
    ref, _ = orc.step(og, wl.fields, wl.t0, wl.dt, 4)
    g = sl.grid_for(wl, sl.SL_F32, integrator="wrk3", trajectory_substeps=2)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    g.step(f, torch.empty_like(f), wl.t0, wl.dt, 4)
    torch.cuda.synchronize()
    got = f.double().cpu().numpy()
    for q in range(wl.nfields):
        l1 = np.abs(got[q] - ref[q]).sum() / max(np.abs(ref[q]).sum(), 1e-30)
        assert l1 <= 1e-4, (q, l1)


@pytest.mark.parametrize("integrator,substeps", [("wrk3", 1), ("wrk3", 3), ("rk4", 2)])
def test_batch_integrators_match_grids_alone(sl, integrator, substeps):
    """Batches evaluate the time factors of every sub-step's stages on the device from each grid's
    time: the batch gives what each grid gives alone (time-dependent swirls at different times)."""
    wls = [inputs.workload_swirl(n, steps=3) for n in (64, 96, 80)]
    kw = dict(integrator=integrator, trajectory_substeps=substeps)
    grids, fields, scratch = [], [], []
    for wl in wls:
        grids.append(sl.grid_for(wl, sl.SL_F32, **kw))
        fields.append(torch.tensor(wl.fields, dtype=torch.float32, device=DEV))
        scratch.append(torch.empty_like(fields[-1]))
    t0 = [0.3, 1.1, 2.0]
    b = sl.Batch(grids, fields, scratch, t0, [wl.dt for wl in wls])
    b.step(3)
    b.step(2)
    torch.cuda.synchronize()
    for q, wl in enumerate(wls):
        g = sl.grid_for(wl, sl.SL_F32, **kw)
        f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
        g.step(f, torch.empty_like(f), t0[q], wl.dt, 5)
        torch.cuda.synchronize()
        diff = (fields[q] - f).abs()
        assert float((diff > 1e-5).float().mean()) <= 1e-3 and float(diff.max()) <= 0.2, (q, float(diff.max()))
