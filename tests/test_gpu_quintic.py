"""The quintic Z-spline Z2 (m_max = 2, six points per axis, orders 2 -> 1 -> 0 near jumps;
Sec. 2.1 and the Appendix) on the CUDA path: whole FP64 steps against the oracle within 1e-12,
FP32 steps to FP32 accuracy, and sampled targets of the 1024^2 swirl at full size."""
import numpy as np
import pytest
import torch

from paper_1410_2817_gb300 import inputs
from tests import tiecheck

pytestmark = pytest.mark.gpu

DEV = "cuda"
TIE = 1e-9


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


def _og(orc, wl, start):
    return orc.OracleGrid(dim=wl.dim, n=wl.n, nfields=wl.nfields, velocity=wl.velocity,
                          velocity_params=list(wl.velocity_params), max_order=wl.max_order, threshold=wl.threshold,
                          start=start)


@pytest.mark.parametrize("name,nsteps", [("swirl128", 8), ("sbr64", 12), ("deform3d16", 3)])
def test_step_parity_f64(sl, orc, name, nsteps):
    """Quintic FP64 steps, each from the GPU's previous result on both sides: every target within
    1e-12 of the oracle unless it is a face tie (the GPU's own element contains it and gives the
    oracle's interpolation there); all three orders occur; one call of nsteps reproduces the
    chained steps bit for bit."""
    if name == "swirl128":
        wl = inputs.workload_swirl(128, steps=nsteps)
    elif name == "sbr64":
        wl = inputs.workload_sbr64()
    else:
        wl = inputs.workload_deform3d(16, steps=nsteps)
    wl.max_order = 2
    og = _og(orc, wl, orc.START_PAPER)
    g = sl.grid_for(wl, sl.SL_F64, walk_start=sl.SL_START_PAPER)
    _, beyond, ties = tiecheck.f64_run_ties(orc, og, g, wl.fields, wl.t0, wl.dt, nsteps)
    assert beyond == ties
    d = g.diagnostics()
    assert d["order_hist"][2] > 0 and d["order_hist"][1] > 0 and d["order_hist"][0] > 0


def test_fp32_step_accuracy(sl, orc):
    wl = inputs.workload_swirl(256, steps=10)
    wl.max_order = 2
    ref, _ = orc.step(_og(orc, wl, orc.START_BACKWARD), wl.fields, wl.t0, wl.dt, 10)
    g = sl.grid_for(wl, sl.SL_F32)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    g.step(f, torch.empty_like(f), wl.t0, wl.dt, 10)
    torch.cuda.synchronize()
    got = f.double().cpu().numpy()
    for q, name in ((0, "gaussian"), (2, "sine")):
        l1 = np.abs(got[q] - ref[q]).sum() / np.abs(ref[q]).sum()
        assert l1 <= 1e-5, (name, l1)
    og1 = orc.OracleGrid(dim=2, n=wl.n, nfields=1)
    for q in (0, 2):
        mr, mg = orc.moments(og1, ref[q], 2), orc.moments(og1, got[q], 2)
        l1 = float(np.abs(ref[q]).sum())
        for p in range(3):
            assert abs(mg[p] - mr[p]) <= 1e-6 * l1, (q, p, mg[p], mr[p])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_sampled(sl, orc, dtype):
    """One remap of the 1024^2 swirl with Z2: 800 sampled targets against the oracle's element
    search and six-point interpolation."""
    n = 1024
    wl = inputs.workload_swirl(n)
    wl.max_order = 2
    og = orc.OracleGrid(dim=2, n=(n, n), nfields=3, velocity="swirl2d", velocity_params=[5.0], max_order=2)
    t = 1.3
    D = orc.advect(og, t, wl.dt)
    h = wl.fields
    fl = orc.flags(og, h)
    sd, td = (sl.SL_F64, torch.float64) if dtype == "f64" else (sl.SL_F32, torch.float32)
    g = sl.grid_for(wl, sd)
    hin = torch.tensor(h, dtype=td, device=DEV)
    hout = torch.empty_like(hin)
    if dtype == "f64":
        g.set_displacement(torch.tensor(D, dtype=td, device=DEV))
    else:
        g.advect(t, wl.dt)
    g.remap(hin, hout)
    torch.cuda.synchronize()
    got = hout.double().cpu().numpy()
    rng = np.random.default_rng(12)
    worst = 0.0
    for (jy, jx) in rng.integers(0, n, size=(800, 2)):
        c, xi, st, _, _ = orc.locate(og, D, (int(jx), int(jy)))
        assert st == orc.OK
        for q in range(3):
            v = orc.interp(og, h[q], c, xi, orc.order(og, fl, c, q))
            if q != 1:
                worst = max(worst, abs(got[q, jy, jx] - v))
            if dtype == "f64" and not np.any(np.minimum(np.abs(xi), np.abs(1 - xi)) < TIE):
                assert abs(got[q, jy, jx] - v) <= 1e-12 * max(1.0, abs(v))
    if dtype == "f32":
        assert worst <= 5e-5, worst


def _shear_displacement(n, a):
    x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    D = np.zeros((n, n, 2))
    D[..., 0] = a * n / (2 * np.pi) * np.sin(2 * np.pi * y / n)
    D[..., 1] = a * n / (2 * np.pi) * np.sin(2 * np.pi * x / n)
    return D


@pytest.mark.parametrize("case", ["swirl", "smooth_ragged", "shear_fallback", "limiter_off", "five_fields",
                                  "one_field"])
def test_tiled_matches_generic_f32(sl, orc, case):
    """The quintic tiled FP32 kernel (staged window, 6x6 and 4x4 flag boxes, 6x6 taps) computes what
    the plain FP32 kernel computes: the same elements and orders away from faces, values up to the
    weight polynomials' and the summation order's rounding; tiles whose window does not fit run on
    global memory (shear case)."""
    rng = np.random.default_rng(31)
    thr = 0.25
    if case == "swirl":
        n = (256, 256)
        og = orc.OracleGrid(dim=2, n=n, nfields=3, velocity="swirl2d", velocity_params=[5.0])
        D, h = orc.advect(og, 0.9, 5 / 256), inputs.swirl_fields(256)
    elif case == "smooth_ragged":
        n = (75, 53)
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=3, shift=(2.3, -1.7))
        h = np.stack([rng.standard_normal((53, 75)).cumsum(axis=1) * 0.1, (rng.uniform(size=(53, 75)) > 0.5) * 1.0])
    elif case == "shear_fallback":
        n = (256, 256)
        D = _shear_displacement(256, 0.9)
        h = inputs.swirl_fields(256)[:2]
    elif case == "limiter_off":
        n, thr = (64, 96), -1.0
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=4, shift=(0.4, 4.2))
        h = rng.standard_normal((4, 96, 64))
    elif case == "five_fields":
        n = (96, 70)
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=12, shift=(2.2, 1.3))
        h = np.stack([rng.standard_normal((70, 96)).cumsum(axis=1) * 0.1 for _ in range(5)])
        h[0] += (np.arange(96)[None, :] > 48) * 1.0
    else:
        n = (40, 40)
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=7, shift=(-1.2, 3.4))
        h = rng.standard_normal((1, 40, 40)).cumsum(axis=2) * 0.1
    nf = h.shape[0]
    outs, diags = {}, {}
    for kname, kern in (("generic", sl.SL_KERNEL_GENERIC), ("tiled", sl.SL_KERNEL_TILED)):
        g = sl.Grid(2, n, nf, sl.SL_F32, max_order=2, limiter_threshold=thr, walk_start=sl.SL_START_BACKWARD,
                    kernel=kern)
        hin = torch.tensor(h, dtype=torch.float32, device=DEV)
        hout = torch.empty_like(hin)
        g.set_displacement(torch.tensor(D, dtype=torch.float32, device=DEV))
        g.remap(hin, hout)
        torch.cuda.synchronize()
        outs[kname] = hout.double().cpu().numpy()
        diags[kname] = g.diagnostics()
    scale = max(1.0, float(np.abs(h).max()))
    diff = np.abs(outs["tiled"] - outs["generic"])
    dg, dt = diags["generic"], diags["tiled"]
    ntar = n[0] * n[1]
    # after the displacement copy: tiled one launch; plain flags + remap
    assert dt["kernel_launches"] == 1 + 1 and dg["kernel_launches"] == 1 + 2
    assert float((diff > 4e-6 * scale).mean()) <= 1e-4, float(diff.max())
    assert dt["targets"] == dg["targets"] == ntar
    assert max(abs(a - b) for a, b in zip(dt["order_hist"], dg["order_hist"])) <= max(2, 1e-4 * ntar)
    if case == "swirl":  # smooth Gaussian and sine, a step: all three orders occur
        assert min(dt["order_hist"]) > 0
    if case == "shear_fallback":
        assert dt["tiles_fallback"] > 0
    else:
        tiles = -(-n[0] // 32) * -(-n[1] // 32)
        assert dt["tiles_fallback"] <= 0.1 * tiles


def test_fused_tiled_step_matches_plain_f32(sl):
    """sl_step with Z2 on the tiled path: one launch per step (the next step's trajectories inside
    the remap launch), the plain FP32 path's values step by step."""
    wl = inputs.workload_swirl(192, steps=4)
    wl.max_order = 2
    gt = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_AUTO)
    gg = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_GENERIC)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    t = 0.25
    for _ in range(3):
        ft, fg = f.clone(), f.clone()
        gt.step(ft, torch.empty_like(ft), t, wl.dt, 2)
        gg.step(fg, torch.empty_like(fg), t, wl.dt, 2)
        torch.cuda.synchronize()
        d = (ft - fg).abs()
        assert float((d > 4e-6).float().mean()) <= 1e-4, float(d.max())
        f, t = fg, t + 2 * wl.dt
    l0 = gt.diagnostics()["kernel_launches"]
    gt.step(f, torch.empty_like(f), 0.0, wl.dt, 6)
    assert gt.diagnostics()["kernel_launches"] - l0 == 1 + 6


@pytest.mark.parametrize("n", [(4, 4), (6, 5), (1 << 20, 4)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_extreme_sides(sl, orc, n, dtype):
    """Sides down to 4 (the six-point stencil wraps more than once round the period) and 2^20:
    FP64 within 1e-12 of the oracle, FP32 (tiled, global path for windows wider than the grid)
    to FP32 accuracy, limiter on for FP64 and off for FP32."""
    n0, n1 = n
    D = inputs.smooth_displacement(n, amplitude=0.3, seed=17, shift=(1.3, -0.6))
    rng = np.random.default_rng(18)
    x = np.arange(n0) / n0
    h = np.stack([np.tile(np.sin(2 * np.pi * x) + 0.3 * np.cos(6 * np.pi * x), (n1, 1)),
                  (rng.uniform(size=(n1, n0)) > 0.6) * 1.0])
    thr = 0.25 if dtype == "f64" else -1.0
    og = orc.OracleGrid(dim=2, n=n, nfields=2, max_order=2, threshold=thr, start=orc.START_BACKWARD)
    fl = orc.flags(og, h)
    sd, td = (sl.SL_F64, torch.float64) if dtype == "f64" else (sl.SL_F32, torch.float32)
    g = sl.Grid(2, n, 2, sd, max_order=2, limiter_threshold=thr, walk_start=sl.SL_START_BACKWARD)
    g.set_displacement(torch.tensor(D, dtype=td, device=DEV))
    hin = torch.tensor(h, dtype=td, device=DEV)
    hout = torch.empty_like(hin)
    g.remap(hin, hout)
    torch.cuda.synchronize()
    got = hout.double().cpu().numpy()
    assert sum(g.diagnostics()[k] for k in ("fail_locate", "fail_newton", "fail_fold")) == 0
    rng2 = np.random.default_rng(19)
    idx = [(a, b) for a in range(n0) for b in range(n1)] if n0 * n1 <= 64 else \
        list(zip(rng2.integers(0, n0, 300), rng2.integers(0, n1, 300)))
    for (jx, jy) in idx:
        c, xi, st, _, _ = orc.locate(og, D, (int(jx), int(jy)))
        assert st == orc.OK
        for q in range(2):
            v = orc.interp(og, h[q], c, xi, orc.order(og, fl, c, q))
            if dtype == "f64":
                if not np.any(np.minimum(np.abs(xi), np.abs(1 - xi)) < TIE):
                    assert abs(got[q, jy, jx] - v) <= 1e-12 * max(1.0, abs(v)), (jx, jy, q)
            else:
                assert abs(got[q, jy, jx] - v) <= 2e-5 * max(1.0, abs(v)), (jx, jy, q, got[q, jy, jx], v)
