"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 bar (per the method's parity contract): bit-exact jump flags, element indices and orders;
field values within 1e-12 of the oracle's, normwise (max |a - b| <= 1e-12 * max |b|).  Where the
located element is not unique -- the target lies within 1e-9 of a shared face -- the GPU's element
must still contain the target and its value must equal the oracle's interpolation in that element.
FP32 paths are compared with the FP64 oracle against the accuracy they promise.
"""
import math

import numpy as np
import pytest
import torch

from paper_1410_2817_gb300 import inputs
from tests import tiecheck

pytestmark = pytest.mark.gpu

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


DEV = "cuda"


def _og(orc, dim, n, nfields, velocity="uniform", params=(0.0, 0.0, 0.0), max_order=1, threshold=0.25,
        start="paper", lo=None, hi=None):
    kw = {}
    if lo is not None:
        kw["lo"], kw["hi"] = lo, hi
    return orc.OracleGrid(dim=dim, n=n, nfields=nfields, velocity=velocity, velocity_params=list(params),
                          max_order=max_order, threshold=threshold,
                          start=orc.START_PAPER if start == "paper" else orc.START_BACKWARD, **kw)


def _gpu_grid(sl, dim, n, nfields, dtype, velocity="uniform", params=(0.0, 0.0, 0.0), max_order=1,
              threshold=0.25, start="paper", **kw):
    return sl.Grid(dim, n, nfields, dtype, velocity=velocity, velocity_params=list(params), max_order=max_order,
                   limiter_threshold=threshold,
                   walk_start=sl.SL_START_PAPER if start == "paper" else sl.SL_START_BACKWARD, **kw)


def _check_remap(orc, og, D, h, ref, got, cell, xi, order, status, tol=1e-12):
    """Compare one remap: returns the number of tie targets handled by the element rule."""
    st_ref = ref.status
    assert np.array_equal(status, st_ref), f"status differs at {np.argwhere(status != st_ref)[:5].tolist()}"
    ok = st_ref == orc.OK
    rx = ref.xi
    tie = ok & np.any((np.abs(rx) < TIE) | (np.abs(rx - 1.0) < TIE), axis=-1)
    strict = ok & ~tie
    bad_cell = strict & (cell != ref.cell)
    assert not bad_cell.any(), f"element differs at {np.argwhere(bad_cell)[:5].tolist()}"
    for f in range(og.nfields):
        assert np.array_equal(order[f][strict], ref.order[f][strict]), f"order differs (field {f})"
        assert np.array_equal(order[f][~ok], ref.order[f][~ok])
    scale = max(1e-300, float(np.abs(ref.h).max()))
    err = np.abs(got - ref.h)
    err_strict = err[:, strict] if strict.any() else np.zeros(1)
    assert float(err_strict.max()) <= tol * scale, f"max err {float(err_strict.max())} at scale {scale}"
    assert np.array_equal(got[:, ~ok], ref.h[:, ~ok])  # failed targets keep their values exactly
    # ties: the GPU's element must contain the target and give the oracle's value in that element
    n = og.n[: og.dim]
    for idx in np.argwhere(tie):
        jj = tuple(idx)
        j = tuple(int(v) for v in reversed(jj))
        cw = int(cell[jj])
        c = []
        rem = cw
        for a in range(og.dim):
            c.append(rem % n[a])
            rem //= n[a]
        c = [ci + n[a] * round((j[a] - ci) / n[a]) for a, ci in enumerate(c)]
        vals, xe, oe, st = orc.eval_in_element(og, D, orc.flags(og, h), h, j, c)
        assert np.all(xe >= -TIE) and np.all(xe <= 1 + TIE), (j, c, xe)
        assert np.max(np.abs(got[(slice(None),) + jj] - vals)) <= tol * scale
    return int(tie.sum())


def _run_remap(sl, orc, dim, n, nfields, D, h, dtype=None, start="paper", max_order=1, threshold=0.25, tol=1e-12):
    dtype = dtype if dtype is not None else sl.SL_F64
    og = _og(orc, dim, n, nfields, max_order=max_order, threshold=threshold, start=start)
    ref = orc.remap(og, D, orc.flags(og, h), h)
    g = _gpu_grid(sl, dim, n, nfields, dtype, max_order=max_order, threshold=threshold, start=start)
    td = torch.float64 if dtype == sl.SL_F64 else torch.float32
    hin = torch.tensor(h.reshape((nfields,) + og.shape), dtype=td, device=DEV)
    hout = torch.empty_like(hin)
    g.set_displacement(torch.tensor(D, dtype=td, device=DEV))
    cell, xi, order, status = g.remap_debug(hin, hout)
    torch.cuda.synchronize()
    got = hout.double().cpu().numpy()
    return og, ref, got, cell.cpu().numpy(), xi.cpu().numpy(), order.cpu().numpy(), status.cpu().numpy(), g


# ------------------------------------------------------------------------------------------------
# jump flags: bit-exact
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["sbr64", "swirl_ragged", "random_jumps", "deform3d_ragged", "disabled"])
def test_flags_bit_exact(sl, orc, case):
    rng = np.random.default_rng(3)
    thr = 0.25
    if case == "sbr64":
        dim, n, h = 2, (64, 64), inputs.workload_sbr64().fields
    elif case == "swirl_ragged":
        dim, n = 2, (97, 70)
        h = np.stack([inputs.swirl_fields(128)[f][:70, :97] for f in range(3)])
    elif case == "random_jumps":
        dim, n = 2, (33, 17)
        h = np.stack([np.round(rng.uniform(0, 3, (17, 33))) * 0.5 + 1e-3 * rng.standard_normal((17, 33))
                      for _ in range(8)])
    elif case == "deform3d_ragged":
        dim, n = 3, (13, 10, 9)
        h = np.stack([rng.standard_normal((9, 10, 13)), (rng.uniform(size=(9, 10, 13)) > 0.6).astype(float)])
    else:
        dim, n, h, thr = 2, (16, 16), rng.standard_normal((2, 16, 16)), -1.0
    nf = h.shape[0]
    og = _og(orc, dim, n, nf, threshold=thr)
    ref = orc.flags(og, h)
    g = _gpu_grid(sl, dim, n, nf, sl.SL_F64, threshold=thr)
    got = g.flags(torch.tensor(h, device=DEV)).cpu().numpy()
    assert np.array_equal(got, ref)
    if thr < 0:
        assert not got.any()


# ------------------------------------------------------------------------------------------------
# trajectories: FP64 within 1e-12 (CUDA sincospi vs the oracle's reduced sin/cos differ in ulps)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,dim,n,params,t,dt", [
    ("uniform", 2, (20, 12), [0.3, -0.7], 0.0, 0.1),
    ("solid_body", 2, (64, 64), [2 * math.pi, 0.5, 0.5], 0.0, 1 / 64),
    ("swirl2d", 2, (128, 96), [5.0], 0.37, 5 / 128),
    ("deform3d", 3, (16, 12, 10), [3.0], 0.8, 0.03),
    ("fourier2d", 2, (48, 48), inputs.fourier2d_params(np.random.default_rng(1)), 0.0, 0.002),
    ("fourier3d", 3, (12, 12, 12), inputs.fourier3d_params(np.random.default_rng(2)), 0.0, 0.001),
])
def test_advect_parity_f64(sl, orc, kind, dim, n, params, t, dt):
    og = _og(orc, dim, n, 1, velocity=kind, params=params)
    ref = orc.advect(og, t, dt)
    g = _gpu_grid(sl, dim, n, 1, sl.SL_F64, velocity=kind, params=params)
    g.advect(t, dt)
    got = g.get_displacement().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, float(np.abs(ref).max()))


@pytest.mark.parametrize("kind,dim,n,params,t,dt", [
    ("swirl2d", 2, (128, 96), [5.0], 0.37, 5 / 128),
    ("deform3d", 3, (16, 12, 10), [3.0], 0.8, 0.03),
    ("fourier2d", 2, (48, 48), inputs.fourier2d_params(np.random.default_rng(1)), 0.0, 0.002),
    ("fourier3d", 3, (12, 12, 12), inputs.fourier3d_params(np.random.default_rng(2)), 0.0, 0.001),
])
def test_advect_f32_trig_accuracy(sl, orc, kind, dim, n, params, t, dt):
    """FP32 trajectories use the library's own sin(pi x) / cos(pi x) (exact argument reduction,
    Taylor polynomials, ~1e-7 absolute): against the FP64 oracle every displacement stays within
    FP32 accuracy -- 2e-6 of the largest for arguments in [0, 1] (swirl, deformation); 1e-5 for the
    Fourier flows, whose mode arguments 2 k.x reach ~16 and carry their own FP32 rounding (a few
    ulp of 16, amplified by 2 pi |k| in the velocity) -- and the stagnation nodes of the
    swirl/deformation flows do not move."""
    og = _og(orc, dim, n, 1, velocity=kind, params=params)
    ref = orc.advect(og, t, dt)
    g = _gpu_grid(sl, dim, n, 1, sl.SL_F32, velocity=kind, params=params)
    g.advect(t, dt)
    got = g.get_displacement().double().cpu().numpy()[..., :dim]
    tol = 1e-5 if kind.startswith("fourier") else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * float(np.abs(ref).max())
    if kind in ("swirl2d", "deform3d"):
        assert np.all(got[ref == 0.0] == 0.0)


def test_advect_f32_accuracy(sl, orc):
    og = _og(orc, 2, (256, 256), 1, velocity="swirl2d", params=[5.0])
    ref = orc.advect(og, 0.3, 5 / 256)
    g = _gpu_grid(sl, 2, (256, 256), 1, sl.SL_F32, velocity="swirl2d", params=[5.0])
    g.advect(0.3, 5 / 256)
    got = g.get_displacement().double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 2e-6 * float(np.abs(ref).max())


# ------------------------------------------------------------------------------------------------
# remap, stage-isolated: the GPU gets the oracle's displacement
# ------------------------------------------------------------------------------------------------
REMAP_CASES = {
    "sbr64_one_step": dict(dim=2, n=(64, 64)),
    "swirl128": dict(dim=2, n=(128, 128)),
    "ragged_smooth_z1": dict(dim=2, n=(70, 45)),
    "ragged_smooth_z0": dict(dim=2, n=(37, 29), max_order=0),
    "ragged_smooth_z2": dict(dim=2, n=(41, 38), max_order=2),
    "eight_fields": dict(dim=2, n=(24, 20)),
    "minimum_grid": dict(dim=2, n=(4, 4)),
    "deform3d_16": dict(dim=3, n=(16, 16, 16)),
    "ragged3d_z2": dict(dim=3, n=(11, 9, 13), max_order=2),
}


def _remap_inputs(orc, case, dim, n):
    rng = np.random.default_rng(abs(hash(case)) % 1000)
    if case == "sbr64_one_step":
        wl = inputs.workload_sbr64()
        og = _og(orc, 2, n, 1, velocity=wl.velocity, params=wl.velocity_params)
        return orc.advect(og, 0.0, wl.dt), wl.fields
    if case == "swirl128":
        og = _og(orc, 2, n, 3, velocity="swirl2d", params=[5.0])
        return orc.advect(og, 0.6, 5 / 128), inputs.swirl_fields(128)
    if case == "deform3d_16":
        og = _og(orc, 3, n, 2, velocity="deform3d", params=[3.0])
        return orc.advect(og, 0.4, 0.03), inputs.deform3d_fields(16)
    shape = tuple(reversed(n))
    D = inputs.smooth_displacement(n, amplitude=0.3, seed=5, shift=tuple(rng.uniform(-2.5, 2.5, dim)))
    nf = 8 if case == "eight_fields" else 2
    h = []
    for f in range(nf):
        if f % 2 == 0:
            h.append(rng.standard_normal(shape).cumsum(axis=-1) * 0.1)
        else:
            h.append((rng.uniform(size=shape) > 0.7).astype(float))
    return D, np.stack(h)


@pytest.mark.parametrize("start", ["paper", "backward"])
@pytest.mark.parametrize("case", sorted(REMAP_CASES))
def test_remap_parity_f64(sl, orc, case, start):
    cfg = REMAP_CASES[case]
    dim, n = cfg["dim"], cfg["n"]
    D, h = _remap_inputs(orc, case, dim, n)
    og, ref, got, cell, xi, order, status, _ = _run_remap(sl, orc, dim, n, h.shape[0], D, h, start=start,
                                                          max_order=cfg.get("max_order", 1))
    _check_remap(orc, og, D, h, ref, got, cell, xi, order, status)


def test_remap_parity_limiter_off_and_failures(sl, orc):
    n = (16, 16)
    D = np.zeros((16, 16, 2))
    D[8, 8] = (-1.6, -1.7)
    h = np.random.default_rng(9).standard_normal((1, 16, 16))
    og, ref, got, cell, xi, order, status, g = _run_remap(sl, orc, 2, n, 1, D, h, threshold=-1.0)
    assert (ref.status != orc.OK).any()
    _check_remap(orc, og, D, h, ref, got, cell, xi, order, status)
    diag = g.diagnostics()
    assert diag["fail_fold"] == int((ref.status == orc.FOLD).sum())
    assert diag["targets"] == 256


# ------------------------------------------------------------------------------------------------
# whole steps: sl_step against the oracle's step
# ------------------------------------------------------------------------------------------------
def _step_compare(sl, orc, wl, nsteps, dtype, tol, kernel=None, newton_mode=None):
    og = _og(orc, wl.dim, wl.n, wl.nfields, velocity=wl.velocity, params=wl.velocity_params,
             max_order=wl.max_order, threshold=wl.threshold)
    ref, nfail = orc.step(og, wl.fields, wl.t0, wl.dt, nsteps)
    kw = {}
    if kernel is not None:
        kw["kernel"] = kernel
    if newton_mode is not None:
        kw["newton_mode"] = newton_mode
    g = sl.grid_for(wl, dtype, **kw)
    td = torch.float64 if dtype == sl.SL_F64 else torch.float32
    f = torch.tensor(wl.fields, dtype=td, device=DEV)
    s = torch.empty_like(f)
    g.step(f, s, wl.t0, wl.dt, nsteps)
    torch.cuda.synchronize()
    got = f.double().cpu().numpy()
    return ref, got, g


@pytest.mark.parametrize("name,nsteps", [("sbr64", 16), ("swirl128", 8), ("deform3d16", 4)])
def test_step_parity_f64(sl, orc, name, nsteps):
    """Whole FP64 steps, each from the GPU's previous result on both sides: every target within
    1e-12 of the oracle (normwise) unless it is a face tie (tiecheck.f64_step_ties: the GPU's own
    element contains it and gives the oracle's interpolation there); the same run as one sl_step
    call reproduces the chained steps bit for bit."""
    if name == "sbr64":
        wl = inputs.workload_sbr64()
    elif name == "swirl128":
        wl = inputs.workload_swirl(128, steps=nsteps)
    else:
        wl = inputs.workload_deform3d(16, steps=nsteps)
    og = _og(orc, wl.dim, wl.n, wl.nfields, velocity=wl.velocity, params=wl.velocity_params,
             max_order=wl.max_order, threshold=wl.threshold)
    g = sl.grid_for(wl, sl.SL_F64, walk_start=sl.SL_START_PAPER)
    _, beyond, ties = tiecheck.f64_run_ties(orc, og, g, wl.fields, wl.t0, wl.dt, nsteps)
    assert beyond == ties


# ------------------------------------------------------------------------------------------------
# moments: FP64 accumulation, Table 1
# ------------------------------------------------------------------------------------------------
def test_moments_parity_and_table1(sl, orc):
    n, lo, hi, h = inputs.table1_grid()
    og = _og(orc, 2, n, 1, lo=lo, hi=hi)
    ref = orc.moments(og, h, 4)
    g = sl.Grid(2, n, 1, sl.SL_F64, lo=lo, hi=hi)
    got = g.moments(torch.tensor(h, device=DEV), 4)
    for a, b in zip(got, ref):
        assert abs(a - b) <= 1e-13 * max(1.0, abs(b))
    printed = [23.3536, -11.6768, 6.0558, -3.0820, 1.6249]
    for a, p in zip(got, printed):
        assert math.trunc(a * 1e4) / 1e4 == pytest.approx(p, abs=1e-12)
    h3 = np.random.default_rng(4).standard_normal((9, 7, 11))
    og3 = _og(orc, 3, (11, 7, 9), 1, lo=(0, -1, 2), hi=(1, 3, 4))
    g3 = sl.Grid(3, (11, 7, 9), 1, sl.SL_F64, lo=(0, -1, 2), hi=(1, 3, 4))
    got3 = g3.moments(torch.tensor(h3, device=DEV), 7)
    ref3 = orc.moments(og3, h3, 7)
    for a, b in zip(got3, ref3):
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b))


# ------------------------------------------------------------------------------------------------
# failure reporting and argument errors through the ABI
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cycling_walks_stop_early(sl, orc, dtype):
    """Sec. 2.2: a walk that returns to an element it has tried gives up at once (the next element
    depends on the current one alone).  On the 64x64 solid-body rotation the seam's failing
    targets are exactly the oracle's, and all the walks of a target together -- FP32 and its FP64
    re-solve -- take fewer hops than one walk run to the 64-hop limit."""
    wl = inputs.workload_sbr64()
    og = _og(orc, 2, wl.n, 1, velocity=wl.velocity, params=wl.velocity_params)
    D = orc.advect(og, 0.0, wl.dt)
    ref = orc.remap(og, D, orc.flags(og, wl.fields), wl.fields)
    nfail = int((ref.status != orc.OK).sum())
    assert nfail > 0
    sd, td = (sl.SL_F64, torch.float64) if dtype == "f64" else (sl.SL_F32, torch.float32)
    g = sl.grid_for(wl, sd)
    f = torch.tensor(wl.fields, dtype=td, device=DEV)
    g.set_displacement(torch.tensor(D, dtype=td, device=DEV))
    g.remap(f, torch.empty_like(f))
    d = g.diagnostics()
    assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == nfail
    # hops_max adds up every walk a target made (FP32 in the window, FP32 from global memory, the
    # FP64 re-solve); before the revisit rule one exhausted walk alone took 64
    assert d["hops_max"] < 64, d


def test_fail_error_policy_reports(sl, orc):
    wl = inputs.workload_sbr64()
    g = sl.grid_for(wl, sl.SL_F64, fail_policy=sl.SL_FAIL_ERROR)
    f = torch.tensor(wl.fields, device=DEV)
    s = torch.empty_like(f)
    with pytest.raises(sl.SLError) as ei:
        g.step(f, s, 0.0, wl.dt, 1)
    assert ei.value.status in (sl.SL_ERR_LOCATE, sl.SL_ERR_NEWTON, sl.SL_ERR_FOLD)
    d = g.diagnostics()
    assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] > 0


def test_argument_errors(sl):
    g = sl.Grid(2, (16, 16), 2, sl.SL_F64)
    f = torch.zeros((2, 16, 16), dtype=torch.float64, device=DEV)
    with pytest.raises(sl.SLError) as ei:
        g.remap(f, f)
    assert ei.value.status == sl.SL_ERR_ARG
    s = torch.zeros_like(f)
    with pytest.raises(sl.SLError):
        g.step(f, s, 0.0, 0.1, -1)
    with pytest.raises(sl.SLError):
        g.moments(f[0], 8)
    g.step(f, s, 0.0, 0.1, 0)  # zero steps is a no-op


# ------------------------------------------------------------------------------------------------
# FP32 production path against the FP64 oracle
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("newton_mode", ["mixed", "f64"])
@pytest.mark.parametrize("kernel", ["auto", "generic"])
def test_fp32_step_accuracy(sl, orc, newton_mode, kernel):
    wl = inputs.workload_swirl(256, steps=10)
    ref, got, g = _step_compare(sl, orc, wl, 10, sl.SL_F32, None,
                                kernel=sl.SL_KERNEL_AUTO if kernel == "auto" else sl.SL_KERNEL_GENERIC,
                                newton_mode=sl.SL_NEWTON_MIXED if newton_mode == "mixed" else sl.SL_NEWTON_F64)
    for f, name in ((0, "gaussian"), (2, "sine")):
        l1 = np.abs(got[f] - ref[f]).sum() / np.abs(ref[f]).sum()
        assert l1 <= 1e-5, (name, l1)
    # moments of the smooth fields, relative to the field's L1 mass (the sine's m0 is ~0)
    og = _og(orc, 2, wl.n, 1)
    for f in (0, 2):
        mr = orc.moments(og, ref[f], 2)
        mg = orc.moments(og, got[f], 2)
        l1 = float(np.abs(ref[f]).sum())
        for p in range(3):
            assert abs(mg[p] - mr[p]) <= 1e-6 * l1, (f, p, mg[p], mr[p])


# ------------------------------------------------------------------------------------------------
# full size (the benchmark's 1024^2 swirl configuration): sampled targets against the oracle
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_sampled(sl, orc, dtype):
    n = 1024
    wl = inputs.workload_swirl(n)
    og = _og(orc, 2, (n, n), 3, velocity="swirl2d", params=[5.0])
    t = 1.3
    D = orc.advect(og, t, wl.dt)
    h = wl.fields
    fl = orc.flags(og, h)
    sd = sl.SL_F64 if dtype == "f64" else sl.SL_F32
    td = torch.float64 if dtype == "f64" else torch.float32
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
    rng = np.random.default_rng(11)
    samples = rng.integers(0, n, size=(1500, 2))
    worst = 0.0
    for (jy, jx) in samples:
        c, xi, st, _, _ = orc.locate(og, D, (jx, jy))
        assert st == orc.OK
        for f in range(3):
            m = orc.order(og, fl, c, f)
            v = orc.interp(og, h[f], c, xi, m)
            worst = max(worst, abs(got[f, jy, jx] - v) if f != 1 else 0.0)
            if dtype == "f64":
                near_face = np.any(np.minimum(np.abs(xi), np.abs(1 - xi)) < TIE)
                if not near_face:
                    assert abs(got[f, jy, jx] - v) <= 1e-12 * max(1.0, abs(v))
    if dtype == "f32":
        # own FP32 trajectories and FP32 limiter decisions: a marginal flag may switch cubic and
        # linear interpolation at a smooth extremum (difference ~ h'' dx^2 / 8)
        assert worst <= 5e-5, worst


# ------------------------------------------------------------------------------------------------
# the shared-memory tiled FP32 kernel computes what the plain FP32 kernel computes
# ------------------------------------------------------------------------------------------------
def _shear_displacement(n, a):
    """Periodic, non-folding displacement with a strong shear (|grad D| up to a < 1): windows of
    some tiles exceed the shared-memory capacity and take the global-gather fallback."""
    x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    D = np.zeros((n, n, 2))
    D[..., 0] = a * n / (2 * np.pi) * np.sin(2 * np.pi * y / n)
    D[..., 1] = a * n / (2 * np.pi) * np.sin(2 * np.pi * x / n)
    return D


@pytest.mark.parametrize("tile_config", [1, 5, 6, 7])
@pytest.mark.parametrize("case", ["swirl", "smooth_ragged", "shear_fallback", "limiter_off", "order0", "many_tiles",
                                  "tma_ragged", "one_field"])
def test_tiled_and_generic_f32_per_target(sl, orc, case, tile_config):
    """The FP32 remap kernels (shared-memory tiled and plain), target by target against the FP64
    oracle on the same FP32 displacement and fields: each value within 2e-6 of the oracle's
    interpolation in the oracle's element and order, or -- for a target within FP32 rounding of a
    face or of a limiter threshold -- in the neighbouring element or with the other order."""
    rng = np.random.default_rng(21)
    max_order, thr = 1, 0.25
    if case == "many_tiles":
        # more 32x32 tiles (21 x 17, ragged) than one per SM: the pipelined kernel stages the next
        # tiles of each CTA while it computes the current one
        n = (650, 530)
        D = inputs.smooth_displacement(n, amplitude=0.4, seed=6, shift=(3.1, -2.6))
        h = np.stack([inputs.swirl_fields(650)[0][:530, :650], (rng.uniform(size=(530, 650)) > 0.7) * 1.0,
                      rng.standard_normal((530, 650)).cumsum(axis=0) * 0.05])
    elif case == "swirl":
        n = (256, 256)
        og = _og(orc, 2, n, 3, velocity="swirl2d", params=[5.0])
        D, h = orc.advect(og, 0.9, 5 / 256), inputs.swirl_fields(256)
    elif case == "smooth_ragged":
        n = (75, 53)
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=3, shift=(2.3, -1.7))
        h = np.stack([rng.standard_normal((53, 75)).cumsum(axis=1) * 0.1, (rng.uniform(size=(53, 75)) > 0.5) * 1.0])
    elif case == "shear_fallback":
        n = (256, 256)
        D = _shear_displacement(256, 0.9)
        h = inputs.swirl_fields(256)[:2]
    elif case == "tma_ragged":
        # rows a multiple of 4 values (box copies) but tiles ragged on both axes; 3 fields
        n = (516, 260)
        D = inputs.smooth_displacement(n, amplitude=0.35, seed=7, shift=(-2.2, 1.4))
        h = np.stack([inputs.swirl_fields(516)[f][:260, :516] for f in range(3)])
    elif case == "one_field":
        n = (320, 192)
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=8, shift=(4.4, -3.1))
        h = (rng.uniform(size=(1, 192, 320)) > 0.6) * 1.0 + 0.1 * rng.standard_normal((1, 192, 320)).cumsum(axis=2)
    elif case == "limiter_off":
        n, thr = (64, 96), -1.0
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=4, shift=(0.4, 4.2))
        h = rng.standard_normal((4, 96, 64))
    else:
        n, max_order = (64, 64), 0
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=5, shift=(-3.4, 0.2))
        h = rng.standard_normal((2, 64, 64))
    nf = h.shape[0]
    # both kernels get the same FP32 displacement and fields; the oracle gets them too, exactly
    D32 = np.asarray(D, dtype=np.float32)
    h32 = np.asarray(h, dtype=np.float32)
    og = _og(orc, 2, n, nf, max_order=max_order, threshold=thr, start="backward")
    diags = {}
    for kname, kern in (("generic", sl.SL_KERNEL_GENERIC), ("tiled", sl.SL_KERNEL_TILED)):
        g = _gpu_grid(sl, 2, n, nf, sl.SL_F32, max_order=max_order, threshold=thr, start="backward", kernel=kern,
                      tile_config=tile_config)
        hin = torch.tensor(h32, device=DEV)
        hout = torch.empty_like(hin)
        g.set_displacement(torch.tensor(D32, device=DEV))
        g.remap(hin, hout)
        torch.cuda.synchronize()
        diags[kname] = g.diagnostics()
        # target by target against the FP64 oracle: the oracle's element and order, or a tie
        counts = tiecheck.f32_remap_targets(orc, og, D32, h32, hout.double().cpu().numpy(), 2e-6, thr=thr)
        ntar = n[0] * n[1]
        assert counts["limiter_ties"] + counts["face_ties"] <= max(8, 1e-3 * ntar), (kname, counts)
    dg, dt = diags["generic"], diags["tiled"]
    assert dt["targets"] == dg["targets"] == ntar
    assert dt["fail_locate"] + dt["fail_newton"] + dt["fail_fold"] == dg["fail_locate"] + dg["fail_newton"] + dg["fail_fold"]
    # the shear's windows exceed every tile's shared-memory capacity somewhere; the benchmark's
    # swirl never does.  (Larger displacements on the other cases may exceed the smaller windows of
    # the persistent configurations; their targets then take the general path, checked above.)
    if case == "shear_fallback":
        assert dt["tiles_fallback"] > 0
    elif case == "swirl" or tile_config in (1, 5):
        assert dt["tiles_fallback"] == 0


def test_fused_step_matches_split_steps_f32(sl):
    """sl_step on the tiled path integrates the trajectories of step k+1 inside the remap of step
    k.  Step by step (same inputs) it matches the plain FP32 path (flags -> advect -> remap) up to
    FP32 rounding, and the displacement it leaves equals sl_advect_nodes'."""
    wl = inputs.workload_swirl(192, steps=6)
    gt = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_AUTO)
    gg = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_GENERIC)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    t = 0.25
    worst = 0.0
    for k in range(4):
        ft, fg = f.clone(), f.clone()
        st_, sg_ = torch.empty_like(f), torch.empty_like(f)
        gt.step(ft, st_, t, wl.dt, 1)
        gg.step(fg, sg_, t, wl.dt, 1)
        torch.cuda.synchronize()
        worst = max(worst, float((ft - fg).abs().max()))
        f = fg
        t += wl.dt
    assert worst <= 2e-6, worst
    # two fused steps: the second remap used the D the first launch integrated for t0 + dt, and
    # the second launch leaves D for the step after the call (t0 + 2 dt)
    ft = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    gt.step(ft, torch.empty_like(ft), 0.25, wl.dt, 2)
    d_fused = gt.get_displacement()
    gg.advect(0.25 + wl.dt + wl.dt, wl.dt)
    d_plain = gg.get_displacement()
    # the fused launch integrates two nodes at a time on packed FP32x2 arithmetic, the trajectory
    # launch one at a time; every rounding of both is explicit, so the bits agree
    assert torch.equal(d_fused, d_plain)
    l0 = gt.diagnostics()["kernel_launches"]
    gt.step(ft, torch.empty_like(ft), 0.0, wl.dt, 6)
    assert gt.diagnostics()["kernel_launches"] - l0 == 1 + 6  # one advect, then one launch per step
    # a call that starts where the last one ended reuses the displacement it left ...
    l0 = gt.diagnostics()["kernel_launches"]
    f_chain = ft.clone()
    gt.step(f_chain, torch.empty_like(ft), 0.0 + 5 * wl.dt + wl.dt, wl.dt, 3)
    assert gt.diagnostics()["kernel_launches"] - l0 == 3 + 1  # three steps, one copy-back (odd count)
    # ... and gives what a fresh integration gives
    gf = sl.grid_for(wl, sl.SL_F32, kernel=sl.SL_KERNEL_AUTO)
    f_fresh = ft.clone()
    gf.step(f_fresh, torch.empty_like(ft), 0.0 + 5 * wl.dt + wl.dt, wl.dt, 3)
    torch.cuda.synchronize()
    # (the trajectory launch and the fused launch round the RK4 alike: the same bits)
    assert torch.equal(f_chain, f_fresh)
    # a displacement set by the caller is never taken for the carried one
    gt.set_displacement(torch.zeros_like(d_fused))
    l0 = gt.diagnostics()["kernel_launches"]
    gt.step(ft, torch.empty_like(ft), 0.0 + 8 * wl.dt + wl.dt, wl.dt, 1)
    assert gt.diagnostics()["kernel_launches"] - l0 == 2 + 1  # advect, one step, one copy-back


@pytest.mark.parametrize("dt", [0.002, 0.05, 0.5])
def test_fused_trajectories_equal_the_trajectory_launch(sl, dt):
    """The fused launch's trajectories (two nodes at a time on packed FP32x2 arithmetic) equal the
    trajectory launch's bit for bit, with stage offsets in every series range: dt = 0.002 keeps
    them below 1/256 of the box (short series), 0.05 mixes short and long series between the two
    nodes of a pair, 0.5 also takes the direct evaluation."""
    wl = inputs.workload_swirl(96, steps=4)
    wl.fields = wl.fields[:2]
    wl.nfields = 2
    n = (96, 64)
    gt = sl.Grid(2, n, 2, sl.SL_F32, velocity="swirl2d", velocity_params=[5.0], walk_start=sl.SL_START_BACKWARD)
    gg = sl.Grid(2, n, 2, sl.SL_F32, velocity="swirl2d", velocity_params=[5.0], walk_start=sl.SL_START_BACKWARD,
                 kernel=sl.SL_KERNEL_GENERIC)
    f = torch.tensor(np.asarray(wl.fields)[:, :64, :], dtype=torch.float32, device=DEV)
    gt.step(f, torch.empty_like(f), 0.7, dt, 1)  # leaves D(t + dt) from the fused launch
    gg.advect(0.7 + dt, dt)
    torch.cuda.synchronize()
    assert torch.equal(gt.get_displacement(), gg.get_displacement())


@pytest.mark.parametrize("dt", [0.003, 0.03, 0.3])
def test_fused_3d_trajectories_equal_the_trajectory_launch(sl, dt):
    """The blocked 3-D launch's next-step trajectories of the deformation flow equal the trajectory
    launch's bit for bit, for stage offsets in each series range."""
    n = (24, 20, 16)
    kw = dict(velocity="deform3d", velocity_params=[3.0], walk_start=sl.SL_START_BACKWARD)
    gt = sl.Grid(3, n, 2, sl.SL_F32, **kw)
    gg = sl.Grid(3, n, 2, sl.SL_F32, kernel=sl.SL_KERNEL_GENERIC, **kw)
    f = torch.tensor(np.asarray(inputs.deform3d_fields(24))[:, :16, :20, :24], dtype=torch.float32, device=DEV)
    gt.step(f, torch.empty_like(f), 0.4, dt, 1)
    gg.advect(0.4 + dt, dt)
    torch.cuda.synchronize()
    assert torch.equal(gt.get_displacement(), gg.get_displacement())


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_step_out_equals_step(sl, dtype):
    """sl_step_out (out of place) computes what sl_step computes in place, for odd and even step
    counts, and leaves its input untouched; one fused FP32 step is one launch with no copy back."""
    wl = inputs.workload_swirl(192, steps=3)
    sd, td = (sl.SL_F64, torch.float64) if dtype == "f64" else (sl.SL_F32, torch.float32)
    for nsteps in (1, 2, 3):
        g1, g2 = sl.grid_for(wl, sd), sl.grid_for(wl, sd)
        f = torch.tensor(wl.fields, dtype=td, device=DEV)
        fin = f.clone()
        g1.step(f, torch.empty_like(f), 0.3, wl.dt, nsteps)
        out = torch.empty_like(fin)
        g2.step_out(fin, out, 0.3, wl.dt, nsteps, scratch=torch.empty_like(fin) if nsteps > 1 else None)
        torch.cuda.synchronize()
        assert torch.equal(out, f), (nsteps, float((out - f).abs().max()))
        assert torch.equal(fin, torch.tensor(wl.fields, dtype=td, device=DEV))
    if dtype == "f32":
        l0 = g2.diagnostics()["kernel_launches"]
        g2.step_out(out, fin, 0.3 + 3 * wl.dt, wl.dt, 1)  # starts where the last call ended
        assert g2.diagnostics()["kernel_launches"] - l0 == 1


@pytest.mark.parametrize("case", ["deform3d_32", "ragged3d", "limiter_off3d"])
def test_blocked3d_matches_generic_f32(sl, orc, case):
    rng = np.random.default_rng(31)
    thr = 0.25
    if case == "deform3d_32":
        n = (32, 32, 32)
        og = _og(orc, 3, n, 2, velocity="deform3d", params=[3.0])
        D, h = orc.advect(og, 0.4, 0.03), inputs.deform3d_fields(32)
    elif case == "ragged3d":
        n = (19, 13, 11)
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=8, shift=(1.6, -2.2, 0.7))
        h = np.stack([rng.standard_normal((11, 13, 19)).cumsum(axis=2) * 0.1, (rng.uniform(size=(11, 13, 19)) > 0.5) * 1.0])
    else:
        n, thr = (16, 16, 16), -1.0
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=9, shift=(-0.6, 3.1, 0.2))
        h = rng.standard_normal((3, 16, 16, 16))
    nf = h.shape[0]
    outs, diags = {}, {}
    for kname, kern in (("generic", sl.SL_KERNEL_GENERIC), ("tiled", sl.SL_KERNEL_TILED)):
        g = _gpu_grid(sl, 3, n, nf, sl.SL_F32, threshold=thr, start="backward", kernel=kern)
        hin = torch.tensor(h, dtype=torch.float32, device=DEV)
        hout = torch.empty_like(hin)
        g.set_displacement(torch.tensor(D, dtype=torch.float32, device=DEV))
        g.remap(hin, hout)
        torch.cuda.synchronize()
        outs[kname] = hout.double().cpu().numpy()
        diags[kname] = g.diagnostics()
    diff = np.abs(outs["tiled"] - outs["generic"])
    assert float(diff.max()) <= 4e-6 * max(1.0, float(np.abs(h).max())), float(diff.max())
    assert diags["tiled"]["order_hist"] == diags["generic"]["order_hist"]
    assert diags["tiled"]["targets"] == int(np.prod(n))


@pytest.mark.parametrize("tile_config", [0, 1])
@pytest.mark.parametrize("newton_mode", ["mixed", "f64"])
@pytest.mark.parametrize("case", ["deform3d_32", "deform3d_64x48x40", "ragged3d"])
def test_blocked3d_f32_per_target(sl, orc, case, newton_mode, tile_config):
    """The 3-D FP32 remap, target by target against the FP64 oracle on the same FP32 displacement
    and fields: each value within 2e-6 of the oracle's interpolation in the oracle's element and
    order, or -- within FP32 rounding of a face or of a limiter threshold -- in the neighbouring
    element or with the other order.  Both inversions: FP32 with FP64 re-solves of failed or
    degenerate targets (mixed), and FP64 for every target (no re-solve is counted); both kernels:
    the staged one (tile configuration 0, plain remaps of up to 2 fields in FP32 inversion; the
    64x48x40 grid copies two thirds of its windows by TMA boxes and the rest element by element
    across the seam) and the blocked one (tile configuration 1)."""
    from tests import tiecheck
    rng = np.random.default_rng(33)
    if case == "deform3d_32":
        n = (32, 32, 32)
        og = _og(orc, 3, n, 2, velocity="deform3d", params=[3.0])
        D, h = orc.advect(og, 0.4, 0.03), inputs.deform3d_fields(32)
    elif case == "deform3d_64x48x40":
        n = (64, 48, 40)
        og = _og(orc, 3, n, 2, velocity="deform3d", params=[3.0])
        D = orc.advect(og, 0.7, 0.03)
        x, y, z = inputs.node_coords(n)
        h = np.stack([np.exp(-((x - 0.4) ** 2 + (y - 0.5) ** 2 + (z - 0.45) ** 2) / 0.02),
                      ((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2 <= 0.09).astype(np.float64)])
    else:
        n = (19, 13, 11)
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=8, shift=(1.6, -2.2, 0.7))
        h = np.stack([rng.standard_normal((11, 13, 19)).cumsum(axis=2) * 0.1, (rng.uniform(size=(11, 13, 19)) > 0.5) * 1.0,
                      rng.standard_normal((11, 13, 19))])
    D32, h32 = np.asarray(D, dtype=np.float32), np.asarray(h, dtype=np.float32)
    nf = h32.shape[0]
    nm = sl.SL_NEWTON_MIXED if newton_mode == "mixed" else sl.SL_NEWTON_F64
    g = _gpu_grid(sl, 3, n, nf, sl.SL_F32, start="backward", kernel=sl.SL_KERNEL_TILED, newton_mode=nm,
                  tile_config=tile_config)
    hin = torch.tensor(h32, device=DEV)
    hout = torch.empty_like(hin)
    g.set_displacement(torch.tensor(D32, device=DEV))
    g.remap(hin, hout)
    torch.cuda.synchronize()
    og = _og(orc, 3, n, nf, start="backward")
    counts = tiecheck.f32_remap_targets(orc, og, D32, h32, hout.double().cpu().numpy(), 2e-6)
    d = g.diagnostics()
    assert counts["oracle_failed"] == 0 and d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0
    assert d["targets"] == int(np.prod(n))
    if newton_mode == "f64":
        assert d["newton_f64"] == 0
    assert counts["face_ties"] + counts["limiter_ties"] <= 0.01 * d["targets"], counts


def test_fp32_3d_step_accuracy(sl, orc):
    wl = inputs.workload_deform3d(32, steps=4)
    ref, got, g = _step_compare(sl, orc, wl, 4, sl.SL_F32, None)
    l1 = np.abs(got[0] - ref[0]).sum() / np.abs(ref[0]).sum()
    assert l1 <= 1e-5, l1
    d = g.diagnostics()
    assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0


def test_full_size_3d_sampled_f32(sl, orc):
    """256^3 deformation flow (the 3-D benchmark size): the GPU's FP32 remap with the oracle's
    displacements against the oracle's own element search, order and tricubic sum at sampled targets."""
    n = 256
    wl = inputs.workload_deform3d(n, steps=1)
    og = _og(orc, 3, (n, n, n), 2, velocity="deform3d", params=[3.0])
    D = orc.advect(og, 0.6, wl.dt)
    h = wl.fields
    fl = orc.flags(og, h)
    g = sl.grid_for(wl, sl.SL_F32)
    hin = torch.tensor(h, dtype=torch.float32, device=DEV)
    hout = torch.empty_like(hin)
    g.set_displacement(torch.tensor(D, dtype=torch.float32, device=DEV))
    g.remap(hin, hout)
    torch.cuda.synchronize()
    rng = np.random.default_rng(12)
    samples = rng.integers(0, n, size=(300, 3))
    errs = []
    for (jz, jy, jx) in samples:
        c, xi, st, _, _ = orc.locate(og, D, (jx, jy, jz))
        assert st == orc.OK
        m = orc.order(og, fl, c, 0)
        v = orc.interp(og, h[0], c, xi, m)
        errs.append(abs(float(hout[0, jz, jy, jx]) - v))
    errs = np.array(errs)
    assert float(np.quantile(errs, 0.99)) <= 1e-5 and float(errs.max()) <= 5e-5, (errs.max(), np.quantile(errs, 0.99))
    d = g.diagnostics()
    assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0


def test_steady_velocity_integrates_once(sl, orc):
    """For a steady velocity the RK4 displacement over dt is the same every step: sl_step
    integrates it once and reuses it (also across calls with the same dt); the result equals the
    oracle's, which integrates every step."""
    wl = inputs.batched_grids(count=1, seed=2, steps=6, side_lo=96, side_hi=96)[0]
    g = sl.grid_for(wl, sl.SL_F32)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    s = torch.empty_like(f)
    g.step(f, s, 0.0, wl.dt, 3)
    l1 = g.diagnostics()["kernel_launches"]
    g.step(f, s, 3 * wl.dt, wl.dt, 3)
    # one integration, three steps and the copy-back of an odd step count; then no integration
    assert l1 == 1 + 3 + 1 and g.diagnostics()["kernel_launches"] == l1 + 3 + 1
    torch.cuda.synchronize()
    og = _og(orc, 2, wl.n, 2, velocity=wl.velocity, params=wl.velocity_params)
    ref, _ = orc.step(og, wl.fields, 0.0, wl.dt, 6)
    got = f.double().cpu().numpy()
    assert np.abs(got[0] - ref[0]).sum() / np.abs(ref[0]).sum() <= 1e-4
    g64 = sl.grid_for(wl, sl.SL_F64)
    f64 = torch.tensor(wl.fields, device=DEV)
    g64.step(f64, torch.empty_like(f64), 0.0, wl.dt, 6)
    torch.cuda.synchronize()
    assert g64.diagnostics()["kernel_launches"] == 1 + 2 * 6  # one advect, then flags + remap per step
    # FP64: every step within 1e-12 of the oracle's from the same fields but for face ties
    g64b = sl.grid_for(wl, sl.SL_F64, walk_start=sl.SL_START_PAPER)
    got64, beyond, ties = tiecheck.f64_run_ties(orc, og, g64b, wl.fields, 0.0, wl.dt, 6)
    assert beyond == ties
    assert np.array_equal(got64, f64.cpu().numpy())
