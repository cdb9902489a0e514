"""The shallow-water system (Sec. 3.3, eq. nlsw, nu = 0) on the CUDA path: FP64 steps against the
oracle within 1e-12 step by step (Kelvin wave, nonlinear simple wave, passive tracers; second- and
fourth-order differences); the FP32 tiled path against the FP32 plain path; FP32 accuracy against
the closed-form Kelvin wave at the oracle's level."""
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


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def _case(name):
    """(n, lo, hi, f0, max_order, fields, dt)"""
    if name.startswith("kelvin"):
        n = 64
        return (n, n), (0.0, -0.5), (1.0, 0.5), 250.0, 2 if name == "kelvin_z2" else 1, inputs.kelvin_fields(n), 0.5 / n
    if name == "simple_wave":
        n, amp = 64, 0.05
        x = np.arange(n) / n
        c0 = np.sqrt(1 + amp * np.sin(2 * np.pi * x))
        h0, u0 = np.tile(c0 ** 2 - 1, (8, 1)), np.tile(2 * (c0 - 1), (8, 1))
        return (n, 8), (0.0, 0.0), (1.0, 1.0), 0.0, 2, np.stack([h0, u0, np.zeros_like(h0)]), 0.5 / n
    # a nonlinear bump with rotation and two passive tracers (one with a jump for the limiter)
    n = (48, 40)
    x1, x2 = inputs.node_coords(n, (0.0, -0.5), (1.0, 0.5))
    h = 0.2 * np.exp(-((x1 - 0.5) ** 2 + x2 ** 2) / 0.02)
    tr = (x1 > 0.5).astype(float)
    return n, (0.0, -0.5), (1.0, 0.5), 20.0, 1, np.stack([h, np.zeros_like(h), np.zeros_like(h), tr, h + x1]), 0.5 / 48


@pytest.mark.parametrize("name,nu", [("kelvin_z2", 0.0), ("kelvin_z1", 0.0), ("simple_wave", 0.0),
                                     ("bump_tracers", 0.0), ("bump_tracers", 0.01), ("kelvin_z2", 0.002),
                                     ("simple_wave", 0.01)])
def test_step_parity_f64(sl, orc, name, nu):
    n, lo, hi, f0, mo, h, dt = _case(name)
    nf = h.shape[0]
    thr = 0.25 if name == "bump_tracers" else -1.0
    params = [f0] if nu == 0.0 else [f0, nu]
    og = orc.OracleGrid(dim=2, n=n, nfields=nf, lo=lo, hi=hi, velocity="nlsw", velocity_params=params, max_order=mo,
                        threshold=thr, start=orc.START_BACKWARD)
    g = sl.Grid(2, n, nf, sl.SL_F64, lo=lo, hi=hi, velocity="nlsw", velocity_params=params, max_order=mo,
                limiter_threshold=thr)
    stage_launches = 4 if nu == 0.0 else 7  # three RK3 stages in four launches, and a stress pass each
    F = np.asarray(h, dtype=np.float64)
    for k in range(4):
        ref, nfail = orc.step(og, F, 0.0, dt, 1)
        assert nfail == 0
        f = torch.tensor(F, dtype=torch.float64, device=DEV)
        l0 = g.diagnostics()["kernel_launches"]
        g.step(f, torch.empty_like(f), 0.0, dt, 1)
        torch.cuda.synchronize()
        assert g.diagnostics()["kernel_launches"] - l0 == stage_launches + 2  # and flags + remap
        got = f.cpu().numpy()
        # no allowance: every target of every field within 1e-12 of the oracle's (normwise)
        for q in range(nf):
            scale = max(float(np.abs(ref[q]).max()), 1e-300)
            err = np.abs(got[q] - ref[q])
            assert float(err.max()) <= 1e-12 * scale, (k, q, int((err > 1e-12 * scale).sum()), float(err.max()), scale)
        F = ref
    d = g.diagnostics()
    assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0


@pytest.mark.parametrize("amp,nu", [(1e-4, 0.0), (0.5, 0.0005)])
def test_kelvin_f32_tiled_matches_plain(sl, amp, nu):
    """The linear Kelvin wave, and the paper's nonlinear run (amplitude 0.5, nu = 0.0005)."""
    n = 128
    h = inputs.kelvin_fields(n, 0.0, amp)
    params = [250.0] if nu == 0.0 else [250.0, nu]
    out = {}
    for name, kern in (("tiled", sl.SL_KERNEL_AUTO), ("plain", sl.SL_KERNEL_GENERIC)):
        g = sl.Grid(2, (n, n), 3, sl.SL_F32, lo=(0.0, -0.5), hi=(1.0, 0.5), velocity="nlsw", velocity_params=params,
                    max_order=2, limiter_threshold=-1.0, kernel=kern)
        f = torch.tensor(h, dtype=torch.float32, device=DEV)
        l0 = g.diagnostics()["kernel_launches"]
        g.step(f, torch.empty_like(f), 0.0, 0.5 / n, 8)
        torch.cuda.synchronize()
        if name == "tiled":
            assert g.diagnostics()["kernel_launches"] - l0 == 8 * ((4 if nu == 0.0 else 7) + 1)
        d = g.diagnostics()
        assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0
        out[name] = f.double().cpu().numpy()
    assert float(np.abs(out["tiled"] - out["plain"]).max()) <= 1e-5 * amp


def test_viscous_shear_decay_f32(sl):
    """A shear wave u1 = 0.05 sin(2 pi x2) with nu = 0.01 decays as exp(-nu (2 pi)^2 t) on the FP32
    production path (Z2, 64^2, to t = 0.5) within 4e-5 of its amplitude (FP32 rounding over 64
    steps; the decay itself is 0.18 of the amplitude)."""
    n, nu, amp, T = 64, 0.01, 0.05, 0.5
    x = np.arange(n) / n
    _, X2 = np.meshgrid(x, x)
    u = amp * np.sin(2 * np.pi * X2)
    g = sl.Grid(2, (n, n), 3, sl.SL_F32, velocity="nlsw", velocity_params=[0.0, nu], max_order=2,
                limiter_threshold=-1.0)
    f = torch.tensor(np.stack([np.zeros_like(u), u, np.zeros_like(u)]), dtype=torch.float32, device=DEV)
    steps = int(round(T / (0.5 / n)))
    g.step(f, torch.empty_like(f), 0.0, T / steps, steps)
    torch.cuda.synchronize()
    got = f.double().cpu().numpy()
    err = float(np.abs(got[1] - np.exp(-nu * (2 * np.pi) ** 2 * T) * u).max())
    assert err <= 4e-5 * amp, err


def test_kelvin_f32_accuracy(sl, orc):
    """The FP32 production path to t = 1 on 128^2 against eq. (kelvin): within 10 % of the FP64
    oracle's own discretisation error (6.3e-4 relative L2 with Z2)."""
    wl = inputs.workload_kelvin(128)
    g = sl.grid_for(wl, sl.SL_F32)
    f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
    g.step(f, torch.empty_like(f), 0.0, wl.dt, wl.steps)
    torch.cuda.synchronize()
    got = f.double().cpu().numpy()
    ex = inputs.kelvin_fields(128, 1.0)
    err32 = float(np.sqrt(((got[0] - ex[0]) ** 2).sum() / (ex[0] ** 2).sum()))
    og = orc.OracleGrid(dim=2, n=(128, 128), nfields=3, lo=(0.0, -0.5), hi=(1.0, 0.5), velocity="nlsw",
                        velocity_params=[250.0], max_order=2, threshold=-1.0)
    ref, _ = orc.step(og, wl.fields, 0.0, wl.dt, wl.steps)
    err64 = float(np.sqrt(((ref[0] - ex[0]) ** 2).sum() / (ex[0] ** 2).sum()))
    assert err32 <= 1.1 * err64, (err32, err64)


def test_shallow_water_grids_step_only(sl):
    g = sl.Grid(2, (32, 32), 3, sl.SL_F32, velocity="nlsw", velocity_params=[250.0])
    with pytest.raises(sl.SLError) as ei:
        g.advect(0.0, 0.01)
    assert ei.value.status == sl.SL_ERR_ARG
    assert sl.sl_batch_workspace_bytes([g]) == 0


@pytest.mark.parametrize("n", [(4, 4), (5, 7)])
@pytest.mark.parametrize("max_order", [1, 2])
def test_smallest_grids_f64(sl, orc, n, max_order):
    """Grids of 4 to 7 nodes per side: the fourth-order difference stencil (offsets -2 .. +2) wraps
    round the period; one step matches the oracle within 1e-12."""
    rng = np.random.default_rng(23)
    h = np.stack([0.05 * rng.standard_normal((n[1], n[0])), 0.05 * rng.standard_normal((n[1], n[0])),
                  0.05 * rng.standard_normal((n[1], n[0]))])
    og = orc.OracleGrid(dim=2, n=n, nfields=3, lo=(0.0, -0.5), hi=(1.0, 0.5), velocity="nlsw", velocity_params=[5.0],
                        max_order=max_order, threshold=-1.0, start=orc.START_BACKWARD)
    ref, nfail = orc.step(og, h, 0.0, 0.02, 1)
    g = sl.Grid(2, n, 3, sl.SL_F64, lo=(0.0, -0.5), hi=(1.0, 0.5), velocity="nlsw", velocity_params=[5.0],
                max_order=max_order, limiter_threshold=-1.0)
    f = torch.tensor(h, dtype=torch.float64, device=DEV)
    g.step(f, torch.empty_like(f), 0.0, 0.02, 1)
    torch.cuda.synchronize()
    assert nfail == 0
    assert np.abs(f.cpu().numpy() - ref).max() <= 1e-12 * max(1.0, float(np.abs(ref).max()))
