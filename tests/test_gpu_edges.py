"""Edge cases of the CUDA path through the C ABI: the largest and the smallest grid sides, targets
that all sit on vertices (zero and integer displacements: the remap must return the shifted input
exactly), one to eight fields (the field groups of the tiled and blocked kernels), and the
pipelined tile configuration against the default one."""
import numpy as np
import pytest
import torch

from paper_1410_2817_gb300 import inputs

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


def _grid(sl, dim, n, nf, dtype, kernel=None, threshold=0.25, tile_config=0):
    kw = {"kernel": kernel} if kernel is not None else {}
    return sl.Grid(dim, n, nf, dtype, velocity="uniform", velocity_params=[0.0, 0.0, 0.0], limiter_threshold=threshold,
                   walk_start=sl.SL_START_BACKWARD, tile_config=tile_config, **kw)


def _smooth_fields(shape, nf, seed):
    """Smooth periodic fields (a few low modes) of the given plane shape (..., ny, nx)."""
    rng = np.random.default_rng(seed)
    axes = [np.arange(s) / s for s in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    out = []
    for _ in range(nf):
        v = np.zeros(shape)
        for _ in range(3):
            k = rng.integers(1, 3, size=len(shape))
            ph = rng.uniform(0, 2 * np.pi)
            v += rng.normal() * np.cos(2 * np.pi * sum(int(kk) * g for kk, g in zip(k, grids)) + ph)
        out.append(v)
    return np.stack(out)


@pytest.mark.parametrize("n", [(1 << 20, 4), (4, 1 << 20), (4, 4)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_extreme_sides(sl, orc, n, dtype):
    """Sides at both ends of the accepted range [4, 2^20]: the FP64 path matches the oracle within
    1e-12 with the limiter on; the FP32 tiled path matches it to FP32 accuracy (limiter off, so
    that FP32 and FP64 threshold decisions cannot differ)."""
    n0, n1 = n
    D = inputs.smooth_displacement(n, amplitude=0.3, seed=7, shift=(1.6, -0.7))
    h = np.stack([_smooth_fields((n1, n0), 2, seed=8)[0], (np.arange(n0 * n1).reshape(n1, n0) % 7 == 0) * 1.0])
    thr = 0.25 if dtype == "f64" else -1.0
    og = orc.OracleGrid(dim=2, n=n, nfields=2, velocity="uniform", velocity_params=[0.0, 0.0, 0.0], threshold=thr,
                        start=orc.START_BACKWARD)
    fl = orc.flags(og, h)
    sd, td = (sl.SL_F64, torch.float64) if dtype == "f64" else (sl.SL_F32, torch.float32)
    g = _grid(sl, 2, n, 2, sd, threshold=thr)
    g.set_displacement(torch.tensor(D, dtype=td, device=DEV))
    hin = torch.tensor(h, dtype=td, device=DEV)
    hout = torch.empty_like(hin)
    g.remap(hin, hout)
    torch.cuda.synchronize()
    got = hout.double().cpu().numpy()
    d = g.diagnostics()
    assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0
    rng = np.random.default_rng(9)
    nsamp = 16 if n == (4, 4) else 400
    idx = [(x, y) for x in range(4) for y in range(4)] if n == (4, 4) else \
        list(zip(rng.integers(0, n0, nsamp), rng.integers(0, n1, nsamp)))
    for (jx, jy) in idx:
        c, xi, st, _, _ = orc.locate(og, D, (int(jx), int(jy)))
        assert st == orc.OK
        for f in range(2):
            v = orc.interp(og, h[f], c, xi, orc.order(og, fl, c, f))
            a = got[f, jy, jx]
            if dtype == "f64":
                if not np.any(np.minimum(np.abs(xi), np.abs(1 - xi)) < TIE):
                    assert abs(a - v) <= 1e-12 * max(1.0, abs(v)), (jx, jy, f, a, v)
            else:
                assert abs(a - v) <= 2e-5 * max(1.0, abs(v)), (jx, jy, f, a, v)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("path", ["f64", "f32_generic", "f32_tiled"])
@pytest.mark.parametrize("shift", [(0, 0, 0), (3, -2, 1)])
def test_vertex_targets_exact(sl, dim, path, shift):
    """Every departure point on a node (zero or integer displacement): each target's element has
    the node as its lower corner and xi = 0, where the Z-spline weights are exactly 1 and 0, so the
    remap returns the periodically shifted input bit for bit (the limiter is on: the order does
    not matter at a node)."""
    n = (20, 12) if dim == 2 else (12, 10, 8)
    nf = 3
    shape = tuple(reversed(n))
    rng = np.random.default_rng(11)
    h = rng.standard_normal((nf,) + shape)
    sd, td = (sl.SL_F64, torch.float64) if path == "f64" else (sl.SL_F32, torch.float32)
    kernel = sl.SL_KERNEL_GENERIC if path == "f32_generic" else None
    g = _grid(sl, dim, n, nf, sd, kernel=kernel)
    D = np.zeros(shape + (dim,))
    for a in range(dim):
        D[..., a] = shift[a]
    g.set_displacement(torch.tensor(D, dtype=td, device=DEV))
    hin = torch.tensor(h, dtype=td, device=DEV)
    hout = torch.empty_like(hin)
    g.remap(hin, hout)
    torch.cuda.synchronize()
    got = hout.cpu().numpy()
    # departure point of target j is j - s: out[j] = in[(j - s) mod n]; numpy axes run (z,) y, x
    roll = tuple(shift[a] for a in reversed(range(dim)))
    want = np.roll(hin.cpu().numpy(), roll, axis=tuple(range(1, dim + 1)))
    assert np.array_equal(got, want)
    d = g.diagnostics()
    assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0
    assert d["newton_f64"] == 0


@pytest.mark.parametrize("nf", [1, 5, 8])
@pytest.mark.parametrize("tile_config", [1, 5])
def test_field_counts_tiled_vs_generic(sl, nf, tile_config):
    """One field (a single lane of a float4 group) and five / eight fields (two float4 groups; the
    pipelined configuration falls back to 32x32 above four fields): the tiled FP32 kernel computes
    what the plain FP32 kernel computes."""
    n = (96, 70)
    D = inputs.smooth_displacement(n, amplitude=0.3, seed=12, shift=(2.2, 1.3))
    h = _smooth_fields((70, 96), nf, seed=13)
    h[0] += (np.arange(96)[None, :] > 48) * 1.0  # a jump for the limiter
    outs = {}
    for name, kern in (("generic", sl.SL_KERNEL_GENERIC), ("tiled", sl.SL_KERNEL_TILED)):
        g = _grid(sl, 2, n, nf, sl.SL_F32, kernel=kern, tile_config=tile_config)
        g.set_displacement(torch.tensor(D, dtype=torch.float32, device=DEV))
        hin = torch.tensor(h, dtype=torch.float32, device=DEV)
        hout = torch.empty_like(hin)
        g.remap(hin, hout)
        torch.cuda.synchronize()
        outs[name] = hout.double().cpu().numpy()
    scale = max(1.0, float(np.abs(h).max()))
    diff = np.abs(outs["tiled"] - outs["generic"])
    # same elements and orders away from faces; a target within the FP32 slack of a face may be
    # taken in the neighbouring element, whose order can differ: such ties stay rare
    assert float((diff > 2e-6 * scale).mean()) <= 2e-4, float(diff.max())


def test_pipelined_step_equals_default_tiles(sl):
    """sl_step on the pipelined configuration (5: persistent CTAs staging the next tiles; the next
    step's trajectories integrated in the same launch) gives bit-for-bit what the default 32x32
    configuration gives: the per-target arithmetic is the same code."""
    wl = inputs.workload_swirl(640, steps=4)  # 20 x 20 tiles: several tiles per CTA on 152 SMs
    outs = {}
    for cfg in (1, 5):
        g = sl.grid_for(wl, sl.SL_F32, tile_config=cfg)
        f = torch.tensor(wl.fields, dtype=torch.float32, device=DEV)
        g.step(f, torch.empty_like(f), 0.1, wl.dt, 4)
        torch.cuda.synchronize()
        outs[cfg] = f.cpu()
        d = g.diagnostics()
        assert d["fail_locate"] + d["fail_newton"] + d["fail_fold"] == 0
    assert torch.equal(outs[1], outs[5])


@pytest.mark.parametrize("nf", [3, 6])
def test_blocked3d_field_counts(sl, nf):
    """3-D blocked kernel with four-field (three used) and eight-field (six used) register groups:
    the same values as the plain FP32 kernel."""
    n = (20, 14, 12)
    D = inputs.smooth_displacement(n, amplitude=0.3, seed=14, shift=(1.3, -0.8, 2.1))
    h = _smooth_fields((12, 14, 20), nf, seed=15)
    h[0] += (np.arange(20)[None, None, :] > 9) * 1.0
    outs = {}
    for name, kern in (("generic", sl.SL_KERNEL_GENERIC), ("tiled", sl.SL_KERNEL_TILED)):
        g = _grid(sl, 3, n, nf, sl.SL_F32, kernel=kern)
        g.set_displacement(torch.tensor(D, dtype=torch.float32, device=DEV))
        hin = torch.tensor(h, dtype=torch.float32, device=DEV)
        hout = torch.empty_like(hin)
        g.remap(hin, hout)
        torch.cuda.synchronize()
        outs[name] = (hout.double().cpu().numpy(), g.diagnostics())
    diff = np.abs(outs["tiled"][0] - outs["generic"][0])
    assert float(diff.max()) <= 4e-6 * max(1.0, float(np.abs(h).max())), float(diff.max())
    assert outs["tiled"][1]["order_hist"] == outs["generic"][1]["order_hist"]
