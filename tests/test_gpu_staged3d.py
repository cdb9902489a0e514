"""The staged 3-D FP32 kernel of plain remaps (the field values of each 16x4x4 block's stencils
copied to shared memory while its targets' element search runs: box copies inside the grid,
per-element copies across the periodic seam, global reads where a target's stencil leaves the
window or a block's window exceeds the capacity) against the blocked kernel that gathers every
value through L1 (tile configuration 1; fused steps always run on it).  Both run the same element search, Newton inversion and tap sums (Sec. 2.2, eq.
mapping1, eq. multiZ) on the same values, so their results and counters must be identical, bit
for bit, whichever way each block was staged.  The oracle
comparisons of the 3-D FP32 path (test_gpu_parity.py) run the staged kernel by default."""
import numpy as np
import pytest
import torch

from paper_1410_2817_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda"
COUNTERS = ("targets", "fail_locate", "fail_newton", "fail_fold", "hops_sum", "hops_max", "iters_sum", "iters_max",
            "newton_f64", "order_hist")


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


def _case(orc, name):
    """(n, D in cells (FP64), fields, velocity kwargs) of one case."""
    rng = np.random.default_rng(41)
    if name.startswith("deform"):
        # the deformation flow at the benchmark's step (the same velocity gradient in cells per
        # cell as on the 256^3 grid) and at three times it (some blocks' windows exceed the
        # capacity): blocks inside the grid copied by boxes (rows of a multiple of 4 nodes), seam
        # blocks element by element
        n = (64, 48, 40)
        dt = 0.03 if name == "deform" else 0.09
        og = orc.OracleGrid(dim=3, n=n, nfields=2, velocity="deform3d", velocity_params=[3.0])
        D = orc.advect(og, 0.4, dt)
        x, y, z = inputs.node_coords(n)
        h = np.stack([np.exp(-((x - 0.4) ** 2 + (y - 0.5) ** 2 + (z - 0.45) ** 2) / 0.02),
                      ((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2 <= 0.09).astype(np.float64)])
        return n, D, h
    if name == "ragged":
        # rows of 19 nodes: no tensor maps, every window copied element by element
        n = (19, 13, 11)
        D = inputs.smooth_displacement(n, amplitude=0.3, seed=8, shift=(1.6, -2.2, 0.7))
        h = np.stack([rng.standard_normal((11, 13, 19)).cumsum(axis=2) * 0.1,
                      (rng.uniform(size=(11, 13, 19)) > 0.5) * 1.0])
        return n, D, h
    # steep displacement: a third of the blocks' windows exceed the capacity and read global
    # memory; elements fold
    n = (48, 32, 24)
    D = inputs.smooth_displacement(n, amplitude=2.5, seed=5, shift=(0.3, 0.2, -0.4))
    h = rng.standard_normal((2, 24, 32, 48))
    return n, D, h


def _remap(sl, n, D, h, nf, tile_config, threshold=0.25):
    g = sl.Grid(3, n, nf, sl.SL_F32, limiter_threshold=threshold, walk_start=sl.SL_START_BACKWARD,
                kernel=sl.SL_KERNEL_TILED, tile_config=tile_config)
    hin = torch.tensor(np.asarray(h[:nf]), dtype=torch.float32, device=DEV)
    hout = torch.empty_like(hin)
    g.set_displacement(torch.tensor(D, dtype=torch.float32, device=DEV))
    g.remap(hin, hout)
    torch.cuda.synchronize()
    return hout, g.diagnostics()


@pytest.mark.parametrize("nf", [1, 2])
@pytest.mark.parametrize("case", ["deform", "deform_3dt", "ragged", "steep"])
def test_staged_equals_blocked(sl, orc, case, nf):
    n, D, h = _case(orc, case)
    out_s, d_s = _remap(sl, n, D, h, nf, 0)
    out_b, d_b = _remap(sl, n, D, h, nf, 1)
    assert torch.equal(out_s, out_b), float((out_s - out_b).abs().max())
    for k in COUNTERS:
        assert d_s[k] == d_b[k], (k, d_s[k], d_b[k])
    assert d_s["targets"] == int(np.prod(n)) and d_s["timeouts"] == 0
    blocks = -(-n[0] // 16) * -(-n[1] // 4) * -(-n[2] // 4)
    if case in ("steep", "deform_3dt"):
        assert 0 < d_s["tiles_fallback"] < blocks  # some blocks read global memory only
    else:
        assert d_s["tiles_fallback"] == 0, (d_s["tiles_fallback"], blocks)


def test_staged_limiter_off_and_linear(sl, orc):
    """The order choice with the limiter off (cubic everywhere) and with max_order 0 (trilinear)."""
    n, D, h = _case(orc, "deform")
    for thr in (-1.0, 0.25):
        out_s, _ = _remap(sl, n, D, h, 2, 0, threshold=thr)
        out_b, _ = _remap(sl, n, D, h, 2, 1, threshold=thr)
        assert torch.equal(out_s, out_b), thr
    outs = []
    for tc in (0, 1):
        g = sl.Grid(3, n, 2, sl.SL_F32, max_order=0, walk_start=sl.SL_START_BACKWARD, kernel=sl.SL_KERNEL_TILED,
                    tile_config=tc)
        hin = torch.tensor(h, dtype=torch.float32, device=DEV)
        hout = torch.empty_like(hin)
        g.set_displacement(torch.tensor(D, dtype=torch.float32, device=DEV))
        g.remap(hin, hout)
        torch.cuda.synchronize()
        outs.append(hout)
        assert g.diagnostics()["order_hist"][0] == 2 * int(np.prod(n))
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("nf", [1, 2])
def test_fused_steps_equal_staged_remaps(sl, nf):
    """A fused step (blocked kernel: the launch also integrates the next trajectories) and a plain
    remap (staged kernel) of the same fields with the same displacement give identical fields, step
    after step."""
    n = (64, 32, 24)
    kw = dict(velocity="deform3d", velocity_params=[3.0], walk_start=sl.SL_START_BACKWARD, kernel=sl.SL_KERNEL_TILED)
    gs = sl.Grid(3, n, nf, sl.SL_F32, **kw)
    gr = sl.Grid(3, n, nf, sl.SL_F32, **kw)
    f0 = torch.tensor(np.asarray(inputs.deform3d_fields(64))[:nf, :24, :32, :64], dtype=torch.float32, device=DEV)
    fs, fr = f0.clone(), f0.clone()
    t, dt = 0.2, 0.06
    for _ in range(3):
        gs.step(fs, torch.empty_like(fs), t, dt, 1)
        gr.advect(t, dt)
        out = torch.empty_like(fr)
        gr.remap(fr, out)
        fr = out
        t += dt
    torch.cuda.synchronize()
    assert torch.equal(fs, fr), float((fs - fr).abs().max())
