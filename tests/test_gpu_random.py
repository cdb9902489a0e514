"""Randomised cases on the CUDA path: grid sides 4-300 (ragged tiles, windows wider than the grid),
1-8 fields, cubic or quintic, limiter on or off, smooth displacements of random size.  The FP32
tiled kernels must compute what the plain FP32 kernels compute, and the FP64 kernels what the
oracle computes on sampled targets."""
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


def _case(seed):
    rng = np.random.default_rng(seed)
    n = (int(rng.integers(4, 300)), int(rng.integers(4, 300)))
    nf = int(rng.integers(1, 9))
    max_order = int(rng.integers(1, 3))
    thr = 0.25 if rng.uniform() < 0.7 else -1.0
    amp = float(rng.uniform(0.05, 0.4))
    D = inputs.smooth_displacement(n, amplitude=amp, seed=seed, shift=tuple(rng.uniform(-4, 4, 2)))
    x = np.arange(n[0]) / n[0]
    y = np.arange(n[1]) / n[1]
    X, Y = np.meshgrid(x, y)
    h = []
    for f in range(nf):
        k = rng.integers(1, 4, 2)
        v = np.sin(2 * np.pi * (k[0] * X + k[1] * Y) + rng.uniform(0, 6))
        if f % 3 == 1:
            v = v + (rng.uniform(size=v.shape) > 0.8)
        h.append(v)
    return n, nf, max_order, thr, D, np.stack(h)


@pytest.mark.parametrize("seed", range(24))
def test_tiled_matches_plain_f32(sl, seed):
    n, nf, mo, thr, D, h = _case(seed)
    outs, diags = {}, {}
    for name, kern in (("tiled", sl.SL_KERNEL_TILED), ("plain", sl.SL_KERNEL_GENERIC)):
        g = sl.Grid(2, n, nf, sl.SL_F32, max_order=mo, limiter_threshold=thr, walk_start=sl.SL_START_BACKWARD,
                    kernel=kern)
        g.set_displacement(torch.tensor(D, dtype=torch.float32, device=DEV))
        hin = torch.tensor(h, dtype=torch.float32, device=DEV)
        hout = torch.empty_like(hin)
        g.remap(hin, hout)
        torch.cuda.synchronize()
        outs[name] = hout.double().cpu().numpy()
        diags[name] = g.diagnostics()
    diff = np.abs(outs["tiled"] - outs["plain"])
    ntar = n[0] * n[1]
    assert float((diff > 4e-6 * 2.0).mean()) <= max(2.0 / (ntar * nf), 2e-4), (n, nf, mo, thr, float(diff.max()))
    dt, dg = diags["tiled"], diags["plain"]
    assert dt["targets"] == dg["targets"] == ntar
    fails = lambda d: d["fail_locate"] + d["fail_newton"] + d["fail_fold"]
    assert fails(dt) == fails(dg) == 0


@pytest.mark.parametrize("seed", range(100, 106))
def test_f64_matches_oracle_sampled(sl, orc, seed):
    n, nf, mo, thr, D, h = _case(seed)
    og = orc.OracleGrid(dim=2, n=n, nfields=nf, max_order=mo, threshold=thr, start=orc.START_BACKWARD)
    fl = orc.flags(og, h)
    g = sl.Grid(2, n, nf, sl.SL_F64, max_order=mo, limiter_threshold=thr, walk_start=sl.SL_START_BACKWARD)
    g.set_displacement(torch.tensor(D, dtype=torch.float64, device=DEV))
    hin = torch.tensor(h, dtype=torch.float64, device=DEV)
    hout = torch.empty_like(hin)
    g.remap(hin, hout)
    torch.cuda.synchronize()
    got = hout.cpu().numpy()
    rng = np.random.default_rng(seed + 7)
    for (jx, jy) in zip(rng.integers(0, n[0], 150), rng.integers(0, n[1], 150)):
        c, xi, st, _, _ = orc.locate(og, D, (int(jx), int(jy)))
        assert st == orc.OK
        if np.any(np.minimum(np.abs(xi), np.abs(1 - xi)) < TIE):
            continue
        for q in range(nf):
            v = orc.interp(og, h[q], c, xi, orc.order(og, fl, c, q))
            assert abs(got[q, jy, jx] - v) <= 1e-12 * max(1.0, abs(v)), (n, nf, mo, jx, jy, q)
