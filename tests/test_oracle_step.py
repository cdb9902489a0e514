"""Pins of the oracle's moments (Sec. 3.1, Table 1) and of the whole FSL step.

* Table 1's Exact row is reproduced (truncated to the 4 printed decimals) by the discrete
  moments of the cosine hill (eq. alpha) on the grid decoded in tests/golden/table1_exact.txt.
* The relative L1 error of the cosine hill after one solid-body turn decays with slope about 3
  (Sec. 3.1) with the cubic Z-spline and the limiter off, at a fixed number of steps per turn.
* Higher order lowers that error (Z2 below Z1 below Z0), as in Table 1's ordering.
* The 3-D deformation flow reverses at t = T: the field returns to its initial state within the
  scheme's error, and the error shrinks with resolution.
"""
import math
import os

import numpy as np
import pytest

from paper_1410_2817_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_exact.txt")


def _golden_row():
    with open(GOLDEN) as f:
        return [float(v) for line in f if not line.startswith("#") for v in line.split()]


def test_table1_exact_row(oracle_mod):
    n, lo, hi, h = inputs.table1_grid()
    g = oracle_mod.OracleGrid(dim=2, n=n, lo=lo, hi=hi)
    m = oracle_mod.moments(g, h, 4)
    printed = _golden_row()
    assert len(printed) == 5
    for got, ref in zip(m, printed):
        assert math.trunc(got * 1e4) / 1e4 == pytest.approx(ref, abs=1e-12), (got, ref)


def test_moments_of_a_point_mass(oracle_mod):
    g = oracle_mod.OracleGrid(dim=3, n=(4, 6, 8), lo=(0, -1, 2), hi=(2, 2, 6))
    h = np.zeros((8, 6, 4))
    h[5, 2, 3] = 2.0  # x = 0 + 3*0.5, y = -1 + 2*0.5, z = 2 + 5*0.5
    x = np.array([1.5, 0.0, 4.5]) - np.array([1.0, 0.5, 4.0])
    m = oracle_mod.moments(g, h, 4)
    assert m[0] == 2.0
    for p in range(1, 5):
        assert m[p] == pytest.approx(2.0 * np.sum(x ** p), abs=1e-14)


def _sbr_error(oracle_mod, n, max_order, steps=32, threshold=-1.0):
    h0 = inputs.cosine_hill((n, n), (0, 0), (1, 1), (0.25, 0.5), 0.1)[None]
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), velocity="solid_body", velocity_params=[2 * math.pi, 0.5, 0.5],
                              max_order=max_order, threshold=threshold)
    h, _ = oracle_mod.step(g, h0, 0.0, 1.0 / steps, steps)
    return float(np.abs(h - h0).sum() / np.abs(h0).sum())


def test_sbr_l1_convergence_slope(oracle_mod):
    ns = (32, 64, 128)
    errs = [_sbr_error(oracle_mod, n, 1) for n in ns]
    slope = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert slope >= 2.5, (errs, slope)


def test_higher_order_is_more_accurate(oracle_mod):
    e = [_sbr_error(oracle_mod, 64, m) for m in (0, 1, 2)]
    assert e[2] < e[1] < e[0], e


def test_dissipation_error_of_z2_far_below_z1(oracle_mod):
    """Sec. 3.1: on the Table 1 grid the dissipation error after one turn is about two orders of
    magnitude smaller with Z2 than with Z1.  The paper gives no step count; at 50 steps per turn
    (limiter off) the oracle's ratio is about 57, and 40-60 over 25-200 steps.  The error is the
    squared change of the standard deviation, less the squared change of the mean (eq. as
    printed; the mean term is below 1e-13 here)."""
    n, lo, hi, h = inputs.table1_grid()
    diss = []
    for m in (1, 2):
        g = oracle_mod.OracleGrid(dim=2, n=n, lo=lo, hi=hi, velocity="solid_body",
                                  velocity_params=[2 * math.pi, 1.0, 1.0], max_order=m, threshold=-1.0)
        out, _ = oracle_mod.step(g, h[None], 0.0, 1.0 / 50, 50)
        diss.append((h.std() - out[0].std()) ** 2 - (h.mean() - out[0].mean()) ** 2)
    assert 0.0 < diss[1] and diss[0] > 30.0 * diss[1], diss


def test_limiter_lowers_order_on_the_hill(oracle_mod):
    """The literal criterion flags the hill's smooth top and foot, so the limited scheme is less
    accurate on this smooth field than the unlimited one, but still well below pure Z0."""
    e_lim = _sbr_error(oracle_mod, 64, 1, threshold=0.25)
    e_free = _sbr_error(oracle_mod, 64, 1)
    e_z0 = _sbr_error(oracle_mod, 64, 0)
    assert e_free < e_lim < e_z0 * 1.05


def test_deform3d_returns_at_period(oracle_mod):
    errs = []
    for n in (24, 32):
        wl = inputs.workload_deform3d(n=n, steps=30, dt=0.1)
        g = oracle_mod.OracleGrid(dim=3, n=(n, n, n), nfields=2, velocity="deform3d", velocity_params=[3.0],
                                  threshold=-1.0)
        h, nfail = oracle_mod.step(g, wl.fields, 0.0, 0.1, 30)
        assert nfail == 0
        errs.append(float(np.abs(h[0] - wl.fields[0]).sum() / np.abs(wl.fields[0]).sum()))
    # the flow stretches the Gaussian (sigma 0.08 = 2-2.6 cells here) into thin sheets; the return
    # error is large at these sizes but must fall with resolution
    assert errs[1] < 0.9 * errs[0] < 0.8, errs


def test_sbr64_workload_runs(oracle_mod):
    """The 64x64 solid-body rotation of a cone and slotted disk: the failed targets (elements
    sheared across the non-periodic seam of the rotation) stay where the fields vanish."""
    wl = inputs.workload_sbr64()
    g = oracle_mod.OracleGrid(dim=2, n=wl.n, nfields=1, velocity=wl.velocity, velocity_params=wl.velocity_params)
    D = oracle_mod.advect(g, 0.0, wl.dt)
    out = oracle_mod.remap(g, D, oracle_mod.flags(g, wl.fields), wl.fields)
    bad = out.status != oracle_mod.OK
    assert bad.any()
    assert np.all(wl.fields[0][bad] == 0.0)
    x, y = inputs.node_coords(wl.n)
    assert np.all(np.maximum(np.abs(x[bad] - 0.5), np.abs(y[bad] - 0.5)) > 0.35)
    assert out.h.min() >= -0.2 and out.h.max() <= 1.2
