"""The time factors cos(pi t / T) of the swirl and the deformation flow (eq. vel) come from one
function compiled for host and device (`cospi_time`, `stage_time_factors` in sl_device.cuh): the
host fills them for single grids, the device for batches.  Compiled here for the host with nvcc
(no GPU needed) and checked against the definition: cos(pi x) within a few units in the last
place, exact at the quarter points, and the stage times of RK4 and of Williamson's RK3."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_2817_gb300", "csrc")

PROGRAM = r"""
#include <stdio.h>
#include "sl_device.cuh"
int main()
{
    double x;
    while (scanf("%lf", &x) == 1) printf("%.17g\n", cospi_time(x));
    // stage factors: RK4 one sub-step, RK4 three sub-steps, RK3 two sub-steps (t = 0.3, dt = 0.2, T = 5)
    double ct[12];
    stage_time_factors<double>(0.3, 0.2, 1, SL_RK4, 5.0, ct);
    for (int k = 0; k < 3; ++k) printf("rk4_1 %.17g\n", ct[k]);
    stage_time_factors<double>(0.3, 0.2, 3, SL_RK4, 5.0, ct);
    for (int k = 0; k < 9; ++k) printf("rk4_3 %.17g\n", ct[k]);
    stage_time_factors<double>(0.3, 0.2, 2, SL_WRK3, 5.0, ct);
    for (int k = 0; k < 6; ++k) printf("wrk3_2 %.17g\n", ct[k]);
    return 0;
}
"""


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("timefactors")
    src, exe = d / "tf.cu", d / "tf"
    src.write_text(PROGRAM)
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2",
                        "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def _run(exe, xs):
    r = subprocess.run([exe], input="\n".join(repr(float(x)) for x in xs), capture_output=True, text=True)
    assert r.returncode == 0
    return r.stdout.split("\n")


def test_cospi_time_against_the_definition(program):
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.uniform(-8, 8, 4000), np.arange(-16, 17) * 0.25, [1e-9, -1e-9, 0.5 + 1e-12]])
    out = _run(program, xs)
    got = np.array([float(v) for v in out[:len(xs)]])
    # the definition, with the argument reduced exactly first (x - 2 round(x/2) is exact)
    ref = np.array([math.cos(math.pi * (x - 2.0 * round(x / 2.0))) for x in xs])
    assert np.max(np.abs(got - ref)) <= 8e-16
    # quarter points: 1, +-sqrt(1/2), 0, -1 exactly where cos is exact
    for x, v in zip(xs, got):
        q = x * 4.0
        if q == int(q) and int(q) % 2 == 0:
            assert v == {0: 1.0, 2: 0.0, 4: -1.0, 6: 0.0}[int(q) % 8], (x, v)


def test_stage_time_factors(program):
    lines = [ln for ln in _run(program, []) if ln]
    vals = {}
    for ln in lines:
        name, v = ln.split()
        vals.setdefault(name, []).append(float(v))
    t, dt, T = 0.3, 0.2, 5.0

    def f(tt):
        return math.cos(math.pi * tt / T)

    assert np.allclose(vals["rk4_1"], [f(t), f(t + dt / 2), f(t + dt)], rtol=0, atol=1e-15)
    h = dt / 3
    want = [f(t + s * h + c * h) for s in range(3) for c in (0.0, 0.5, 1.0)]
    assert np.allclose(vals["rk4_3"], want, rtol=0, atol=1e-15)
    h = dt / 2
    want = [f(t + s * h + c * h) for s in range(2) for c in (0.0, 1.0 / 3.0, 0.75)]
    assert np.allclose(vals["wrk3_2"], want, rtol=0, atol=1e-15)
