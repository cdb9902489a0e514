"""Oracle pins for the carried velocity (Sec. 3.2, Burgers): every node moves with the velocity it
carries as a transported field (Du/Dt = 0), so its trajectory over a step is the straight line
X + dt u(X), whatever the integrator; a constant carried velocity reduces to the uniform flow; and
a smooth 1-D profile follows the exact solution of the inviscid Burgers equation (characteristics)
up to the interpolation error, which falls at the Z-spline's order under refinement."""
import numpy as np
import pytest

from paper_1410_2817_gb300 import inputs


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("integrator,substeps", [("rk4", 1), ("wrk3", 1), ("wrk3", 3), ("rk4", 4)])
def test_carried_displacement_is_the_straight_line(orc, integrator, substeps):
    n = (24, 20)
    rng = np.random.default_rng(3)
    h = rng.uniform(-1.0, 1.0, size=(3, 20, 24))
    dt = 0.013
    # velocity components taken from fields 2 (x) and 0 (y)
    g = orc.OracleGrid(dim=2, n=n, nfields=3, velocity="carried", velocity_params=[2, 0], integrator=integrator,
                       substeps=substeps)
    D = orc.advect_carried(g, h, dt)
    assert np.allclose(D[..., 0], dt * h[2] * n[0], rtol=0, atol=1e-12)
    assert np.allclose(D[..., 1], dt * h[0] * n[1], rtol=0, atol=1e-12)
    # default components: the first dim fields
    g0 = orc.OracleGrid(dim=2, n=n, nfields=3, velocity="carried", velocity_params=[])
    D0 = orc.advect_carried(g0, h, dt)
    assert np.allclose(D0[..., 0], dt * h[0] * n[0], rtol=0, atol=1e-12)
    assert np.allclose(D0[..., 1], dt * h[1] * n[1], rtol=0, atol=1e-12)


def test_carried_3d_components(orc):
    n = (8, 6, 5)
    rng = np.random.default_rng(4)
    h = rng.uniform(-1.0, 1.0, size=(3, 5, 6, 8))
    g = orc.OracleGrid(dim=3, n=n, nfields=3, velocity="carried", velocity_params=[])
    D = orc.advect_carried(g, h, 0.02)
    for a in range(3):
        assert np.allclose(D[..., a], 0.02 * h[a] * n[a], rtol=0, atol=1e-12)


def test_constant_carried_velocity_is_the_uniform_flow(orc):
    """Fields u = 0.37, v = -0.21 everywhere (carried) move a passive third field exactly as the
    uniform flow (0.37, -0.21) does; the velocity fields stay constant."""
    n = (32, 28)
    rng = np.random.default_rng(5)
    tracer = rng.uniform(0.0, 1.0, size=(28, 32))
    h = np.stack([np.full((28, 32), 0.37), np.full((28, 32), -0.21), tracer])
    gc = orc.OracleGrid(dim=2, n=n, nfields=3, velocity="carried", velocity_params=[])
    out_c, fail_c = orc.step(gc, h, 0.0, 0.05, 3)
    gu = orc.OracleGrid(dim=2, n=n, nfields=1, velocity="uniform", velocity_params=[0.37, -0.21])
    out_u, fail_u = orc.step(gu, tracer[None], 0.0, 0.05, 3)
    assert fail_c == 0 and fail_u == 0
    assert np.max(np.abs(out_c[2] - out_u[0])) <= 1e-13
    assert np.max(np.abs(out_c[0] - 0.37)) <= 1e-14 and np.max(np.abs(out_c[1] + 0.21)) <= 1e-14


def _burgers_exact(x, t, amp):
    """u(x, t) of u_t + u u_x = 0, u(x, 0) = amp sin(2 pi x), before the shock: u = u0(s) with
    s + t u0(s) = x (Newton on the characteristic foot s)."""
    s = x.copy()
    for _ in range(60):
        f = s + t * amp * np.sin(2 * np.pi * s) - x
        df = 1.0 + t * amp * 2 * np.pi * np.cos(2 * np.pi * s)
        s = s - f / df
    return amp * np.sin(2 * np.pi * s)


@pytest.mark.parametrize("max_order,min_rate", [(1, 1.8), (0, 0.85)])
def test_smooth_burgers_follows_the_characteristics(orc, max_order, min_rate):
    """u0 = 0.1 sin(2 pi x), v = 0 on a 2-D grid with 4 nodes in y, limiter off, to t = 0.8 (the
    shock forms at t = 1/(0.2 pi) = 1.59), dt proportional to dx (CFL 0.64).  Each remap locates
    the targets through the multilinear element map, exact only for displacements linear across
    an element: on this curved deformation it misplaces a target by O(dx^2 dt), so after T/dt
    remaps the error is O(dx^2) for the cubic Z1 (its own interpolation error, O(dx^4) per remap,
    is smaller); the linear Z0 loses O(dx^2) per remap, O(dx) in all.  The max error against
    the exact solution falls at least at those rates from 64 to 128 nodes (measured 2.0 and
    0.94)."""
    amp, t_end = 0.1, 0.8
    errs = []
    for nx in (64, 128):
        steps = nx // 8
        dt = t_end / steps
        x = np.arange(nx) / nx
        u0 = np.tile(amp * np.sin(2 * np.pi * x), (4, 1))
        h = np.stack([u0, np.zeros_like(u0)])
        g = orc.OracleGrid(dim=2, n=(nx, 4), nfields=2, velocity="carried", velocity_params=[], threshold=-1.0,
                           max_order=max_order)
        out, nfail = orc.step(g, h, 0.0, dt, steps)
        assert nfail == 0
        assert np.max(np.abs(out[1])) == 0.0
        exact = _burgers_exact(x, t_end, amp)
        errs.append(float(np.max(np.abs(out[0] - exact[None, :]))))
    rate = np.log2(errs[0] / errs[1])
    assert rate >= min_rate, (errs, rate)


def test_burgers_workload_initial_condition():
    """The Sec. 3.2 pulse: radial, |u| peaks at 1 on the ring r = 0.2, zero at the centre node."""
    wl = inputs.workload_burgers(64)
    u, v = wl.fields
    speed = np.hypot(u, v)
    assert abs(float(speed.max()) - 1.0) < 0.02
    assert speed[32, 32] == 0.0
    x, y = inputs.node_coords((64, 64))
    # parallel to (x - 1/2, y - 1/2): the cross product vanishes
    assert np.max(np.abs(u * (y - 0.5) - v * (x - 0.5))) < 1e-15
    assert wl.velocity == "carried" and wl.steps * wl.dt >= 0.4
