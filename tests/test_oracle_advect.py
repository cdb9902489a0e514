"""Pins of the oracle's trajectories (eq. vel) and velocity fields.

* Solid-body rotation is a linear ODE x' = A (x - c); one classical RK4 step maps x - c by the
  degree-4 Taylor polynomial of exp(dt A) exactly, so the displacement has a closed form.
* Uniform flow: D = u dt / dx exactly.
* Swirl flow: against a tight-tolerance ODE solve, the error shrinks like dt^5 (local order of
  RK4), which fixes the stage times and weights.
* Velocity fields: stagnation lines are exact zeros, the flows are divergence-free, the
  deformation flows stop at t = T/2.
* Williamson's low-storage RK3 and sub-stepping: on the linear rotation ODE every three-stage
  third-order method maps x - c by the degree-3 Taylor polynomial of exp(h A), and k sub-steps by
  its k-th power; on the (time-dependent) swirl the local error shrinks like h^4, which a wrong
  stage time or weight would drop to h^3; uniform flow stays exact.
"""
import math

import numpy as np
import pytest

from paper_1410_2817_gb300 import inputs


def test_solid_body_rk4_closed_form(oracle_mod):
    n, dt, om = 16, 0.05, 2 * math.pi
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), velocity="solid_body", velocity_params=[om, 0.5, 0.5])
    D = oracle_mod.advect(g, 0.3, dt)
    A = np.array([[0.0, -om], [om, 0.0]])
    hA = dt * A
    M = np.eye(2) + hA + hA @ hA / 2 + hA @ hA @ hA / 6 + hA @ hA @ hA @ hA / 24
    x, y = inputs.node_coords((n, n))
    r = np.stack([x - 0.5, y - 0.5], axis=-1)
    expect = (r @ (M - np.eye(2)).T) * n
    assert np.max(np.abs(D - expect)) <= 1e-12


def test_uniform_flow_exact(oracle_mod):
    g = oracle_mod.OracleGrid(dim=3, n=(4, 5, 6), velocity="uniform", velocity_params=[0.3, -0.2, 0.7])
    D = oracle_mod.advect(g, 0.0, 0.25)
    for a, (u, n) in enumerate(zip([0.3, -0.2, 0.7], (4, 5, 6))):
        assert np.max(np.abs(D[..., a] - u * 0.25 * n)) <= 1e-14


def test_swirl_local_error_order(oracle_mod):
    integ = pytest.importorskip("scipy.integrate")
    n = 8
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), velocity="swirl2d", velocity_params=[5.0])
    t0 = 0.7

    def rhs(t, x):
        return oracle_mod.velocity_at(g, x, t)[0]

    errs = []
    for dt in (0.08, 0.04):
        D = oracle_mod.advect(g, t0, dt)
        worst = 0.0
        for (iy, ix) in [(1, 1), (2, 5), (3, 3), (6, 2)]:
            x0 = np.array([ix / n, iy / n])
            sol = integ.solve_ivp(rhs, (t0, t0 + dt), x0, rtol=1e-13, atol=1e-15, method="DOP853")
            exact = (sol.y[:, -1] - x0) * n
            worst = max(worst, float(np.max(np.abs(D[iy, ix] - exact))))
        errs.append(worst)
    ratio = errs[0] / errs[1]
    assert 20.0 < ratio < 48.0, errs  # 2^5 = 32


def test_swirl_stagnation_and_symmetry(oracle_mod):
    g = oracle_mod.OracleGrid(dim=2, n=(8, 8), velocity="swirl2d", velocity_params=[5.0])
    pts = np.array([[0.0, 0.3], [0.5, 0.7], [0.2, 0.0], [0.9, 0.5]])
    u = oracle_mod.velocity_at(g, pts, 0.4)
    assert u[0, 0] == 0.0 and u[2, 0] == 0.0 and u[2, 1] == 0.0 and u[3, 0] == 0.0
    assert np.all(oracle_mod.velocity_at(g, pts, 2.5) == 0.0)  # cos(pi t / T) = 0 at t = T/2
    np.testing.assert_allclose(oracle_mod.velocity_at(g, [[0.5, 0.25]], 0.0), [[1.0, 0.0]], atol=1e-15)


@pytest.mark.parametrize("kind,dim,params", [
    ("swirl2d", 2, [5.0]),
    ("deform3d", 3, [3.0]),
    ("fourier2d", 2, inputs.fourier2d_params(np.random.default_rng(3))),
    ("fourier3d", 3, inputs.fourier3d_params(np.random.default_rng(4))),
])
def test_divergence_free(oracle_mod, kind, dim, params):
    g = oracle_mod.OracleGrid(dim=dim, n=(8,) * dim, velocity=kind, velocity_params=params)
    rng = np.random.default_rng(5)
    eps = 1e-5
    scale = 1.0
    for x in rng.uniform(0, 1, (10, dim)):
        div = 0.0
        for a in range(dim):
            e = np.zeros(dim)
            e[a] = eps
            up = oracle_mod.velocity_at(g, x + e, 0.37)[0, a]
            um = oracle_mod.velocity_at(g, x - e, 0.37)[0, a]
            div += (up - um) / (2 * eps)
        scale = max(scale, float(np.max(np.abs(oracle_mod.velocity_at(g, x, 0.37)))))
        assert abs(div) <= 1e-6 * scale * 10


def test_deform3d_components(oracle_mod):
    """u = 2 sin^2(pi x) sin(2 pi y) sin(2 pi z) c, v, w cyclic with amplitude -1."""
    g = oracle_mod.OracleGrid(dim=3, n=(4, 4, 4), velocity="deform3d", velocity_params=[3.0])
    x = np.array([0.5, 0.25, 0.25])  # sin^2(pi/2) = 1, sin(pi/2) = 1
    np.testing.assert_allclose(oracle_mod.velocity_at(g, x, 0.0)[0], [2.0, 0.0, 0.0], atol=1e-15)
    x = np.array([0.25, 0.5, 0.25])
    np.testing.assert_allclose(oracle_mod.velocity_at(g, x, 0.0)[0], [0.0, -1.0, 0.0], atol=1e-15)
    assert np.all(oracle_mod.velocity_at(g, [0.3, 0.6, 0.1], 1.5) == 0.0)


def test_fourier_periodic(oracle_mod):
    p = inputs.fourier2d_params(np.random.default_rng(7))
    g = oracle_mod.OracleGrid(dim=2, n=(8, 8), velocity="fourier2d", velocity_params=p)
    a = oracle_mod.velocity_at(g, [[0.13, 0.71]], 0.0)
    b = oracle_mod.velocity_at(g, [[1.13, -0.29]], 0.0)
    assert np.max(np.abs(a - b)) <= 1e-12


def _taylor(hA, order):
    M, term = np.eye(2), np.eye(2)
    for k in range(1, order + 1):
        term = term @ hA / k
        M = M + term
    return M


@pytest.mark.parametrize("integrator,order", [("rk4", 4), ("wrk3", 3)])
@pytest.mark.parametrize("substeps", [1, 3])
def test_solid_body_substeps_closed_form(oracle_mod, integrator, order, substeps):
    n, dt, om = 16, 0.05, 2 * math.pi
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), velocity="solid_body", velocity_params=[om, 0.5, 0.5],
                              integrator=integrator, substeps=substeps)
    D = oracle_mod.advect(g, 0.3, dt)
    A = np.array([[0.0, -om], [om, 0.0]])
    M = np.linalg.matrix_power(_taylor(dt / substeps * A, order), substeps)
    x, y = inputs.node_coords((n, n))
    r = np.stack([x - 0.5, y - 0.5], axis=-1)
    expect = (r @ (M - np.eye(2)).T) * n
    assert np.max(np.abs(D - expect)) <= 1e-12


def test_wrk3_uniform_flow_exact(oracle_mod):
    g = oracle_mod.OracleGrid(dim=3, n=(4, 5, 6), velocity="uniform", velocity_params=[0.3, -0.2, 0.7],
                              integrator="wrk3", substeps=4)
    D = oracle_mod.advect(g, 0.0, 0.25)
    for a, (u, n) in enumerate(zip([0.3, -0.2, 0.7], (4, 5, 6))):
        assert np.max(np.abs(D[..., a] - u * 0.25 * n)) <= 1e-13


def test_wrk3_swirl_local_error_order(oracle_mod):
    integ = pytest.importorskip("scipy.integrate")
    n = 8
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), velocity="swirl2d", velocity_params=[5.0], integrator="wrk3")
    t0 = 0.7

    def rhs(t, x):
        return oracle_mod.velocity_at(g, x, t)[0]

    errs = []
    for dt in (0.08, 0.04):
        D = oracle_mod.advect(g, t0, dt)
        worst = 0.0
        for (iy, ix) in [(1, 1), (2, 5), (3, 3), (6, 2)]:
            x0 = np.array([ix / n, iy / n])
            sol = integ.solve_ivp(rhs, (t0, t0 + dt), x0, rtol=1e-13, atol=1e-15, method="DOP853")
            exact = (sol.y[:, -1] - x0) * n
            worst = max(worst, float(np.max(np.abs(D[iy, ix] - exact))))
        errs.append(worst)
    ratio = errs[0] / errs[1]
    assert 10.0 < ratio < 24.0, errs  # 2^4 = 16



@pytest.mark.parametrize("integrator,order", [("rk4", 4), ("wrk3", 3)])
def test_substeps_converge_to_the_trajectory(oracle_mod, integrator, order):
    """k sub-steps of h = dt/k over a step of the time-dependent swirl: the local error falls by
    about k^order against one step of dt (each sub-step starts where the last ended, at its own
    time)."""
    integ = pytest.importorskip("scipy.integrate")
    n, t0, dt = 8, 0.7, 0.16
    errs = {}
    for k in (1, 4):
        g = oracle_mod.OracleGrid(dim=2, n=(n, n), velocity="swirl2d", velocity_params=[5.0],
                                  integrator=integrator, substeps=k)

        def rhs(t, x):
            return oracle_mod.velocity_at(g, x, t)[0]

        D = oracle_mod.advect(g, t0, dt)
        worst = 0.0
        for (iy, ix) in [(1, 1), (2, 5), (3, 3), (6, 2)]:
            x0 = np.array([ix / n, iy / n])
            sol = integ.solve_ivp(rhs, (t0, t0 + dt), x0, rtol=1e-13, atol=1e-15, method="DOP853")
            worst = max(worst, float(np.max(np.abs(D[iy, ix] - (sol.y[:, -1] - x0) * n))))
        errs[k] = worst
    assert errs[1] / errs[4] > 0.3 * 4 ** order, errs
