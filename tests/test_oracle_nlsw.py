"""Oracle pins for the shallow-water system (Sec. 3.3, eq. nlsw) on the moving nodes: closed-form
solutions the paper names or that the equations admit -- the equatorial Kelvin wave (eq. kelvin),
a standing gravity wave (linear dispersion omega = kappa), a nonlinear simple wave (Riemann
invariant u - 2 sqrt(1 + h) constant), with viscosity a decaying shear wave and a damped gravity
wave -- each with its convergence rate or bound; the zonal absolute momentum a node keeps on the
beta plane; and the finite differences pinned to the Z-spline derivatives they are defined by."""
import numpy as np
import pytest

F0 = 250.0


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def _kelvin(n, t, amp=1e-4, f0=F0):
    """eq. (kelvin) on [0, 1] x [-0.5, 0.5]: h = u1 = exp(-f0 x2^2 / 2) K(x1 - t), u2 = 0 with
    K(s) = amp exp(-f0 s^2 / 2) (nearest periodic image)."""
    x1 = np.arange(n) / n
    x2 = -0.5 + np.arange(n) / n
    X1, X2 = np.meshgrid(x1, x2)
    s = (X1 - t + 0.5) % 1.0 - 0.5
    h = np.exp(-f0 * X2 ** 2 / 2) * amp * np.exp(-f0 * s ** 2 / 2)
    return np.stack([h, h, np.zeros_like(h)])


def _nlsw_grid(orc, n, max_order, f0=F0, lo=(0.0, -0.5), hi=(1.0, 0.5), nfields=3):
    return orc.OracleGrid(dim=2, n=n, nfields=nfields, lo=lo, hi=hi, velocity="nlsw", velocity_params=[f0],
                          max_order=max_order, threshold=-1.0)


def test_differences_are_the_zspline_derivatives(orc):
    """The lattice derivative is the derivative at a node of the Z-spline interpolant: its weights
    are Z'(k) at the integer offsets (central differences of the oracle's own Z-splines)."""
    eps = 1e-6

    def dz(m, x):
        return float((orc.zspline(m, np.array([x + eps])) - orc.zspline(m, np.array([x - eps])))[0] / (2 * eps))

    # (the second derivative jumps at the knots, so the central difference is good to ~eps)
    assert abs(dz(1, 1.0) + 0.5) < 1e-5 and abs(dz(1, 2.0)) < 1e-5
    assert abs(dz(2, 1.0) + 2.0 / 3.0) < 1e-5 and abs(dz(2, 2.0) - 1.0 / 12.0) < 1e-5 and abs(dz(2, 3.0)) < 1e-5


@pytest.mark.parametrize("max_order,min_rate,max_err", [(2, 3.0, 1e-3), (1, 1.7, 0.08)])
def test_kelvin_wave_converges(orc, max_order, min_rate, max_err):
    """f0 = 250, amplitude 1e-4 (the paper's linear Kelvin test), limiter off, dt = dx / 2, to
    t = 1 (once round the periodic box): relative L2 error of h against eq. (kelvin).  The paper
    reports third order; the quintic's fourth-order differences with the third-order RK3 give
    3.9, the cubic's second-order differences 1.9."""
    errs = []
    for n in (64, 128):
        steps = 2 * n
        out, nfail = _run(orc, _nlsw_grid(orc, (n, n), max_order), _kelvin(n, 0.0), 1.0 / steps, steps)
        assert nfail == 0
        ex = _kelvin(n, 1.0)
        errs.append(float(np.sqrt(((out[0] - ex[0]) ** 2).sum() / (ex[0] ** 2).sum())))
    assert np.log2(errs[0] / errs[1]) >= min_rate, errs
    assert errs[1] <= max_err, errs


def _run(orc, g, h, dt, steps):
    return orc.step(g, h, 0.0, dt, steps)


def test_standing_gravity_wave(orc):
    """f0 = 0, 1-D: h = A cos(2 pi k x), u = 0 oscillates as h = A cos(2 pi k x) cos(2 pi k t),
    u = A sin(2 pi k x) sin(2 pi k t) (linear dispersion omega = kappa, unit wave speed); A = 1e-4,
    so the nonlinear terms leave a relative 1e-4."""
    n, kap, amp, T = 64, 2, 1e-4, 0.3
    steps = int(round(T / (0.5 / n)))
    x = np.arange(n) / n
    h0 = np.tile(amp * np.cos(2 * np.pi * kap * x), (4, 1))
    g = _nlsw_grid(orc, (n, 4), 2, f0=0.0, lo=(0.0, 0.0), hi=(1.0, 1.0))
    out, _ = _run(orc, g, np.stack([h0, np.zeros_like(h0), np.zeros_like(h0)]), T / steps, steps)
    he = amp * np.cos(2 * np.pi * kap * x) * np.cos(2 * np.pi * kap * T)
    ue = amp * np.sin(2 * np.pi * kap * x) * np.sin(2 * np.pi * kap * T)
    assert np.abs(out[0] - he[None]).max() <= 1e-3 * amp
    assert np.abs(out[1] - ue[None]).max() <= 1e-3 * amp
    assert np.abs(out[2]).max() == 0.0


def _simple_wave(x, t, amp):
    """Right-moving simple wave of the 1-D system (f = 0): c = sqrt(1 + h) is constant along
    dx/dt = 3c - 2 when u = 2 (c - 1) initially; h = c^2 - 1, u = 2 (c - 1) at the foot s of the
    characteristic through x (Newton on s + (3 c0(s) - 2) t = x)."""
    def c0(s):
        return np.sqrt(1 + amp * np.sin(2 * np.pi * s))

    def dc0(s):
        return amp * np.pi * np.cos(2 * np.pi * s) / c0(s)

    s = x - t
    for _ in range(80):
        s = s - (s + (3 * c0(s) - 2) * t - x) / (1 + 3 * dc0(s) * t)
    c = c0(s)
    return c * c - 1, 2 * (c - 1)


@pytest.mark.parametrize("max_order,min_rate,max_err", [(2, 2.5, 1e-6), (1, 1.8, 3e-4)])
def test_nonlinear_simple_wave(orc, max_order, min_rate, max_err):
    """h0 = 0.05 sin(2 pi x) (+1 inside the square root), u0 = 2 (sqrt(1 + h0) - 1), f0 = 0, to
    t = 0.5 (the wave breaks near t = 2.1): the nonlinear factor (1 + h), the node motion and the
    chain rule through the moving nodes all enter.  Max error of h and u against the
    characteristics; measured rates 2.9 (Z2) and 2.0 (Z1)."""
    amp, T = 0.05, 0.5
    errs = []
    for n in (64, 128):
        steps = int(round(T / (0.5 / n)))
        x = np.arange(n) / n
        c0 = np.sqrt(1 + amp * np.sin(2 * np.pi * x))
        h0, u0 = np.tile(c0 ** 2 - 1, (4, 1)), np.tile(2 * (c0 - 1), (4, 1))
        g = _nlsw_grid(orc, (n, 4), max_order, f0=0.0, lo=(0.0, 0.0), hi=(1.0, 1.0))
        out, nfail = _run(orc, g, np.stack([h0, u0, np.zeros_like(h0)]), T / steps, steps)
        assert nfail == 0 and np.abs(out[2]).max() == 0.0
        he, ue = _simple_wave(x, T, amp)
        errs.append(max(float(np.abs(out[0] - he[None]).max()), float(np.abs(out[1] - ue[None]).max())))
    assert np.log2(errs[0] / errs[1]) >= min_rate, errs
    assert errs[1] <= max_err, errs


def test_uniform_stream_moves_a_tracer_like_the_uniform_flow(orc):
    """h = 0, u = (0.3, -0.2) everywhere, f0 = 0: every source vanishes, the nodes translate, and a
    passive fourth field moves exactly as under the uniform velocity; the rest state stays at rest."""
    n = (32, 24)
    rng = np.random.default_rng(8)
    tracer = rng.uniform(size=(24, 32))
    h = np.stack([np.zeros((24, 32)), np.full((24, 32), 0.3), np.full((24, 32), -0.2), tracer])
    g = _nlsw_grid(orc, n, 1, f0=0.0, lo=(0.0, 0.0), hi=(1.0, 1.0), nfields=4)
    out, _ = _run(orc, g, h, 0.04, 3)
    gu = orc.OracleGrid(dim=2, n=n, nfields=1, velocity="uniform", velocity_params=[0.3, -0.2], max_order=1,
                        threshold=-1.0)
    ref, _ = orc.step(gu, tracer[None], 0.0, 0.04, 3)
    assert np.abs(out[3] - ref[0]).max() <= 1e-13
    assert np.abs(out[0]).max() <= 1e-15 and np.abs(out[1] - 0.3).max() <= 1e-15
    rest, _ = _run(orc, _nlsw_grid(orc, (16, 16), 2), np.zeros((3, 16, 16)), 0.01, 4)
    assert np.abs(rest).max() == 0.0


@pytest.mark.parametrize("orient", ["u1_of_x2", "u2_of_x1"])
@pytest.mark.parametrize("max_order,min_rate,max_err", [(2, 3.5, 3e-6), (1, 1.8, 1e-3)])
def test_viscous_shear_decays(orc, orient, max_order, min_rate, max_err):
    """nu = 0.01, h = 0, f0 = 0, a shear wave u1 = A sin(2 pi x2) (or u2 = A sin(2 pi x1)): the
    advection and pressure terms vanish and the wave decays as exp(-nu (2 pi)^2 t) (eq. nlsw's
    viscous term reduces to nu times the Laplacian); rates measured 4.0 (Z2) and 2.0 (Z1)."""
    nu, amp, T = 0.01, 0.05, 0.5
    errs = []
    for n in (32, 64):
        steps = int(round(T / (0.5 / n)))
        x = np.arange(n) / n
        X1, X2 = np.meshgrid(x, x)
        prof = amp * np.sin(2 * np.pi * (X2 if orient == "u1_of_x2" else X1))
        u, v = (prof, np.zeros_like(prof)) if orient == "u1_of_x2" else (np.zeros_like(prof), prof)
        g = orc.OracleGrid(dim=2, n=(n, n), nfields=3, velocity="nlsw", velocity_params=[0.0, nu],
                           max_order=max_order, threshold=-1.0)
        out, nfail = _run(orc, g, np.stack([np.zeros_like(u), u, v]), T / steps, steps)
        assert nfail == 0 and np.abs(out[0]).max() == 0.0
        comp = out[1] if orient == "u1_of_x2" else out[2]
        errs.append(float(np.abs(comp - np.exp(-nu * (2 * np.pi) ** 2 * T) * prof).max()) / amp)
    assert np.log2(errs[0] / errs[1]) >= min_rate, errs
    assert errs[1] <= max_err, errs


def test_viscous_damped_gravity_wave(orc):
    """f0 = 0, nu = 0.01, 1-D standing wave h = A cos(k x), u = 0 (A = 1e-4): the linearised
    system h_t = -u_x, u_t = -h_x + 2 nu u_xx (the stress's normal component carries the factor
    2) gives h = A cos(k x) exp(-a t) (cos w t + a / w sin w t), a = nu k^2, w^2 = k^2 - a^2.
    Without the factor 2 the error would be ~0.1 A."""
    n, kap, amp, nu, T = 64, 4 * np.pi, 1e-4, 0.01, 0.3
    steps = int(round(T / (0.5 / n)))
    x = np.arange(n) / n
    h0 = np.tile(amp * np.cos(kap * x), (4, 1))
    g = orc.OracleGrid(dim=2, n=(n, 4), nfields=3, velocity="nlsw", velocity_params=[0.0, nu], max_order=2,
                       threshold=-1.0)
    out, _ = _run(orc, g, np.stack([h0, np.zeros_like(h0), np.zeros_like(h0)]), T / steps, steps)
    a = nu * kap ** 2
    w = np.sqrt(kap ** 2 - a ** 2)
    H = amp * np.exp(-a * T) * (np.cos(w * T) + a / w * np.sin(w * T))
    assert np.abs(out[0] - H * np.cos(kap * x)[None]).max() <= 2e-4 * amp


def test_zonal_absolute_momentum_on_the_beta_plane(orc):
    """Reading of eq. (nlsw): the Coriolis parameter f = f0 x2 is taken at the node's current
    position.  For fields independent of x1 there is no zonal pressure force, so each node keeps
    its absolute momentum u1 - f0 x2^2 / 2; while h stays O(dt^3) (one step from rest in h with a
    uniform meridional stream V) a node follows x2' = u2, u1' = f0 x2 u2, u2' = -f0 x2 u1.  The
    oracle's step against that ODE solved tightly and traced back from every target; f taken at
    the node's starting position instead would shift u1 by f0 (V dt)^2 / 2 = 5.6e-4."""
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    brentq = pytest.importorskip("scipy.optimize").brentq
    f0, V, ny, dt = 5.0, 0.3, 32, 0.05
    g = _nlsw_grid(orc, (4, ny), 1, f0=f0)
    h = np.zeros((3, ny, 4))
    h[2] = V
    out, nfail = _run(orc, g, h, dt, 1)
    assert nfail == 0

    def node(y0):
        r = solve_ivp(lambda t, s: [s[2], f0 * s[0] * s[2], -f0 * s[0] * s[1]], (0.0, dt), [y0, 0.0, V],
                      rtol=1e-13, atol=1e-15)
        return r.y[:, -1]

    y = -0.5 + np.arange(ny) / ny
    # away from the periodic seam, where f = f0 x2 jumps from +f0/2 to -f0/2
    for j in np.nonzero(np.abs(y) < 0.3)[0]:
        y0 = brentq(lambda a: node(a)[0] - y[j], y[j] - 0.1, y[j] + 0.1, xtol=1e-15)
        _, ue, ve = node(y0)
        assert np.abs(out[1][j] - ue).max() <= 5e-6, (y[j], out[1][j], ue)
        assert np.abs(out[2][j] - ve).max() <= 5e-6, (y[j], out[2][j], ve)
        assert np.abs(out[:, j] - out[:, j, :1]).max() == 0.0  # still independent of x1
