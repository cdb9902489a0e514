"""Pins of the oracle's element map inversion and element search (Sec. 2.2, eq. mapping1).

* 2-D: Newton's answer equals the closed-form inverse of the bilinear map (a quadratic).
* 3-D: it equals an independent root finder (scipy) and leaves a residual at rounding level.
* Affine elements are solved by the linear initial guess (one Newton step leaves them unchanged).
* Element search: on tiny grids with smooth non-folding displacements, the element found is the
  one that a brute-force scan of every element identifies as containing the target.
"""
import itertools

import numpy as np
import pytest

from paper_1410_2817_gb300 import inputs


def _bilinear_inverse(P):
    """Closed form: P00 + s a + t b + s t e = 0 with a = P10-P00, b = P01-P00, e = P11-P10-P01+P00.
    Crossing with (b + s e) removes t: (P00 + s a) x (b + s e) = 0, a quadratic in s."""
    P00, P10, P01, P11 = P[0], P[1], P[2], P[3]
    a, b, e = P10 - P00, P01 - P00, P11 - P10 - P01 + P00
    cross = lambda u, v: u[0] * v[1] - u[1] * v[0]
    A2, A1, A0 = cross(a, e), cross(P00, e) + cross(a, b), cross(P00, b)
    if abs(A2) < 1e-14 * max(1.0, abs(A1)):
        roots = [-A0 / A1]
    else:
        disc = np.sqrt(A1 * A1 - 4 * A2 * A0)
        q = -0.5 * (A1 + np.copysign(disc, A1))
        roots = [q / A2, A0 / q]
    best = None
    for s in roots:
        v = b + s * e
        t = -np.dot(P00 + s * a, v) / np.dot(v, v)
        cand = np.array([s, t])
        if best is None or np.max(np.abs(cand - 0.5)) < np.max(np.abs(best - 0.5)):
            best = cand
    return best


def _random_cell(rng, d, distortion):
    """Vertices of a distorted unit cell containing the origin, relative to the target."""
    target = rng.uniform(0.05, 0.95, d)
    P = []
    for v in range(1 << d):
        corner = np.array([(v >> a) & 1 for a in range(d)], dtype=float)
        P.append(corner + rng.uniform(-distortion, distortion, d) - target)
    return np.array(P)


def test_newton_matches_closed_form_2d(oracle_mod):
    rng = np.random.default_rng(10)
    checked, its = 0, []
    for _ in range(400):
        P = _random_cell(rng, 2, 0.3)
        xi, st, it = oracle_mod.newton(P)
        if st != oracle_mod.OK:
            continue
        ref = _bilinear_inverse(P)
        assert np.max(np.abs(xi - ref)) <= 1e-12
        its.append(it)
        checked += 1
    assert checked > 350
    assert np.mean(its) <= 4.5  # quadratic convergence from the linear guess


def test_newton_matches_scipy_3d(oracle_mod):
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(11)

    def trilinear(xi, P):
        out = np.zeros(3)
        for v in range(8):
            w = 1.0
            for a in range(3):
                w *= xi[a] if (v >> a) & 1 else 1.0 - xi[a]
            out += w * P[v]
        return out

    for _ in range(100):
        P = _random_cell(rng, 3, 0.2)
        xi, st, it = oracle_mod.newton(P)
        assert st == oracle_mod.OK
        ref = scipy_opt.fsolve(trilinear, np.full(3, 0.5), args=(P,), xtol=1e-13)
        assert np.max(np.abs(xi - ref)) <= 1e-11
        assert np.max(np.abs(trilinear(xi, P))) <= 1e-13


@pytest.mark.parametrize("d", (2, 3))
def test_affine_cell_solved_by_linear_guess(oracle_mod, d):
    rng = np.random.default_rng(12)
    A = np.eye(d) + rng.uniform(-0.3, 0.3, (d, d))
    b = rng.uniform(-2, 2, d)
    P = np.array([A @ np.array([(v >> a) & 1 for a in range(d)], dtype=float) + b for v in range(1 << d)])
    xi, st, it = oracle_mod.newton(P)
    assert st == oracle_mod.OK and it == 1
    assert np.max(np.abs(xi - np.linalg.solve(A, -b))) <= 1e-13


def test_folded_cell_reports_fold(oracle_mod):
    P = np.array([[0.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [-1.0, 1.0]]) - 0.3  # mirrored: det < 0
    xi, st, _ = oracle_mod.newton(P)
    assert st == oracle_mod.FOLD


def _brute_force_cells(oracle_mod, g, D, j, R):
    """All elements (unwrapped lower corners c within R of j) whose bilinear/trilinear image
    contains target j, checked with an independent inverse."""
    d = g.dim
    n = np.array(g.n[:d])
    found = []
    for off in itertools.product(range(-R, R + 1), repeat=d):
        c = np.array(j) + np.array(off)
        P = []
        for v in range(1 << d):
            k = c + np.array([(v >> a) & 1 for a in range(d)])
            kw = tuple(int(x) for x in np.mod(k, n))
            P.append(k - np.array(j) + D[kw[::-1]])
        P = np.array(P)
        # x(xi) on the unit cell is a convex combination of the vertices: skip elements whose
        # vertex bounding box misses the target
        if np.any(P.min(axis=0) > 1e-9) or np.any(P.max(axis=0) < -1e-9):
            continue
        if d == 2:
            xi = _bilinear_inverse(P)
        else:
            import scipy.optimize as so

            def f(x):
                out = np.zeros(3)
                for v in range(8):
                    w = 1.0
                    for a in range(3):
                        w *= x[a] if (v >> a) & 1 else 1.0 - x[a]
                    out += w * P[v]
                return out
            xi = so.fsolve(f, np.full(3, 0.5), xtol=1e-13)
            if np.max(np.abs(f(xi))) > 1e-10:
                continue
        if np.all(xi >= -1e-9) and np.all(xi <= 1 + 1e-9):
            found.append((tuple(np.mod(c, n)), xi, np.min(np.minimum(np.abs(xi), np.abs(1 - xi)))))
    return found


@pytest.mark.parametrize("d,n,shift,start", [(2, 12, (1.3, -2.6), 0), (2, 12, (1.3, -2.6), 1),
                                              (2, 10, (-0.4, 0.7), 0), (3, 6, (0.6, -1.2, 0.3), 0)])
def test_locate_matches_brute_force(oracle_mod, d, n, shift, start):
    D = inputs.smooth_displacement((n,) * d, amplitude=0.35, seed=20 + d, shift=shift)
    g = oracle_mod.OracleGrid(dim=d, n=(n,) * d, start=start)
    R = int(np.ceil(np.max(np.abs(D)))) + 2
    for j in itertools.product(range(n), repeat=d):
        c, xi, st, hops, _ = oracle_mod.locate(g, D, j)
        assert st == oracle_mod.OK
        cw = tuple(int(x) for x in np.mod(c, n))
        found = _brute_force_cells(oracle_mod, g, D, j, R)
        assert found, j
        interior = [f for f in found if f[2] > 1e-7]
        if len(found) == 1 or interior:
            # the containing element is unique away from faces
            assert len(interior) == 1 and cw == interior[0][0], (j, cw, found)
            assert np.max(np.abs(xi - interior[0][1])) <= 1e-9
        else:
            assert cw in [f[0] for f in found]


def test_paper_start_walk_length_tracks_cfl(oracle_mod):
    """From the element next to node j the walk needs about |D| hops (one neighbour per hop)."""
    n = 16
    D = np.zeros((n, n, 2))
    D[..., 0] = 5.5
    g = oracle_mod.OracleGrid(dim=2, n=(n, n))
    c, xi, st, hops, _ = oracle_mod.locate(g, D, (7, 7))
    assert st == oracle_mod.OK and tuple(c) == (1, 7) and hops == 6
    np.testing.assert_allclose(xi, [0.5, 0.0], atol=1e-15)
    gb = oracle_mod.OracleGrid(dim=2, n=(n, n), start=oracle_mod.START_BACKWARD)
    c2, xi2, st2, hops2, _ = oracle_mod.locate(gb, D, (7, 7))
    assert st2 == oracle_mod.OK and tuple(c2) == (1, 7) and hops2 == 1


def test_walk_gives_up(oracle_mod):
    n = 16
    D = np.zeros((n, n, 2))
    D[..., 0] = 7.5
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), walk_max=3)
    _, _, st, hops, _ = oracle_mod.locate(g, D, (7, 7))
    assert st == oracle_mod.LOCATE and hops == 3


def _replay_walk(oracle_mod, g, D, j, c0, walk_max):
    """The walk of Sec. 2.2 replayed step by step with no revisit rule: invert in the current
    element and step one element along every axis whose local coordinate is out of range.
    Returns (status, hops, elements tried)."""
    d = g.dim
    n = np.array(g.n[:d])
    c = np.array(c0, dtype=np.int64)
    tried = []
    for hop in range(walk_max):
        P = []
        for v in range(1 << d):
            k = c + np.array([(v >> a) & 1 for a in range(d)])
            kw = tuple(int(x) for x in np.mod(k, n))
            P.append(k - np.array(j) + D[kw[::-1]])
        xi, st, _ = oracle_mod.newton(np.array(P))
        tried.append(tuple(int(x) for x in c))
        if not np.all(np.isfinite(xi)):
            return ("newton" if st == oracle_mod.OK else st), hop + 1, tried
        if np.all(xi >= -1e-12) and np.all(xi <= 1 + 1e-12):
            return st, hop + 1, tried
        c = c + np.where(xi < -1e-12, -1, 0) + np.where(xi > 1 + 1e-12, 1, 0)
    return oracle_mod.LOCATE, walk_max, tried


def test_walk_stops_on_a_revisit(oracle_mod):
    """Sec. 2.2: the next element depends on the current one alone, so a walk that comes back to
    an element it has tried would cycle until walk_max.  The oracle gives up at the first repeat
    (Brent's test).  On the 64x64 solid-body rotation, whose elements sheared across the seam
    make walks fail, every target's status equals that of the walk replayed without the rule for
    the full 64 hops; every failure is such a cycle and is found within a few hops; and the
    targets that succeed take exactly the replay's hops."""
    wl = inputs.workload_sbr64()
    g = oracle_mod.OracleGrid(dim=2, n=wl.n, nfields=1, velocity=wl.velocity, velocity_params=wl.velocity_params)
    D = oracle_mod.advect(g, 0.0, wl.dt)
    nfail = 0
    for jy in range(wl.n[1]):
        for jx in range(wl.n[0]):
            j = (jx, jy)
            c0 = (jx - (1 if D[jy, jx, 0] > 0 else 0), jy - (1 if D[jy, jx, 1] > 0 else 0))
            c, xi, st, hops, _ = oracle_mod.locate(g, D, j)
            rst, rhops, tried = _replay_walk(oracle_mod, g, D, j, c0, 64)
            assert st == rst, (j, st, rst)
            if st == oracle_mod.LOCATE:
                nfail += 1
                assert len(set(tried)) < len(tried), j  # the replayed walk revisits an element
                first_repeat = next(k for k in range(len(tried)) if tried[k] in tried[:k])
                assert hops <= 3 * first_repeat + 2 and hops < 64, (j, hops, first_repeat)
            else:
                assert hops == rhops, (j, hops, rhops)
    assert nfail > 0
