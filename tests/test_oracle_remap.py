"""Pins of the oracle's remap: eq. (multiZ) in the deformed element's logical coordinates,
with the order chosen by the jump criterion (Sec. 2.1-2.3).

The expected values do not come from the oracle: for a uniform shift by delta cells the logical
coordinate of target j is exactly j - delta; for a general displacement it is the closed-form
inverse of the bilinear element map.  Polynomials of degree <= 2m per axis are reproduced
(moment property (b)); integer shifts move the data exactly; mass and low moments are kept.
"""
import numpy as np
import pytest

from paper_1410_2817_gb300 import inputs

from .test_oracle_mapping import _bilinear_inverse


def _poly(deg):
    rng = np.random.default_rng(100 + deg)
    coef = rng.uniform(-1, 1, (deg + 1, deg + 1)) / 10.0 ** np.add.outer(np.arange(deg + 1), np.arange(deg + 1))

    def p(sx, sy):
        return sum(coef[a, b] * sx ** a * sy ** b for a in range(deg + 1) for b in range(deg + 1))
    return p


def _translation_grid(oracle_mod, n, delta, m, threshold=-1.0, nfields=1):
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), nfields=nfields, max_order=m, threshold=threshold)
    D = np.zeros((n, n, 2))
    D[..., 0], D[..., 1] = delta
    return g, D


@pytest.mark.parametrize("m,deg", [(0, 1), (1, 2), (2, 4)])
def test_shift_reproduces_polynomials(oracle_mod, m, deg):
    n, delta = 28, (0.3, -0.45)
    g, D = _translation_grid(oracle_mod, n, delta, m)
    p = _poly(deg)
    ky, kx = np.mgrid[0:n, 0:n].astype(float)
    h = p(kx, ky)
    out = oracle_mod.remap(g, D, np.zeros((n, n), np.uint8), h[None])
    assert out.nfail == 0
    sl = slice(m + 3, n - m - 3)
    expect = p(kx - delta[0], ky - delta[1])
    scale = np.max(np.abs(h))
    assert np.max(np.abs(out.h[0][sl, sl] - expect[sl, sl])) <= 1e-13 * scale
    # one degree more is not reproduced
    q = lambda sx, sy: p(sx, sy) + 1e-3 * sx ** (deg + 1)
    out2 = oracle_mod.remap(g, D, np.zeros((n, n), np.uint8), q(kx, ky)[None])
    assert np.max(np.abs(out2.h[0][sl, sl] - q(kx - delta[0], ky - delta[1])[sl, sl])) > 1e-9


def test_deformed_grid_reproduces_quadratics(oracle_mod):
    """Non-affine displacement: value = p(logical coordinate of the target), the latter from the
    closed-form bilinear inverse of the element found."""
    n = 24
    D = inputs.smooth_displacement((n, n), amplitude=0.3, seed=7, shift=(0.7, -1.4))
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), max_order=1, threshold=-1.0)
    p = _poly(2)
    ky, kx = np.mgrid[0:n, 0:n].astype(float)
    out = oracle_mod.remap(g, D, np.zeros((n, n), np.uint8), p(kx, ky)[None])
    assert out.nfail == 0
    checked = 0
    for jy in range(6, n - 6):
        for jx in range(6, n - 6):
            cw = out.cell[jy, jx]
            cx, cy = cw % n, cw // n
            # unwrap the element near the target
            cx += n * round((jx - 1 - cx) / n)
            cy += n * round((jy - 1 - cy) / n)
            P = []
            for v in range(4):
                kxv, kyv = cx + (v & 1), cy + ((v >> 1) & 1)
                P.append([kxv - jx + D[kyv % n, kxv % n, 0], kyv - jy + D[kyv % n, kxv % n, 1]])
            s = _bilinear_inverse(np.array(P))
            assert abs(out.h[0, jy, jx] - p(cx + s[0], cy + s[1])) <= 1e-12
            checked += 1
    assert checked == (n - 12) ** 2


def test_integer_shift_is_exact_with_limiter(oracle_mod):
    n = 20
    g, D = _translation_grid(oracle_mod, n, (3.0, -2.0), 1, threshold=0.25, nfields=2)
    rng = np.random.default_rng(8)
    h = np.stack([rng.standard_normal((n, n)), (rng.uniform(size=(n, n)) > 0.5).astype(float)])
    out = oracle_mod.remap(g, D, oracle_mod.flags(g, h), h)
    expect = np.roll(np.roll(h, 3, axis=2), -2, axis=1)
    assert np.array_equal(out.h, expect)


def test_shift_preserves_mass_and_moments(oracle_mod):
    """Uniform shift with one order everywhere: sum_j p(X_j) h_new_j = sum_i p(X_i + D) h_i for
    deg p <= 2m (Z1: mass, first and second moments)."""
    n, delta = 64, (0.37, 0.81)
    g, D = _translation_grid(oracle_mod, n, delta, 1)
    ky, kx = np.mgrid[0:n, 0:n].astype(float)
    h = np.exp(-((kx - 30.0) ** 2 + (ky - 33.0) ** 2) / (2 * 3.0 ** 2))  # tails below 1e-20 at the seam
    out = oracle_mod.remap(g, D, np.zeros((n, n), np.uint8), h[None]).h[0]
    for px, py in [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]:
        lhs = np.sum(kx ** px * ky ** py * out)
        rhs = np.sum((kx + delta[0]) ** px * (ky + delta[1]) ** py * h)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs)), (px, py)
    lhs3 = np.sum(kx ** 3 * out)
    rhs3 = np.sum((kx + delta[0]) ** 3 * h)
    assert abs(lhs3 - rhs3) > 1e-6 * abs(rhs3)  # the cubic moment is not kept by Z1


def test_constant_field_stays_constant(oracle_mod):
    n = 32
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), nfields=1, velocity="swirl2d", velocity_params=[5.0])
    D = oracle_mod.advect(g, 0.2, 5.0 / n)
    h = np.full((1, n, n), 2.5)
    out = oracle_mod.remap(g, D, oracle_mod.flags(g, h), h)
    assert out.nfail == 0
    assert np.max(np.abs(out.h - 2.5)) <= 1e-14 * 2.5 * 8


def test_order_follows_flags_near_a_step(oracle_mod):
    """A step along x shifted by a fraction of a cell: elements whose stencil holds a flag use
    linear interpolation, the others the cubic (Hermite) interpolant."""
    from .test_oracle_basis import _hermite_cubic

    n, i0, dx = 32, 16, 0.4
    g, D = _translation_grid(oracle_mod, n, (dx, 0.0), 1, threshold=0.25)
    row = np.where(np.arange(n) >= i0, 1.0, 0.0) + 0.01 * np.arange(n) ** 2 / n
    h = np.tile(row, (n, 1))
    fl = oracle_mod.flags(g, h)
    out = oracle_mod.remap(g, D, fl, h[None])
    for j in range(6, n - 6):
        c = j - 1  # s = j - 0.4 lies in [j - 1, j)
        flagged = [k for k in range(c - 1, c + 3) if fl[5, k % n]]
        m = out.order[0, 5, j]
        assert m == (0 if flagged else 1), j
        s = j - dx
        ref = np.interp(s, np.arange(n), row) if m == 0 else _hermite_cubic(np.concatenate([row, row]), s)
        assert abs(out.h[0, 5, j] - ref) <= 1e-13, j
    assert set(np.nonzero(fl[5])[0].tolist()) >= {i0 - 1, i0}


def test_folded_grid_keeps_values_and_reports(oracle_mod):
    n = 16
    D = np.zeros((n, n, 2))
    D[8, 8] = (-1.6, -1.7)  # node (8, 8) jumps across its lower-left neighbour: elements invert
    g = oracle_mod.OracleGrid(dim=2, n=(n, n), nfields=1, threshold=-1.0)
    rng = np.random.default_rng(9)
    h = rng.standard_normal((1, n, n))
    out = oracle_mod.remap(g, D, np.zeros((n, n), np.uint8), h)
    bad = out.status != oracle_mod.OK
    assert bad.any() and out.nfail == int(bad.sum())
    assert np.array_equal(out.h[0][bad], h[0][bad])
    assert np.all(out.cell[bad] == -1)
    far = np.zeros((n, n), bool)
    far[:4, :] = True
    assert np.all(out.status[far] == oracle_mod.OK)
    assert np.array_equal(out.h[0][far], h[0][far])  # D = 0 there: the identity map


@pytest.mark.parametrize("m,deg", [(1, 2), (2, 4)])
def test_3d_shift_reproduces_polynomials(oracle_mod, m, deg):
    n, delta = 14, (0.25, -0.6, 0.4)
    g = oracle_mod.OracleGrid(dim=3, n=(n, n, n), max_order=m, threshold=-1.0)
    D = np.zeros((n, n, n, 3))
    for a in range(3):
        D[..., a] = delta[a]
    kz, ky, kx = np.mgrid[0:n, 0:n, 0:n].astype(float)
    rng = np.random.default_rng(11)
    cx, cy, cz = rng.uniform(-1, 1, 3) / 10
    p = lambda x, y, z: 0.5 + cx * x ** deg + cy * x * y ** (deg - 1) + cz * z ** deg * y
    out = oracle_mod.remap(g, D, np.zeros((n, n, n), np.uint8), p(kx, ky, kz)[None])
    sl = slice(m + 3, n - m - 3)
    expect = p(kx - delta[0], ky - delta[1], kz - delta[2])
    assert np.max(np.abs(out.h[0][sl, sl, sl] - expect[sl, sl, sl])) <= 1e-12 * np.max(np.abs(expect))


@pytest.mark.parametrize("dim,m", [(2, 0), (2, 1), (2, 2), (3, 1), (3, 2)])
def test_random_affine_grids_reproduce_polynomials(oracle_mod, dim, m):
    """Randomised: under an affine displacement D(X) = b + S X (cell units) the element maps are
    affine, so the logical coordinate of target x is s = (I + S)^-1 (x - b) in closed form, and
    eq. (multiZ) must return p(s) for every p of degree <= 2m per axis (moment property (b)),
    at every order m and on random such grids (targets whose departure point and search stay
    clear of the periodic seam, where an affine D is not periodic)."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies
    n = 20 if dim == 2 else 16
    smax, bmax = (0.15, 2.0) if dim == 2 else (0.08, 1.5)

    @hyp.settings(max_examples=20 if dim == 2 else 8, deadline=None, derandomize=True)
    @hyp.given(b=st.tuples(*[st.floats(-bmax, bmax)] * dim), S=st.tuples(*[st.floats(-smax, smax)] * (dim * dim)),
               seed=st.integers(0, 2 ** 31 - 1))
    def check(b, S, seed):
        A = np.eye(dim) + np.array(S).reshape(dim, dim)
        k = [c.astype(float) for c in reversed(np.mgrid[tuple([slice(0, n)] * dim)])]  # k[0] = x index
        D = np.stack([b[a] + sum((A[a, c] - (a == c)) * k[c] for c in range(dim)) for a in range(dim)], axis=-1)
        deg = max(1, 2 * m)
        coef = np.random.default_rng(seed).uniform(-1, 1, (deg + 1,) * dim)
        coef /= 10.0 ** sum(np.ix_(*[np.arange(deg + 1)] * dim))

        def p(x):
            return sum(cv * np.prod([x[a] ** e[a] for a in range(dim)], axis=0) for e, cv in np.ndenumerate(coef))

        g = oracle_mod.OracleGrid(dim=dim, n=(n,) * dim, max_order=m, threshold=-1.0)
        out = oracle_mod.remap(g, D, np.zeros((n,) * dim, np.uint8), p(k)[None])
        Ai = np.linalg.inv(A)
        sdep = [sum(Ai[a, c] * (k[c] - b[c]) for c in range(dim)) for a in range(dim)]
        lo, hi = m + 3, n - m - 4
        inner = np.ones((n,) * dim, bool)
        for a in range(dim):
            inner &= (sdep[a] >= lo) & (sdep[a] <= hi) & (k[a] >= lo) & (k[a] <= hi)
        hyp.assume(inner.sum() >= 4)
        expect = p(sdep)
        scale = max(1.0, float(np.abs(expect[inner]).max()))
        assert np.all(out.status[inner] == oracle_mod.OK)
        assert np.max(np.abs(out.h[0][inner] - expect[inner])) <= 1e-12 * scale

    check()
