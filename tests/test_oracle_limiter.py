"""Pins of the oracle's jump criterion and order reduction (Sec. 2.3, Fig. 2 caption).

Expected flags and orders are derived by hand from the criterion
|h+ - 2h + h-| / max(|h+ - h|, |h - h-|) > 0.25 and from the rule "reduce the order while a flag
lies among the points the interpolation needs, down to linear".
"""
import numpy as np
import pytest


def _grid(oracle_mod, n, nfields=1, max_order=1, threshold=0.25, dim=2):
    return oracle_mod.OracleGrid(dim=dim, n=(n,) * dim, nfields=nfields, max_order=max_order, threshold=threshold)


def test_step_flags_both_sides_only(oracle_mod):
    n = 16
    g = _grid(oracle_mod, n)
    h = np.zeros((n, n))
    h[:, 6:11] = 1.0  # jumps between x = 5|6 and 10|11, constant along y
    fl = oracle_mod.flags(g, h)
    flagged_x = sorted(set(np.nonzero(fl)[1].tolist()))
    assert flagged_x == [5, 6, 10, 11]
    assert np.all(fl[:, [5, 6, 10, 11]] == 1)


def test_flat_and_linear_never_flagged(oracle_mod):
    n = 16
    g = _grid(oracle_mod, n)
    assert not oracle_mod.flags(g, np.full((n, n), 3.5)).any()  # 0/0 is not a jump
    x = np.arange(n, dtype=float)
    lin = np.tile(0.25 * x, (n, 1))  # linear in x (wraps at the periodic seam)
    fl = oracle_mod.flags(g, lin)
    assert not fl[:, 1:-1].any()
    assert fl[:, 0].all() and fl[:, -1].all()  # the periodic wrap is a jump


def test_smooth_extremum_is_flagged(oracle_mod):
    """At a smooth extremum the two one-sided slopes have opposite signs, so the ratio is about 2:
    the literal criterion flags it (faithful to the paper's statement)."""
    n = 32
    g = _grid(oracle_mod, n)
    x = np.arange(n, dtype=float)
    h = np.tile(np.sin(2 * np.pi * x / n), (n, 1))
    fl = oracle_mod.flags(g, h)[0]
    assert fl[8] == 1 and fl[24] == 1        # the maximum and the minimum of the sine
    assert fl[4] == 0 and fl[12] == 0         # the steep parts are smooth


def test_threshold_is_strict(oracle_mod):
    g = _grid(oracle_mod, 8)
    h = np.zeros((8, 8))
    # node x=3: h- = 0, h = 4, h+ = 7: slopes 4 and 3; |3 - 4| = 1 = 0.25 * 4 -> not flagged
    h[:, 3], h[:, 4], h[:, 5], h[:, 6], h[:, 7] = 4.0, 7.0, 10.0, 13.0, 16.0
    h[:, 0:3] = [[-8.0, -4.0, 0.0]] * 8
    fl = oracle_mod.flags(g, h)[0]
    assert fl[3] == 0
    h2 = h.copy()
    h2[:, 4] = 6.99  # |2.99 - 4| = 1.01 > 1 -> flagged
    assert oracle_mod.flags(g, h2)[0][3] == 1
    # a different threshold moves the decision
    g3 = _grid(oracle_mod, 8, threshold=0.5)
    assert oracle_mod.flags(g3, h2)[0][3] == 0


def test_disabled_limiter_and_per_field_bits(oracle_mod):
    n = 12
    g = _grid(oracle_mod, n, nfields=3)
    h = np.zeros((3, n, n))
    h[0, :, 4:] = 1.0       # field 0: jump along x
    h[2, 7:, :] = 1.0       # field 2: jump along y
    fl = oracle_mod.flags(g, h)
    bit0_x = sorted(set(np.nonzero(fl & 1)[1].tolist()))
    bit2_y = sorted(set(np.nonzero(fl & 4)[0].tolist()))
    assert bit0_x == [0, 3, 4, 11]          # x = 3|4 and the periodic wrap 11|0
    assert bit2_y == [0, 6, 7, 11]          # y = 6|7 and the periodic wrap
    assert np.all(fl[:, 3] & 1) and np.all(fl[7, :] & 4)
    assert not (fl & 2).any()  # field 1 is flat
    assert fl[6, 3] == 5 and fl[5, 5] == 0
    assert not oracle_mod.flags(_grid(oracle_mod, n, nfields=3, threshold=-1.0), h).any()


def test_flags_3d_axes(oracle_mod):
    n = 8
    g = _grid(oracle_mod, n, dim=3)
    h = np.zeros((n, n, n))
    h[3:, :, :] = 1.0  # jump along z only
    fl = oracle_mod.flags(g, h)
    assert fl[2].all() and fl[3].all() and not fl[4:7].any() and not fl[1].any()


@pytest.mark.parametrize("max_order,expect", [
    (1, {5: 1, 6: 1, 7: 1, 8: 0, 9: 0, 10: 0, 11: 0, 12: 1, 13: 1, 14: 1}),
    (2, {5: 2, 6: 2, 7: 1, 8: 0, 9: 0, 10: 0, 11: 0, 12: 1, 13: 2, 14: 2}),
])
def test_order_pattern_single_flag(oracle_mod, max_order, expect):
    """One flagged node at x = 10.  Element c needs nodes [c-m, c+m+1]: order m survives only if
    the flag is outside that range, so Z1 drops to linear for c in 8..11 and Z2 additionally
    uses the cubic in c = 7 and c = 12 (Fig. 2: quintic far away, cubic near, linear at the jump)."""
    n = 24
    g = _grid(oracle_mod, n, max_order=max_order)
    fl = np.zeros((n, n), dtype=np.uint8)
    fl[:, 10] = 1
    for c, m in expect.items():
        assert oracle_mod.order(g, fl, (c, 12), 0) == m, c


def test_order_isotropic_2d_box(oracle_mod):
    n = 24
    g = _grid(oracle_mod, n, max_order=1)
    fl = np.zeros((n, n), dtype=np.uint8)
    fl[12, 10] = 1  # (y=12, x=10)
    for cy in range(8, 16):
        for cx in range(6, 14):
            inside = (cx - 1 <= 10 <= cx + 2) and (cy - 1 <= 12 <= cy + 2)
            assert oracle_mod.order(g, fl, (cx, cy), 0) == (0 if inside else 1)
    fl2 = np.zeros((n, n), dtype=np.uint8)
    fl2[12, 10] = 2  # flag of field 1 does not lower field 0
    assert oracle_mod.order(g, fl2, (10, 12), 0) == 1
    assert oracle_mod.order(g, fl2, (10, 12), 1) == 0
    # periodic wrap of the stencil: element at x = n-1 needs x = 0
    fl3 = np.zeros((n, n), dtype=np.uint8)
    fl3[5, 0] = 1
    assert oracle_mod.order(g, fl3, (n - 1, 5), 0) == 0
    assert oracle_mod.order(g, fl3, (n - 4, 5), 0) == 1
