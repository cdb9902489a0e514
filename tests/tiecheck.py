"""Target-by-target comparison of the CUDA path with the oracle, with ties classified.

A target's value may legitimately differ from the oracle's only where the method's own decisions
are not unique (Sec. 2.2, 2.3):

* face tie -- the target lies on (within rounding of) a face shared by two elements, so either
  element is a correct result of the element search; the value is then the interpolation in the
  element the GPU chose;
* limiter tie -- a node of the stencil has |h+ - 2h + h-| within rounding of the threshold times
  max(|h+ - h|, |h - h-|), so either jump flag is a correct result of the criterion; the value is
  then the interpolation with the other order.

Everything else must agree within the stated tolerance.  The helpers return how many targets
took each route; a target that matches no allowed candidate fails the calling test.
"""
from __future__ import annotations

import itertools

import numpy as np
import torch

FACE_TIE_F64 = 1e-9
FACE_TIE_F32 = 2e-5   # the FP32 kernels accept a target within 1e-5 of a face, plus Newton's error
LIMITER_TIE_F32 = 1e-6


def _coords(jj_flat, shape):
    """(x, y[, z]) of a flat target index in a plane of `shape` (z, y, x order)."""
    idx = np.unravel_index(int(jj_flat), shape)
    return tuple(int(v) for v in reversed(idx))


def _unwrap_cell(cell_wrapped, j, n):
    """Unwrapped lower corner of a wrapped element index, placed next to target j."""
    c, rem = [], int(cell_wrapped)
    for a in range(len(n)):
        c.append(rem % n[a])
        rem //= n[a]
    return [ci + n[a] * round((j[a] - ci) / n[a]) for a, ci in enumerate(c)]


def f64_step_ties(orc, og, g, F, t, dt, velocity_from_fields=False, tol=1e-12):
    """One FP64 step on the GPU (sl_step, one step) and in the oracle from the same fields F.

    Both sides integrate their own trajectories (the GPU's sincospi and the oracle's sin differ in
    the last bits), so a target may differ by more than `tol` (normwise) only at a face tie.  The
    jump flags come from the same fields on both sides and must agree bit for bit, so no limiter
    tie can arise.  For every target beyond `tol` the GPU's element (from sl_remap_fields_debug
    with the GPU's own displacement, whose output must equal the step's bit for bit) must differ
    from the oracle's, the oracle's coordinates must lie within 1e-9 of a face, the GPU's element
    must contain the target (the oracle's Newton in it lands within 1e-9 of [0, 1]^d) and the GPU's
    value must equal the oracle's interpolation in the GPU's element and order within `tol`.

    Returns (GPU fields after the step as float64 numpy, targets beyond tol, face ties)."""
    F = np.asarray(F, dtype=np.float64)
    fl = orc.flags(og, F)
    D = orc.advect_carried(og, F, dt) if velocity_from_fields else orc.advect(og, t, dt)
    ref = orc.remap(og, D, fl, F)
    ref_step, _ = orc.step(og, F, t, dt, 1)
    assert np.array_equal(ref_step, ref.h), "the oracle's step is not its stage functions composed"
    f = torch.tensor(F, dtype=torch.float64, device="cuda")
    g.step(f, torch.empty_like(f), t, dt, 1)
    torch.cuda.synchronize()
    got = f.cpu().numpy()
    assert np.array_equal(g.flags(torch.tensor(F, device="cuda")).cpu().numpy(), fl), "jump flags differ"
    if velocity_from_fields:
        g.advect_carried(torch.tensor(F, device="cuda"), dt)
    hin = torch.tensor(F, device="cuda")
    hout = torch.empty_like(hin)
    cell, xi, order, status = g.remap_debug(hin, hout)
    torch.cuda.synchronize()
    assert np.array_equal(hout.cpu().numpy(), got), "the debug remap is not the step's remap"
    cell, order, status = cell.cpu().numpy(), order.cpu().numpy(), status.cpu().numpy()
    assert np.array_equal(status, ref.status), f"status differs at {np.argwhere(status != ref.status)[:5].tolist()}"
    ok = ref.status == orc.OK
    assert np.array_equal(got[:, ~ok], F[:, ~ok]), "a failed target did not keep its value"
    scale = max(1e-300, float(np.abs(ref.h).max()))
    err = np.abs(got - ref.h).max(axis=0)
    beyond = np.flatnonzero(err.ravel() > tol * scale)
    n = og.n[: og.dim]
    shape = ref.status.shape
    ties = 0
    for jj in beyond:
        j = _coords(jj, shape)
        idx = np.unravel_index(int(jj), shape)
        why = f"target {j}: err {err[idx]:.3e} (scale {scale:.3e})"
        assert cell[idx] != ref.cell[idx], why + ": same element, value differs"
        rxi = ref.xi[idx]
        assert np.min(np.minimum(np.abs(rxi), np.abs(1.0 - rxi))) < FACE_TIE_F64, why + f": not on a face (xi {rxi})"
        c = _unwrap_cell(cell[idx], j, n)
        vals, xe, oe, st = orc.eval_in_element(og, D, fl, F, j, c)
        assert st == orc.OK and np.all(xe >= -FACE_TIE_F64) and np.all(xe <= 1 + FACE_TIE_F64), \
            why + f": the GPU's element {c} does not contain it (xi {xe})"
        assert np.array_equal(oe, order[(slice(None),) + idx]), why + ": order in the GPU's element differs"
        assert np.max(np.abs(got[(slice(None),) + idx] - vals)) <= tol * scale, why + ": value in the GPU's element"
        ties += 1
    return got, int(beyond.size), ties


def _limiter_bounds(h, thr, margin):
    """Per node and field: flagged for certain, and possibly flagged, when the jump test is taken
    in FP32 (its differences carry relative rounding of 2^-24 each).  Bit masks like the flags."""
    nf = h.shape[0]
    sure = np.zeros(h.shape[1:], dtype=np.uint8)
    maybe = np.zeros(h.shape[1:], dtype=np.uint8)
    for f in range(nf):
        s_f = np.zeros(h.shape[1:], dtype=bool)
        m_f = np.zeros(h.shape[1:], dtype=bool)
        for ax in range(h.ndim - 1):
            hp = np.roll(h[f], -1, axis=ax)
            hm = np.roll(h[f], 1, axis=ax)
            dp, dm = hp - h[f], h[f] - hm
            c = np.abs(dp - dm)
            q = thr * np.maximum(np.abs(dp), np.abs(dm))
            mg = margin * (np.abs(dp) + np.abs(dm))
            s_f |= c > q + mg
            m_f |= c > q - mg
        sure |= (s_f.astype(np.uint8) << f)
        maybe |= (m_f.astype(np.uint8) << f)
    return sure, maybe


def f32_remap_targets(orc, og, D, h, got, tol, thr=0.25):
    """Every target of an FP32 remap (GPU values `got`, computed from the FP32 displacement D and
    FP32 fields h, both given to the oracle as they are) against the FP64 oracle.

    A target passes when each field's value is within `tol` of the oracle's interpolation in
    either the oracle's element or, when the oracle's coordinates lie within 2e-5 of a face, a
    neighbouring element across that face, with an order allowed by the FP32 limiter: between the
    order of the flags that hold for certain and that of the flags that may hold, given the
    rounding of the FP32 jump test.  Targets whose search fails in the oracle must keep their
    values.  Returns {"primary", "limiter_ties", "face_ties", "oracle_failed"} counts.
    """
    D = np.asarray(D, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    fl = orc.flags(og, h)
    ref = orc.remap(og, D, fl, h)
    # where the oracle's search or inversion fails the target keeps its value on both sides
    failed = ref.status != orc.OK
    assert np.array_equal(got[:, failed], h[:, failed]), "the GPU interpolated a target the oracle fails"
    nf = og.nfields
    scale = max(1.0, float(np.abs(h).max()))
    err = np.abs(got - ref.h)
    bad = np.flatnonzero(((err > tol * scale).any(axis=0) & ~failed).ravel())
    counts = {"primary": int((~failed).sum() - bad.size), "limiter_ties": 0, "face_ties": 0,
              "oracle_failed": int(failed.sum())}
    if bad.size == 0:
        return counts
    sure, maybe = _limiter_bounds(h, thr, LIMITER_TIE_F32) if thr >= 0 else (fl * 0, fl * 0)
    n = og.n[: og.dim]
    shape = ref.status.shape
    for jj in bad:
        j = _coords(jj, shape)
        idx = np.unravel_index(int(jj), shape)
        c0 = list(_unwrap_cell(ref.cell[idx], j, n))
        rxi = ref.xi[idx]
        elements = [(c0, rxi)]
        near = [a for a in range(og.dim) if min(abs(rxi[a]), abs(1 - rxi[a])) < FACE_TIE_F32]
        for sub in itertools.product(*[(0, -1 if rxi[a] < 0.5 else 1) for a in near]):
            if not any(sub):
                continue
            cn = list(c0)
            for a, s in zip(near, sub):
                cn[a] += s
            _, xn, _, st = orc.eval_in_element(og, D, fl, h, j, cn)
            if st == orc.OK:
                elements.append((cn, xn))
        route = None
        for f in range(nf):
            if err[(f,) + idx] <= tol * scale:
                continue
            matched = None
            for k, (ce, xe) in enumerate(elements):
                # A neighbour across a face is reached with its coordinates up to 2e-5 outside
                # [0, 1]; the kernels then evaluate that element's basis pieces there, while the
                # oracle's basis is cut off at the end of its support.  For the hat (order 0) the two
                # differ by up to the excess times the stencil's values on each axis; the cubic and
                # quintic pieces meet their neighbours with matching slopes, so for them the
                # difference is of second order.
                excess = float(np.max(np.maximum(0.0, np.maximum(-np.asarray(xe), np.asarray(xe) - 1.0))))
                box = tuple(np.mod(np.arange(ce[a] - 2, ce[a] + 4), n[a]) for a in reversed(range(og.dim)))
                hbox = float(np.abs(h[f][np.ix_(*box)]).max())
                allow = tol * scale + 2 * og.dim * excess * hbox
                lo_m, hi_m = orc.order(og, maybe, ce, f), orc.order(og, sure, ce, f)
                for m in range(min(lo_m, hi_m), max(lo_m, hi_m) + 1):
                    v = orc.interp(og, h[f], ce, xe, m)
                    if abs(got[(f,) + idx] - v) <= allow:
                        matched = "face_ties" if k > 0 else "limiter_ties"
                        break
                if matched:
                    break
            assert matched, (f"target {j} field {f}: GPU {got[(f,) + idx]!r} matches no allowed element and order "
                             f"(oracle {ref.h[(f,) + idx]!r}, element {c0}, xi {rxi}, order {ref.order[(f,) + idx]})")
            route = "face_ties" if (route == "face_ties" or matched == "face_ties") else matched
        counts[route] += 1
    return counts


def f64_run_ties(orc, og, g, F0, t0, dt, nsteps, velocity_from_fields=False, tol=1e-12):
    """nsteps FP64 steps, each checked by f64_step_ties from the GPU's previous result (t_k =
    t0 + k dt, as the library forms it); then the same run as ONE sl_step call must reproduce the
    chained steps bit for bit.  Returns (fields, targets beyond tol, face ties) summed over steps."""
    F = np.asarray(F0, dtype=np.float64)
    beyond = ties = 0
    for k in range(nsteps):
        F, b, ti = f64_step_ties(orc, og, g, F, t0 + k * dt, dt, velocity_from_fields, tol)
        beyond += b
        ties += ti
    f = torch.tensor(np.asarray(F0, dtype=np.float64), device="cuda")
    g.step(f, torch.empty_like(f), t0, dt, nsteps)
    torch.cuda.synchronize()
    assert np.array_equal(f.cpu().numpy(), F), "one multi-step call differs from the chained single steps"
    return F, beyond, ties
