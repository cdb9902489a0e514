"""sl_moments_noalloc: moments without any device allocation, for callers that cannot allocate
(an application whose own allocator owns all device memory, a real-time path where cudaMalloc
would synchronise the device, a caller holding only the plane it was given).  Its results must
equal sl_moments on a grid, call after call, although every call reuses the same fixed scratch.
This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1410_2817_gb300 import build, sl as slmod
    build.build()
    L = slmod.lib()
    L.sl_moments_noalloc.restype = C.c_int
    L.sl_moments_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p]
    return slmod


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def _noalloc(sl, dim, n, lo, hi, dtype, field, pmax):
    nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    lo_ = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
    hi_ = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
    out = (C.c_double * (pmax + 1))()
    st = sl.lib().sl_moments_noalloc(dim, nn, lo_, hi_, dtype, C.c_void_p(field.data_ptr()), pmax, out,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, [float(v) for v in out]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_moments_match_grid_moments(sl, orc, dtype):
    sd = sl.SL_F64 if dtype == "f64" else sl.SL_F32
    td = torch.float64 if dtype == "f64" else torch.float32
    cases = [(2, (96, 70), (0.0, -1.0), (2.0, 1.5), 4), (3, (11, 7, 9), (0.0, -1.0, 2.0), (1.0, 3.0, 4.0), 7)]
    rng = np.random.default_rng(17)
    for dim, n, lo, hi, pmax in cases:
        g = sl.Grid(dim, n, 1, sd, lo=lo, hi=hi)
        for call in range(2):  # two calls in a row reuse the same static scratch
            field = torch.tensor(rng.standard_normal(tuple(reversed(n))), dtype=td, device="cuda")
            ref = g.moments(field, pmax)
            st, got = _noalloc(sl, dim, n, lo, hi, sd, field, pmax)
            assert st == sl.SL_OK
            for a, b in zip(got, ref):
                assert abs(a - b) <= 1e-13 * max(1.0, abs(b)), (dim, call, a, b)
            # and against the oracle's moments of the same plane
            og = orc.OracleGrid(dim=dim, n=n, nfields=1, lo=lo, hi=hi)
            for a, b in zip(got, orc.moments(og, field.double().cpu().numpy(), pmax)):
                assert abs(a - b) <= 1e-12 * max(1.0, abs(b)), (dim, call, a, b)


def test_noalloc_rejects_sizes_beyond_its_scratch(sl):
    field = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    st, _ = _noalloc(sl, 2, (8, 8), (0, 0), (1, 1), sl.SL_F64, field, 8)
    assert st == sl.SL_ERR_ARG
    assert "pmax" in sl.lib().sl_last_error().decode()
    st, _ = _noalloc(sl, 2, (1 << 16, 1 << 16), (0, 0), (1, 1), sl.SL_F64, field, 2)
    assert st == sl.SL_ERR_ARG
