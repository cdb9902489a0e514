"""The C-ABI library loads and exports every entry point declared in include/sl.h; host-side
argument checks answer without a GPU (no kernel is launched here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libsl():
    from paper_1410_2817_gb300 import build, sl
    build.build()
    return sl


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sl_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(libsl):
    names = _declared_symbols()
    assert "sl_step" in names and "sl_create_grid" in names and len(names) >= 16
    L = C.CDLL(libsl.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_workspace_bytes_and_validation(libsl):
    sl = libsl
    d = sl.make_desc(2, (64, 64), 1, sl.SL_F64, velocity="swirl2d", velocity_params=[5.0])
    nb = sl.sl_grid_workspace_bytes(d)
    # two displacement buffers of 64*64*2 doubles plus flags and counters
    assert nb >= 2 * 64 * 64 * 2 * 8 + 64 * 64
    d32 = sl.make_desc(2, (64, 64), 1, sl.SL_F32, velocity="swirl2d", velocity_params=[5.0])
    assert sl.sl_grid_workspace_bytes(d32) < nb
    bad = [
        sl.make_desc(4, (64, 64), 1),
        sl.make_desc(2, (2, 64), 1),
        sl.make_desc(2, (64, 64), 9),
        sl.make_desc(2, (64, 64), 1, max_order=3),
        sl.make_desc(2, (64, 64), 1, velocity="deform3d", velocity_params=[3.0]),
        sl.make_desc(3, (8, 8, 8), 1, velocity="swirl2d", velocity_params=[5.0]),
        sl.make_desc(2, (64, 64), 1, sl.SL_F64, newton_mode=sl.SL_NEWTON_MIXED),
        sl.make_desc(2, (64, 64), 1, velocity="fourier2d", velocity_params=[3.0, 1, 1, 0.5, 0.5]),
        sl.make_desc(2, (64, 64), 1, velocity="swirl2d", velocity_params=[0.0]),
        sl.make_desc(2, (64, 64), 1, integrator=2),
        sl.make_desc(2, (64, 64), 1, velocity="carried", velocity_params=[]),        # fewer fields than axes
        sl.make_desc(2, (64, 64), 3, velocity="carried", velocity_params=[0]),       # one index in 2-D
        sl.make_desc(2, (64, 64), 3, velocity="carried", velocity_params=[0, 3]),    # index out of range
        sl.make_desc(2, (64, 64), 3, velocity="carried", velocity_params=[1, 1]),    # repeated index
        sl.make_desc(2, (64, 64), 3, velocity="carried", velocity_params=[0, 1.5]),  # not an integer
        sl.make_desc(2, (64, 64), 3, velocity="nlsw", velocity_params=[250.0], integrator="rk4"),
        sl.make_desc(2, (64, 64), 2, velocity="nlsw", velocity_params=[250.0]),          # needs h, u1, u2
        sl.make_desc(3, (8, 8, 8), 3, velocity="nlsw", velocity_params=[250.0]),         # 2-D only
        sl.make_desc(2, (64, 64), 3, velocity="nlsw", velocity_params=[250.0], trajectory_substeps=2),
        sl.make_desc(2, (64, 64), 3, velocity="nlsw", velocity_params=[250.0, -0.1]),    # negative viscosity
        sl.make_desc(2, (64, 64), 3, velocity="nlsw", velocity_params=[250.0, 0.1, 1.0]),
        sl.make_desc(2, (64, 64), 1, trajectory_substeps=sl.SL_MAX_SUBSTEPS + 1),
    ]
    for b in bad:
        assert sl.sl_grid_workspace_bytes(b) == 0
    for ok in (sl.make_desc(2, (64, 64), 1, integrator="wrk3"),
               sl.make_desc(2, (64, 64), 1, trajectory_substeps=sl.SL_MAX_SUBSTEPS),
               sl.make_desc(3, (8, 8, 8), 1, velocity="deform3d", velocity_params=[3.0], integrator="wrk3",
                            trajectory_substeps=3),
               sl.make_desc(2, (64, 64), 2, velocity="carried", velocity_params=[]),
               sl.make_desc(2, (64, 64), 3, velocity="carried", velocity_params=[2, 0]),
               sl.make_desc(3, (8, 8, 8), 3, velocity="carried", velocity_params=[]),
               sl.make_desc(2, (64, 64), 4, velocity="nlsw", velocity_params=[250.0]),
               sl.make_desc(2, (64, 64), 3, velocity="nlsw", velocity_params=[250.0, 0.0005])):
        assert sl.sl_grid_workspace_bytes(ok) > 0
    # shallow-water grids also hold two sets of RK3 registers (h, u1, u2 and the displacement) and
    # the viscous stress
    base = sl.make_desc(2, (64, 64), 4, velocity="uniform", velocity_params=[0.1, 0.2])
    sw = sl.make_desc(2, (64, 64), 4, velocity="nlsw", velocity_params=[250.0])
    assert sl.sl_grid_workspace_bytes(sw) >= sl.sl_grid_workspace_bytes(base) + 13 * 64 * 64 * 4


def test_create_rejects_bad_workspace_without_gpu(libsl):
    sl = libsl
    d = sl.make_desc(2, (16, 16), 1, sl.SL_F64)
    h = C.c_void_p()
    L = sl.lib()
    # misaligned pointer is rejected before any CUDA call
    st = L.sl_create_grid(C.byref(d), C.c_void_p(0x1001), 1 << 30, C.byref(h))
    assert st == sl.SL_ERR_ARG
    st = L.sl_create_grid(C.byref(d), C.c_void_p(0x100000), 16, C.byref(h))
    assert st == sl.SL_ERR_NOMEM
    assert "too small" in L.sl_last_error().decode()
    assert L.sl_status_string(sl.SL_ERR_FOLD).decode() == "folded element"
    assert L.sl_destroy_grid(None) == sl.SL_ERR_ARG


def test_missing_library_fails_loudly(libsl, monkeypatch, tmp_path):
    """Without libsl.so the binding raises; there is no CPU fallback behind any entry point."""
    sl = libsl
    monkeypatch.setattr(sl, "LIB_PATH", str(tmp_path / "libsl.so"))
    monkeypatch.setattr(sl, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        sl.lib()
    with pytest.raises(RuntimeError, match="no fallback"):
        sl.sl_grid_workspace_bytes(sl.make_desc(2, (16, 16), 1))
