"""Python wrapper of the FP64 CPU oracle (``sl_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's CPU-baseline
leg call this module; the CUDA library never does.  It imports nothing from the CUDA package.

Each wrapper states the paper passage its C function restates (arXiv:1410.2817):
``zspline`` (Appendix), ``flags`` (Sec. 2.3), ``velocity``/``advect`` (eq. vel, RK4),
``newton``/``locate`` (Sec. 2.2, eq. mapping1), ``remap`` (eq. multiZ with order reduction),
``moments`` (Sec. 3.1, Table 1), ``step`` (the whole FSL step).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SL_ORACLE_SOURCE / SL_ORACLE_BUILD_DIR build another copy of the source (the mutation test plants
# mistakes in a copy and checks that the pin tests catch them)
_SRC = os.environ.get("SL_ORACLE_SOURCE", os.path.join(_HERE, "sl_oracle.c"))
_BUILD = os.environ.get("SL_ORACLE_BUILD_DIR", os.path.join(_HERE, "_build"))
_LIB_PATH = os.path.join(_BUILD, "libsl_oracle.so")
_lock = threading.Lock()
_lib = None

# target status codes (oracle-local)
OK, LOCATE, NEWTON, FOLD = 0, 1, 2, 3
VELOCITY_KINDS = {"uniform": 0, "solid_body": 1, "swirl2d": 2, "deform3d": 3, "fourier2d": 4, "fourier3d": 5,
                  "carried": 6, "nlsw": 7}
START_PAPER, START_BACKWARD = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP over target nodes)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nfields", C.c_int), ("n", C.c_int64 * 3),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("max_order", C.c_int), ("threshold", C.c_double),
        ("vel_kind", C.c_int), ("n_vel_params", C.c_int), ("vel_params", C.POINTER(C.c_double)),
        ("newton_max_iter", C.c_int), ("newton_tol", C.c_double), ("walk_max", C.c_int),
        ("slack", C.c_double), ("start_mode", C.c_int), ("fail_keep", C.c_int), ("nthreads", C.c_int),
        ("integrator", C.c_int), ("substeps", C.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        dp, u8p, i64p, i32p, gp = (C.POINTER(C.c_double), C.POINTER(C.c_uint8), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int32), C.POINTER(_Grid))
        lib.or_zspline.argtypes = [C.c_int, C.c_double]
        lib.or_zspline.restype = C.c_double
        lib.or_zspline_array.argtypes = [C.c_int, C.c_int64, dp, dp]
        lib.or_sinpi.argtypes = [C.c_double]
        lib.or_sinpi.restype = C.c_double
        lib.or_cospi.argtypes = [C.c_double]
        lib.or_cospi.restype = C.c_double
        lib.or_flags.argtypes = [gp, dp, u8p]
        lib.or_velocity.argtypes = [gp, dp, C.c_double, dp]
        lib.or_advect.argtypes = [gp, C.c_double, C.c_double, dp]
        lib.or_advect_carried.argtypes = [gp, dp, C.c_double, dp]
        lib.or_newton.argtypes = [C.c_int, dp, C.c_int, C.c_double, dp, C.POINTER(C.c_int)]
        lib.or_newton.restype = C.c_int
        lib.or_locate.argtypes = [gp, dp, i64p, i64p, dp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.or_locate.restype = C.c_int
        lib.or_order.argtypes = [gp, u8p, i64p, C.c_int]
        lib.or_order.restype = C.c_int
        lib.or_interp.argtypes = [gp, dp, i64p, dp, C.c_int]
        lib.or_interp.restype = C.c_double
        lib.or_remap.argtypes = [gp, dp, u8p, dp, dp, i64p, dp, u8p, u8p, i32p, i32p]
        lib.or_remap.restype = C.c_int64
        lib.or_eval_in_element.argtypes = [gp, dp, u8p, dp, i64p, i64p, dp, dp, u8p]
        lib.or_eval_in_element.restype = C.c_int
        lib.or_step.argtypes = [gp, dp, C.c_double, C.c_double, C.c_int]
        lib.or_step.restype = C.c_int64
        lib.or_moments.argtypes = [gp, dp, C.c_int, dp]
        lib.or_max_threads.restype = C.c_int
        _lib = lib
        return lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


@dataclass
class OracleGrid:
    """Grid and method parameters of the oracle (plain values; no dependency on the CUDA package)."""
    dim: int
    n: Sequence[int]
    nfields: int = 1
    lo: Sequence[float] = (0.0, 0.0, 0.0)
    hi: Sequence[float] = (1.0, 1.0, 1.0)
    max_order: int = 1
    threshold: float = 0.25
    velocity: str = "uniform"
    velocity_params: Sequence[float] = field(default_factory=lambda: [0.0, 0.0, 0.0])
    newton_max_iter: int = 8
    newton_tol: float = 1e-14
    walk_max: int = 64
    slack: float = 1e-12
    start: int = START_PAPER
    nthreads: int = 0
    integrator: str = "rk4"       # "rk4" (classical) or "wrk3" (Williamson's low-storage RK3)
    substeps: int = 1             # integrator steps of dt / substeps per remap

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n) + (1,) * (3 - len(self.n))
        self.lo = tuple(float(v) for v in self.lo) + (0.0,) * (3 - len(self.lo))
        self.hi = tuple(float(v) for v in self.hi) + (1.0,) * (3 - len(self.hi))
        self._params = np.ascontiguousarray(np.asarray(self.velocity_params, dtype=np.float64).ravel())
        self._nparams = int(self._params.size)
        if self._params.size == 0:
            self._params = np.zeros(1)

    @property
    def shape(self):
        """numpy shape of one field plane (slowest axis first; x is the last, fastest axis)."""
        return tuple(reversed(self.n[: self.dim]))

    @property
    def nnodes(self):
        return int(np.prod(self.n[: self.dim]))

    def _c(self) -> _Grid:
        g = _Grid()
        g.dim, g.nfields = self.dim, self.nfields
        g.n[:] = list(self.n)
        g.lo[:] = list(self.lo)
        g.hi[:] = list(self.hi)
        g.max_order, g.threshold = self.max_order, self.threshold
        g.vel_kind = VELOCITY_KINDS[self.velocity]
        g.n_vel_params = self._nparams
        g.vel_params = _ptr(self._params, C.c_double)
        g.newton_max_iter, g.newton_tol, g.walk_max = self.newton_max_iter, self.newton_tol, self.walk_max
        g.slack, g.start_mode, g.fail_keep, g.nthreads = self.slack, self.start, 1, self.nthreads
        g.integrator = {"rk4": 0, "wrk3": 1}[self.integrator]
        g.substeps = int(self.substeps)
        return g


def _fields(grid: OracleGrid, h) -> np.ndarray:
    h = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    if h.size != grid.nfields * grid.nnodes:
        raise ValueError("field array has the wrong size")
    return h


def max_threads() -> int:
    return int(_load().or_max_threads())


def zspline(m: int, x) -> np.ndarray:
    """Cardinal Z-spline basis function Z~_m (Appendix; Z~_0 is the hat)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    _load().or_zspline_array(m, x.size, _ptr(x, C.c_double), _ptr(out, C.c_double))
    return out


def sinpi(x: float) -> float:
    return float(_load().or_sinpi(x))


def cospi(x: float) -> float:
    return float(_load().or_cospi(x))


def flags(grid: OracleGrid, h) -> np.ndarray:
    """Jump-criterion flags (Sec. 2.3): uint8 per node, bit f for field f."""
    h = _fields(grid, h)
    out = np.empty(grid.shape, dtype=np.uint8)
    g = grid._c()
    _load().or_flags(C.byref(g), _ptr(h, C.c_double), _ptr(out, C.c_uint8))
    return out


def velocity_at(grid: OracleGrid, points, t: float) -> np.ndarray:
    """Velocity of the grid's flow at physical points (rows), time t."""
    pts = np.asarray(points, dtype=np.float64).reshape(-1, grid.dim)
    out = np.empty_like(pts)
    g = grid._c()
    lib = _load()
    xb, ub = np.zeros(3), np.zeros(3)
    for r in range(pts.shape[0]):
        xb[: grid.dim] = pts[r]
        lib.or_velocity(C.byref(g), _ptr(xb, C.c_double), float(t), _ptr(ub, C.c_double))
        out[r] = ub[: grid.dim]
    return out


def advect(grid: OracleGrid, t: float, dt: float) -> np.ndarray:
    """RK4 displacement of every Lagrangian node over [t, t+dt], in cell units; shape (*shape, dim)."""
    D = np.empty(grid.shape + (grid.dim,), dtype=np.float64)
    g = grid._c()
    _load().or_advect(C.byref(g), float(t), float(dt), _ptr(D, C.c_double))
    return D


def advect_carried(grid: OracleGrid, h, dt: float) -> np.ndarray:
    """Displacement over dt of every node moving with the velocity it carries (velocity kind
    "carried": the fields named by velocity_params, default the first dim fields), in cell units;
    shape (*shape, dim)."""
    h = _fields(grid, h)
    D = np.empty(grid.shape + (grid.dim,), dtype=np.float64)
    g = grid._c()
    _load().or_advect_carried(C.byref(g), _ptr(h, C.c_double), float(dt), _ptr(D, C.c_double))
    return D


def newton(P, max_iter: int = 8, tol: float = 1e-14):
    """Newton inversion of the multilinear element map (eq. mapping1).  P: (2^d, d) vertices
    relative to the target.  Returns (xi, status, iterations)."""
    P = np.ascontiguousarray(np.asarray(P, dtype=np.float64))
    d = P.shape[1]
    xi = np.zeros(3)
    it = C.c_int(0)
    st = _load().or_newton(d, _ptr(P, C.c_double), max_iter, tol, _ptr(xi, C.c_double), C.byref(it))
    return xi[:d].copy(), int(st), int(it.value)


def locate(grid: OracleGrid, D, j):
    """Element search for target node j (Sec. 2.2).  Returns (cell vector, xi, status, hops, iters)."""
    D = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
    jv = np.zeros(3, dtype=np.int64)
    jv[: grid.dim] = j
    c = np.zeros(3, dtype=np.int64)
    xi = np.zeros(3)
    hops, iters = C.c_int(0), C.c_int(0)
    g = grid._c()
    st = _load().or_locate(C.byref(g), _ptr(D, C.c_double), _ptr(jv, C.c_int64), _ptr(c, C.c_int64),
                           _ptr(xi, C.c_double), C.byref(hops), C.byref(iters))
    return c[: grid.dim].copy(), xi[: grid.dim].copy(), int(st), int(hops.value), int(iters.value)


def order(grid: OracleGrid, flag_arr, c, f: int) -> int:
    fl = np.ascontiguousarray(np.asarray(flag_arr, dtype=np.uint8))
    cv = np.zeros(3, dtype=np.int64)
    cv[: grid.dim] = c
    g = grid._c()
    return int(_load().or_order(C.byref(g), _ptr(fl, C.c_uint8), _ptr(cv, C.c_int64), f))


def interp(grid: OracleGrid, hf, c, xi, m: int) -> float:
    """eq. (multiZ) in logical coordinates: value of one field plane at c + xi with order m."""
    hf = np.ascontiguousarray(np.asarray(hf, dtype=np.float64))
    cv = np.zeros(3, dtype=np.int64)
    cv[: grid.dim] = c
    xv = np.zeros(3)
    xv[: grid.dim] = xi
    g = grid._c()
    return float(_load().or_interp(C.byref(g), _ptr(hf, C.c_double), _ptr(cv, C.c_int64),
                                   _ptr(xv, C.c_double), m))


@dataclass
class RemapResult:
    h: np.ndarray          # (nfields, *shape)
    cell: np.ndarray       # (*shape) wrapped linear index of the element's lower corner, -1 = failed
    xi: np.ndarray         # (*shape, dim)
    order: np.ndarray      # (nfields, *shape); 255 = failed
    status: np.ndarray     # (*shape)
    hops: np.ndarray
    iters: np.ndarray
    nfail: int


def remap(grid: OracleGrid, D, flag_arr, h) -> RemapResult:
    """Reconstruct every field on the reference mesh (Sec. 2, 2.2, 2.3, eq. multiZ)."""
    D = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
    fl = np.ascontiguousarray(np.asarray(flag_arr, dtype=np.uint8))
    h = _fields(grid, h)
    shp = grid.shape
    out = np.empty((grid.nfields,) + shp)
    cell = np.empty(shp, dtype=np.int64)
    xi = np.empty(shp + (grid.dim,))
    order_ = np.empty((grid.nfields,) + shp, dtype=np.uint8)
    status = np.empty(shp, dtype=np.uint8)
    hops = np.empty(shp, dtype=np.int32)
    iters = np.empty(shp, dtype=np.int32)
    g = grid._c()
    nfail = _load().or_remap(C.byref(g), _ptr(D, C.c_double), _ptr(fl, C.c_uint8), _ptr(h, C.c_double),
                             _ptr(out, C.c_double), _ptr(cell, C.c_int64), _ptr(xi, C.c_double),
                             _ptr(order_, C.c_uint8), _ptr(status, C.c_uint8), _ptr(hops, C.c_int32),
                             _ptr(iters, C.c_int32))
    return RemapResult(out, cell, xi, order_, status, hops, iters, int(nfail))


def remap_values(grid: OracleGrid, D, flag_arr, h) -> np.ndarray:
    """Remapped fields only (no per-target diagnostics)."""
    D = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
    fl = np.ascontiguousarray(np.asarray(flag_arr, dtype=np.uint8))
    h = _fields(grid, h)
    out = np.empty((grid.nfields,) + grid.shape)
    g = grid._c()
    _load().or_remap(C.byref(g), _ptr(D, C.c_double), _ptr(fl, C.c_uint8), _ptr(h, C.c_double),
                     _ptr(out, C.c_double), None, None, None, None, None, None)
    return out


def eval_in_element(grid: OracleGrid, D, flag_arr, h, j, c):
    """Fields at target j interpolated in element c (Newton in that element, order from flags)."""
    D = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
    fl = np.ascontiguousarray(np.asarray(flag_arr, dtype=np.uint8))
    h = _fields(grid, h)
    jv = np.zeros(3, dtype=np.int64)
    jv[: grid.dim] = j
    cv = np.zeros(3, dtype=np.int64)
    cv[: grid.dim] = c
    out = np.empty(grid.nfields)
    xi = np.zeros(3)
    order_ = np.zeros(grid.nfields, dtype=np.uint8)
    g = grid._c()
    st = _load().or_eval_in_element(C.byref(g), _ptr(D, C.c_double), _ptr(fl, C.c_uint8), _ptr(h, C.c_double),
                                    _ptr(jv, C.c_int64), _ptr(cv, C.c_int64), _ptr(out, C.c_double),
                                    _ptr(xi, C.c_double), _ptr(order_, C.c_uint8))
    return out, xi[: grid.dim].copy(), order_, int(st)


def step(grid: OracleGrid, h, t0: float, dt: float, nsteps: int):
    """nsteps full FSL steps (flags -> RK4 trajectories -> remap).  Returns (fields, failures)."""
    h = _fields(grid, h).copy()
    g = grid._c()
    nfail = _load().or_step(C.byref(g), _ptr(h, C.c_double), float(t0), float(dt), int(nsteps))
    return h.reshape((grid.nfields,) + grid.shape), int(nfail)


def moments(grid: OracleGrid, hf, pmax: int = 4) -> np.ndarray:
    """Discrete moments m_0..m_pmax about the box centre (Sec. 3.1, Table 1)."""
    hf = np.ascontiguousarray(np.asarray(hf, dtype=np.float64))
    if hf.size != grid.nnodes:
        raise ValueError("moments take one field plane")
    out = np.zeros(pmax + 1)
    g = grid._c()
    _load().or_moments(C.byref(g), _ptr(hf, C.c_double), pmax, _ptr(out, C.c_double))
    return out
