"""Python binding of libsl.so (include/sl.h): argument marshalling only.

The functions carry the C names.  Device buffers are torch CUDA tensors (only their data pointers
cross the boundary); streams default to torch's current CUDA stream.  Every step of the method runs
in the library's CUDA kernels: there is no Python or CPU fallback, and a missing library raises.

``Grid`` wraps a grid handle with its workspace tensor for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsl.so")

SL_OK, SL_ERR_ARG, SL_ERR_CUDA, SL_ERR_NOMEM, SL_ERR_BUDGET = 0, 1, 2, 3, 4
SL_ERR_LOCATE, SL_ERR_NEWTON, SL_ERR_FOLD, SL_ERR_UNSUPPORTED = 5, 6, 7, 8
SL_F64, SL_F32 = 0, 1
SL_RK4, SL_WRK3 = 0, 1
SL_MAX_SUBSTEPS = 16
INTEGRATOR = {"rk4": SL_RK4, "wrk3": SL_WRK3}
VELOCITY = {"uniform": 0, "solid_body": 1, "swirl2d": 2, "deform3d": 3, "fourier2d": 4, "fourier3d": 5, "carried": 6,
            "nlsw": 7}
SL_NEWTON_F64, SL_NEWTON_MIXED = 0, 1
SL_FAIL_KEEP, SL_FAIL_ERROR = 0, 1
SL_START_BACKWARD, SL_START_PAPER = 0, 1
SL_KERNEL_AUTO, SL_KERNEL_GENERIC, SL_KERNEL_TILED = 0, 1, 2

_DTYPES = {SL_F64: torch.float64, SL_F32: torch.float32}


class SLError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class sl_grid_desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int64 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("nfields", C.c_int), ("dtype", C.c_int), ("max_order", C.c_int), ("limiter_threshold", C.c_double),
        ("integrator", C.c_int), ("velocity_kind", C.c_int), ("velocity_params", C.POINTER(C.c_double)),
        ("n_velocity_params", C.c_int), ("newton_mode", C.c_int), ("newton_max_iter", C.c_int),
        ("walk_max", C.c_int), ("fail_policy", C.c_int), ("walk_start", C.c_int), ("kernel", C.c_int),
        ("tile_config", C.c_int), ("trajectory_substeps", C.c_int),
    ]


class sl_diag(C.Structure):
    _fields_ = [(name, C.c_uint64) for name in (
        "targets", "fail_locate", "fail_newton", "fail_fold", "hops_sum", "hops_max", "iters_sum", "iters_max",
        "newton_f64")] + [("order_hist", C.c_uint64 * 3), ("tiles_fallback", C.c_uint64),
                    ("kernel_launches", C.c_uint64), ("timeouts", C.c_uint64)]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "order_hist"}
        d["order_hist"] = [int(v) for v in self.order_hist]
        return d


class sl_remap_debug(C.Structure):
    _fields_ = [("cell", C.c_void_p), ("xi", C.c_void_p), ("order", C.c_void_p), ("status", C.c_void_p)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libsl.so (built in-tree by paper_1410_2817_gb300.build).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1410_2817_gb300.build.build() "
                               "(the CUDA path has no fallback)")
        L = C.CDLL(LIB_PATH)
        vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
        pp = C.POINTER(C.c_void_p)
        sig = {
            "sl_grid_workspace_bytes": (C.c_size_t, [C.POINTER(sl_grid_desc)]),
            "sl_create_grid": (C.c_int, [C.POINTER(sl_grid_desc), vp, C.c_size_t, C.POINTER(vp)]),
            "sl_destroy_grid": (C.c_int, [vp]),
            "sl_advect_nodes": (C.c_int, [vp, C.c_double, C.c_double, vp]),
            "sl_advect_nodes_carried": (C.c_int, [vp, pp, C.c_double, vp]),
            "sl_remap_fields": (C.c_int, [vp, pp, pp, vp]),
            "sl_remap_fields_debug": (C.c_int, [vp, pp, pp, C.POINTER(sl_remap_debug), vp]),
            "sl_step": (C.c_int, [vp, pp, pp, C.c_double, C.c_double, C.c_int, vp]),
            "sl_step_out": (C.c_int, [vp, pp, pp, pp, C.c_double, C.c_double, C.c_int, vp]),
            "sl_moments": (C.c_int, [vp, vp, C.c_int, dp, vp]),
            "sl_compute_flags": (C.c_int, [vp, pp, vp, vp]),
            "sl_set_displacement": (C.c_int, [vp, vp, i64, vp]),
            "sl_get_displacement": (C.c_int, [vp, vp, i64, vp]),
            "sl_get_diagnostics": (C.c_int, [vp, C.POINTER(sl_diag), vp]),
            "sl_reset_diagnostics": (C.c_int, [vp, vp]),
            "sl_batch_workspace_bytes": (C.c_size_t, [C.POINTER(vp), C.c_int, C.c_int]),
            "sl_batch_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(pp), C.POINTER(pp), dp, dp, C.c_int, vp,
                                          C.c_size_t, C.POINTER(vp)]),
            "sl_batch_step": (C.c_int, [vp, C.c_int, C.c_int, vp]),
            "sl_batch_info": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_ulonglong), dp]),
            "sl_batch_destroy": (C.c_int, [vp]),
            "sl_status_string": (C.c_char_p, [C.c_int]),
            "sl_last_error": (C.c_char_p, []),
            "sl_version": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args
        _lib = L
        return L


def _check(status: int, where: str):
    if status != SL_OK:
        L = lib()
        detail = L.sl_status_string(status).decode()
        extra = L.sl_last_error().decode()
        raise SLError(status, where, f"{detail}; {extra}" if extra else detail)


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _planes(ts):
    """Host array of plane pointers: from a sequence of contiguous CUDA tensors, or from one
    contiguous CUDA tensor whose leading axis indexes the planes (no per-plane views)."""
    if isinstance(ts, torch.Tensor):
        if not ts.is_cuda or not ts.is_contiguous() or ts.dim() < 2:
            raise ValueError("field planes must be contiguous CUDA tensors")
        nplanes = ts.shape[0]
        step = (ts.numel() // max(nplanes, 1)) * ts.element_size()
        base = ts.data_ptr()
        arr = (C.c_void_p * nplanes)(*[base + q * step for q in range(nplanes)])
        return C.cast(arr, C.POINTER(C.c_void_p)), arr
    arr = (C.c_void_p * len(ts))()
    for q, t in enumerate(ts):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("field planes must be contiguous CUDA tensors")
        arr[q] = t.data_ptr()
    return C.cast(arr, C.POINTER(C.c_void_p)), arr


# ------------------------------------------------------------------------------------------------
# thin wrappers with the C names
# ------------------------------------------------------------------------------------------------
def make_desc(dim, n, nfields, dtype=SL_F32, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), max_order=1,
              limiter_threshold=0.25, velocity="uniform", velocity_params=(0.0, 0.0, 0.0),
              newton_mode=None, newton_max_iter=0, walk_max=0, fail_policy=SL_FAIL_KEEP,
              walk_start=SL_START_BACKWARD, kernel=SL_KERNEL_AUTO, tile_config=0, integrator=None,
              trajectory_substeps=0):
    d = sl_grid_desc()
    d.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    d.n[:] = [int(v) for v in nn]
    d.lo[:] = [float(v) for v in list(lo) + [0.0] * (3 - len(lo))]
    d.hi[:] = [float(v) for v in list(hi) + [1.0] * (3 - len(hi))]
    d.nfields, d.dtype, d.max_order = nfields, dtype, max_order
    d.limiter_threshold = float(limiter_threshold)
    if integrator is None:  # the shallow-water system integrates with the paper's RK3
        integrator = SL_WRK3 if velocity in ("nlsw", 7) else SL_RK4
    d.integrator = INTEGRATOR[integrator] if isinstance(integrator, str) else int(integrator)
    d.trajectory_substeps = int(trajectory_substeps)
    d.velocity_kind = VELOCITY[velocity] if isinstance(velocity, str) else int(velocity)
    params = (C.c_double * max(1, len(velocity_params)))(*[float(v) for v in velocity_params])
    d.velocity_params = C.cast(params, C.POINTER(C.c_double))
    d.n_velocity_params = len(velocity_params)
    d._params_keepalive = params
    if newton_mode is None:
        newton_mode = SL_NEWTON_MIXED if dtype == SL_F32 else SL_NEWTON_F64
    d.newton_mode, d.newton_max_iter, d.walk_max = newton_mode, newton_max_iter, walk_max
    d.fail_policy, d.walk_start, d.kernel, d.tile_config = fail_policy, walk_start, kernel, tile_config
    return d


def sl_grid_workspace_bytes(desc: sl_grid_desc) -> int:
    return int(lib().sl_grid_workspace_bytes(C.byref(desc)))


def sl_create_grid(desc: sl_grid_desc, workspace: torch.Tensor) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().sl_create_grid(C.byref(desc), C.c_void_p(workspace.data_ptr()),
                                workspace.numel() * workspace.element_size(), C.byref(h)), "sl_create_grid")
    return h


def sl_destroy_grid(h):
    _check(lib().sl_destroy_grid(h), "sl_destroy_grid")


def sl_advect_nodes(h, t: float, dt: float, stream=None):
    _check(lib().sl_advect_nodes(h, float(t), float(dt), _stream(stream)), "sl_advect_nodes")


def sl_advect_nodes_carried(h, fields: Sequence[torch.Tensor], dt: float, stream=None):
    pf, _a = _planes(fields)
    _check(lib().sl_advect_nodes_carried(h, pf, float(dt), _stream(stream)), "sl_advect_nodes_carried")


def sl_remap_fields(h, fin: Sequence[torch.Tensor], fout: Sequence[torch.Tensor], stream=None):
    pi, _a = _planes(fin)
    po, _b = _planes(fout)
    _check(lib().sl_remap_fields(h, pi, po, _stream(stream)), "sl_remap_fields")


def sl_remap_fields_debug(h, fin, fout, cell=None, xi=None, order=None, status=None, stream=None):
    pi, _a = _planes(fin)
    po, _b = _planes(fout)
    dbg = sl_remap_debug()
    for name, t in (("cell", cell), ("xi", xi), ("order", order), ("status", status)):
        setattr(dbg, name, t.data_ptr() if t is not None else None)
    _check(lib().sl_remap_fields_debug(h, pi, po, C.byref(dbg), _stream(stream)), "sl_remap_fields_debug")


def sl_step(h, fields, scratch, t0: float, dt: float, nsteps: int, stream=None):
    pf, _a = _planes(fields)
    ps, _b = _planes(scratch)
    _check(lib().sl_step(h, pf, ps, float(t0), float(dt), int(nsteps), _stream(stream)), "sl_step")


def sl_step_out(h, fin, fout, scratch, t0: float, dt: float, nsteps: int, stream=None):
    pi, _a = _planes(fin)
    po, _b = _planes(fout)
    ps, _c = _planes(scratch) if scratch is not None else (None, None)
    _check(lib().sl_step_out(h, pi, po, ps, float(t0), float(dt), int(nsteps), _stream(stream)), "sl_step_out")


def sl_moments(h, field: torch.Tensor, pmax: int = 4, stream=None):
    out = (C.c_double * (pmax + 1))()
    _check(lib().sl_moments(h, C.c_void_p(field.data_ptr()), int(pmax), out, _stream(stream)), "sl_moments")
    return [float(v) for v in out]


def sl_compute_flags(h, fields, flags_out: torch.Tensor, stream=None):
    pf, _a = _planes(fields)
    _check(lib().sl_compute_flags(h, pf, C.c_void_p(flags_out.data_ptr()), _stream(stream)), "sl_compute_flags")


def sl_set_displacement(h, D: torch.Tensor, stride: int, stream=None):
    _check(lib().sl_set_displacement(h, C.c_void_p(D.data_ptr()), int(stride), _stream(stream)),
           "sl_set_displacement")


def sl_get_displacement(h, D_out: torch.Tensor, stride: int, stream=None):
    _check(lib().sl_get_displacement(h, C.c_void_p(D_out.data_ptr()), int(stride), _stream(stream)),
           "sl_get_displacement")


def sl_get_diagnostics(h, stream=None) -> dict:
    d = sl_diag()
    _check(lib().sl_get_diagnostics(h, C.byref(d), _stream(stream)), "sl_get_diagnostics")
    return d.as_dict()


def sl_reset_diagnostics(h, stream=None):
    _check(lib().sl_reset_diagnostics(h, _stream(stream)), "sl_reset_diagnostics")


def sl_status_string(status: int) -> str:
    return lib().sl_status_string(int(status)).decode()


def sl_version() -> str:
    return lib().sl_version().decode()


# ------------------------------------------------------------------------------------------------
# convenience object
# ------------------------------------------------------------------------------------------------
class Grid:
    """A grid handle plus the workspace tensor it borrows (allocated through torch)."""

    def __init__(self, dim, n, nfields, dtype=SL_F32, device="cuda", **kw):
        self.desc = make_desc(dim, n, nfields, dtype, **kw)
        self.dim, self.nfields, self.dtype = dim, nfields, dtype
        self.n = tuple(int(v) for v in n)
        self.torch_dtype = _DTYPES[dtype]
        nbytes = sl_grid_workspace_bytes(self.desc)
        if nbytes == 0:
            raise SLError(SL_ERR_ARG, "Grid", "invalid grid descriptor")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.handle = sl_create_grid(self.desc, self.workspace)

    @property
    def shape(self):
        return tuple(reversed(self.n[: self.dim]))

    @property
    def nnodes(self):
        p = 1
        for v in self.n[: self.dim]:
            p *= v
        return p

    def close(self):
        if getattr(self, "handle", None) is not None:
            sl_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_fields(self):
        return torch.empty((self.nfields,) + self.shape, dtype=self.torch_dtype, device=self.workspace.device)

    def advect(self, t, dt, stream=None):
        """Trajectories of the grid's analytic velocity over [t, t + dt] into the grid's D."""
        sl_advect_nodes(self.handle, t, dt, stream)

    def advect_carried(self, fields, dt, stream=None):
        """Trajectories of a carried velocity (velocity="carried"): D = dt u / dx from the fields."""
        sl_advect_nodes_carried(self.handle, self._fit(fields), dt, stream)

    def _fit(self, planes):
        """The nfields planes of this grid (a stacked tensor or a sequence); others raise."""
        n = planes.shape[0] if isinstance(planes, torch.Tensor) else len(planes)
        size = planes[0].numel() if n > 0 else 0
        if n != self.nfields or size != self.nnodes:
            raise ValueError(f"expected {self.nfields} planes of {self.nnodes} values")
        return planes

    def remap(self, fin: torch.Tensor, fout: torch.Tensor, stream=None):
        sl_remap_fields(self.handle, self._fit(fin), self._fit(fout), stream)

    def remap_debug(self, fin, fout, stream=None):
        """sl_remap_fields with per-target outputs: (cell, xi, order, status) tensors."""
        dev = fin.device
        cell = torch.empty(self.shape, dtype=torch.int64, device=dev)
        xi = torch.empty(self.shape + (self.dim,), dtype=torch.float64, device=dev)
        order = torch.empty((self.nfields,) + self.shape, dtype=torch.uint8, device=dev)
        status = torch.empty(self.shape, dtype=torch.uint8, device=dev)
        sl_remap_fields_debug(self.handle, list(fin), list(fout), cell, xi, order, status, stream)
        return cell, xi, order, status

    def step(self, fields: torch.Tensor, scratch: torch.Tensor, t0, dt, nsteps, stream=None):
        """nsteps full steps from t0, in place on `fields` (`scratch`: the other half of the
        ping-pong pair, same shape)."""
        sl_step(self.handle, self._fit(fields), self._fit(scratch), t0, dt, nsteps, stream)

    def step_out(self, fin: torch.Tensor, fout: torch.Tensor, t0, dt, nsteps, scratch=None, stream=None):
        """nsteps full steps from t0 of `fin` (read only) into `fout`; `scratch` (same shape) is
        needed for nsteps > 1."""
        sl_step_out(self.handle, self._fit(fin), self._fit(fout), None if scratch is None else self._fit(scratch),
                    t0, dt, nsteps, stream)

    def moments(self, field: torch.Tensor, pmax=4, stream=None):
        return sl_moments(self.handle, field, pmax, stream)

    def flags(self, fields: torch.Tensor, stream=None):
        out = torch.empty(self.shape, dtype=torch.uint8, device=fields.device)
        sl_compute_flags(self.handle, list(fields), out, stream)
        return out

    def set_displacement(self, D: torch.Tensor, stream=None):
        D = D.contiguous()
        sl_set_displacement(self.handle, D, D.shape[-1], stream)

    def get_displacement(self, stream=None):
        out = torch.empty(self.shape + (self.dim,), dtype=self.torch_dtype, device=self.workspace.device)
        sl_get_displacement(self.handle, out, self.dim, stream)
        return out

    def diagnostics(self, stream=None):
        return sl_get_diagnostics(self.handle, stream)

    def reset_diagnostics(self, stream=None):
        sl_reset_diagnostics(self.handle, stream)


def sl_batch_workspace_bytes(grids: Sequence["Grid"], tile_config: int = 0) -> int:
    arr = (C.c_void_p * len(grids))(*[g.handle.value for g in grids])
    return int(lib().sl_batch_workspace_bytes(arr, len(grids), int(tile_config)))


class Batch:
    """Grids advanced together by sl_batch_step (one persistent launch per step).  fields[q] and
    scratch[q] are (nfields, ny, nx) FP32 CUDA tensors of grid q."""

    def __init__(self, grids: Sequence["Grid"], fields, scratch, t0, dt, tile_config: int = 0, device="cuda"):
        self.grids = list(grids)
        n = len(self.grids)
        self._keep = []
        arr = (C.c_void_p * n)(*[g.handle.value for g in self.grids])
        fps = (C.POINTER(C.c_void_p) * n)()
        sps = (C.POINTER(C.c_void_p) * n)()
        for q in range(n):
            pf, a = _planes(list(fields[q]))
            ps, b = _planes(list(scratch[q]))
            fps[q], sps[q] = pf, ps
            self._keep += [a, b]
        t0a = (C.c_double * n)(*[float(v) for v in t0])
        dta = (C.c_double * n)(*[float(v) for v in dt])
        nb = int(lib().sl_batch_workspace_bytes(arr, n, int(tile_config)))
        if nb == 0:
            raise SLError(SL_ERR_UNSUPPORTED, "Batch", "grids not eligible for a batch")
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=device)
        h = C.c_void_p()
        _check(lib().sl_batch_create(arr, n, fps, sps, t0a, dta, int(tile_config), C.c_void_p(self.workspace.data_ptr()),
                                     nb, C.byref(h)), "sl_batch_create")
        self.handle = h
        self.fields, self.scratch = fields, scratch

    def step(self, nsteps: int, use_graph: bool = False, stream=None):
        _check(lib().sl_batch_step(self.handle, int(nsteps), 1 if use_graph else 0, _stream(stream)), "sl_batch_step")

    def info(self):
        ni, nl, t = C.c_int(), C.c_ulonglong(), C.c_double()
        _check(lib().sl_batch_info(self.handle, C.byref(ni), C.byref(nl), C.byref(t)), "sl_batch_info")
        return {"items": ni.value, "launches": nl.value, "t_first": t.value}

    def close(self):
        if getattr(self, "handle", None) is not None:
            lib().sl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_for(workload, dtype=SL_F32, **kw) -> Grid:
    """Grid for an inputs.Workload (same velocity, order and limiter settings)."""
    return Grid(workload.dim, list(workload.n)[: workload.dim], workload.nfields, dtype,
                lo=workload.lo, hi=workload.hi, max_order=workload.max_order,
                limiter_threshold=workload.threshold, velocity=workload.velocity,
                velocity_params=list(workload.velocity_params), **kw)
