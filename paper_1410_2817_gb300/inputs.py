"""Seeded synthetic inputs for the forward semi-Lagrangian step (arXiv:1410.2817).

This module holds only workload descriptions and initial conditions; it contains none of the
method's arithmetic (no trajectories, no limiter, no interpolation).  Both the CUDA path and the
CPU oracle take their inputs from here.

Field planes are numpy arrays of shape (nz, ny, nx) / (ny, nx): x is the fastest axis, node i
sits at lo + i*dx with dx = (hi - lo)/n (periodic box).  Velocity fields are named by kind with a
flat parameter vector:

* ``uniform``     (u, v[, w])
* ``solid_body``  (Omega, cx, cy):          u = Omega (cy - y, x - cx)         (Sec. 3.1)
* ``swirl2d``     (T,):                     2-D swirling deformation flow, period T
* ``deform3d``    (T,):                     3-D deformation flow, period T
* ``fourier2d``   (nmodes, [kx, ky, a, b] * nmodes): streamfunction of Fourier modes
* ``fourier3d``   (nmodes, [k(3), a(3), b(3)] * nmodes): curl of a Fourier vector potential
* ``carried``     ([field index per axis]):  the velocity is itself transported by the nodes
                                            (Burgers, Sec. 3.2); default the first dim fields
* ``nlsw``        (f0,):                    shallow-water system of Sec. 3.3 on fields (h, u1, u2)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np


@dataclass
class Workload:
    name: str
    dim: int
    n: Sequence[int]
    nfields: int
    velocity: str
    velocity_params: Sequence[float]
    dt: float
    steps: int
    t0: float = 0.0
    lo: Sequence[float] = (0.0, 0.0, 0.0)
    hi: Sequence[float] = (1.0, 1.0, 1.0)
    max_order: int = 1
    threshold: float = 0.25
    fail_keep: bool = True
    fields: np.ndarray | None = field(default=None, repr=False)

    @property
    def shape(self):
        return tuple(reversed(list(self.n)[: self.dim]))

    @property
    def nnodes(self) -> int:
        return int(np.prod(list(self.n)[: self.dim]))


def node_coords(n: Sequence[int], lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Physical coordinates of the nodes, one array per axis, shaped like a field plane."""
    dim = len(n)
    axes = [lo[a] + np.arange(n[a], dtype=np.float64) * ((hi[a] - lo[a]) / n[a]) for a in range(dim)]
    grids = np.meshgrid(*reversed(axes), indexing="ij")
    return list(reversed(grids))  # [x, y(, z)] each of shape (.., ny, nx)


def _min_image(d):
    return d - np.round(d)


# ---------------------------------------------------------------------------------------------
# 2-D 64x64 solid-body rotation: cone + slotted disk, one field
# ---------------------------------------------------------------------------------------------
def cone_slotted_disk(n: int) -> np.ndarray:
    """Cone of radius 0.15 (height 1) at (0.5, 0.75) plus a slotted disk of radius 0.15 at
    (0.5, 0.25) with a vertical slot of width 0.05 reaching up to y = 0.35."""
    x, y = node_coords((n, n))
    rc = np.hypot(x - 0.5, y - 0.75)
    cone = np.maximum(0.0, 1.0 - rc / 0.15)
    rd = np.hypot(x - 0.5, y - 0.25)
    disk = (rd <= 0.15) & ~((np.abs(x - 0.5) <= 0.025) & (y <= 0.35))
    return (cone + disk.astype(np.float64))[None]


def workload_sbr64(n: int = 64, steps: int = 16) -> Workload:
    """2-D periodic unit square, FP64, solid-body rotation Omega = 2 pi about the centre,
    dt = 1/64 (a quarter turn in 16 steps, CFL about 4)."""
    return Workload("sbr2d_64", 2, (n, n), 1, "solid_body", [2.0 * math.pi, 0.5, 0.5], 1.0 / 64.0, steps,
                    fields=cone_slotted_disk(n))


# ---------------------------------------------------------------------------------------------
# 2-D 1024^2 swirling deformation flow, three fields
# ---------------------------------------------------------------------------------------------
def swirl_fields(n: int) -> np.ndarray:
    """Gaussian (sigma 0.1) at (0.5, 0.75); step = 1 inside r < 0.2 about (0.5, 0.5);
    sin(2 pi x) sin(2 pi y).  Minimum-image distances."""
    x, y = node_coords((n, n))
    r2 = _min_image(x - 0.5) ** 2 + _min_image(y - 0.75) ** 2
    gauss = np.exp(-r2 / (2.0 * 0.1 ** 2))
    rs = np.hypot(_min_image(x - 0.5), _min_image(y - 0.5))
    stepf = (rs < 0.2).astype(np.float64)
    wave = np.sin(2.0 * np.pi * x) * np.sin(2.0 * np.pi * y)
    return np.stack([gauss, stepf, wave])


def workload_swirl(n: int = 1024, steps: int = 200, cfl: float = 5.0) -> Workload:
    """2-D swirl u = sin^2(pi x) sin(2 pi y) cos(pi t/T), v = -sin^2(pi y) sin(2 pi x) cos(pi t/T),
    T = 5; dt = cfl * dx / max|u| with max|u| = 1."""
    return Workload(f"swirl2d_{n}", 2, (n, n), 3, "swirl2d", [5.0], cfl / n, steps, fields=swirl_fields(n))


# ---------------------------------------------------------------------------------------------
# 2-D inviscid Burgers (Sec. 3.2): the two velocity components are the transported fields
# ---------------------------------------------------------------------------------------------
def burgers_fields(n) -> np.ndarray:
    """Radial pulse u = exp(-150 (r - 0.2)^2) (x - 1/2, y - 1/2) / r about the box centre (zero
    for r <= 0.001), the initial condition of Sec. 3.2; |u| <= 1.  n: side, or (nx, ny)."""
    x, y = node_coords((n, n) if np.isscalar(n) else tuple(n))
    rx, ry = x - 0.5, y - 0.5
    r = np.hypot(rx, ry)
    amp = np.where(r > 0.001, np.exp(-150.0 * (r - 0.2) ** 2) / np.maximum(r, 0.001), 0.0)
    return np.stack([amp * rx, amp * ry])


def workload_burgers(n: int = 1024, steps: int | None = None, cfl: float = 0.5, t_end: float = 0.4) -> Workload:
    """2-D Burgers on the unit square: dt = cfl * dx / max|u| (max|u| = 1; cfl < 1 keeps the
    converging elements at the shock unfolded for one step); by default enough steps to reach
    t_end = 0.4, the last time the paper shows."""
    dt = cfl / n
    if steps is None:
        steps = int(math.ceil(t_end / dt))
    return Workload(f"burgers2d_{n}", 2, (n, n), 2, "carried", [], dt, steps, fields=burgers_fields(n))


# ---------------------------------------------------------------------------------------------
# Shallow water (Sec. 3.3): the equatorial Kelvin wave, eq. (kelvin)
# ---------------------------------------------------------------------------------------------
def kelvin_fields(n: int, t: float = 0.0, amp: float = 1e-4, f0: float = 250.0) -> np.ndarray:
    """h = u1 = exp(-f0 x2^2 / 2) K(x1 - t), u2 = 0 with K(s) = amp exp(-f0 s^2 / 2) (nearest
    periodic image) on [0, 1] x [-0.5, 0.5], n x n nodes; planes (h, u1, u2)."""
    x1 = np.arange(n) / n
    x2 = -0.5 + np.arange(n) / n
    X1, X2 = np.meshgrid(x1, x2)
    s = (X1 - t + 0.5) % 1.0 - 0.5
    h = np.exp(-f0 * X2 ** 2 / 2) * amp * np.exp(-f0 * s ** 2 / 2)
    return np.stack([h, h, np.zeros_like(h)])


def workload_kelvin(n: int = 1024, amp: float = 1e-4, f0: float = 250.0, cfl: float = 0.5,
                    max_order: int = 2, nu: float = 0.0) -> Workload:
    """The paper's Kelvin-wave tests: f0 = 250, amplitude 1e-4 (linear; nu = 0), or amplitude 0.5
    with nu = 0.0005 (the nonlinear Kelvin-Poincare run), limiter off, to t = 1 (once round the
    periodic box) with dt = cfl dx (unit wave speed)."""
    steps = int(round(1.0 / (cfl / n)))
    params = [f0] if nu == 0.0 else [f0, nu]
    return Workload(f"kelvin_{n}", 2, (n, n), 3, "nlsw", params, 1.0 / steps, steps, lo=(0.0, -0.5, 0.0),
                    hi=(1.0, 0.5, 1.0), max_order=max_order, threshold=-1.0,
                    fields=kelvin_fields(n, 0.0, amp, f0))


# ---------------------------------------------------------------------------------------------
# 3-D deformation flow, two fields
# ---------------------------------------------------------------------------------------------
def deform3d_fields(n: int) -> np.ndarray:
    """Gaussian (sigma 0.08) at (0.35, 0.35, 0.35); indicator of the sphere of radius 0.15 about
    the centre."""
    x, y, z = node_coords((n, n, n))
    r2 = _min_image(x - 0.35) ** 2 + _min_image(y - 0.35) ** 2 + _min_image(z - 0.35) ** 2
    gauss = np.exp(-r2 / (2.0 * 0.08 ** 2))
    rs2 = _min_image(x - 0.5) ** 2 + _min_image(y - 0.5) ** 2 + _min_image(z - 0.5) ** 2
    sphere = (rs2 <= 0.15 ** 2).astype(np.float64)
    return np.stack([gauss, sphere])


def workload_deform3d(n: int = 256, steps: int = 100, dt: float = 0.03) -> Workload:
    """3-D deformation flow with period T = 3; 100 steps of 0.03 end at t = T where the flow has
    reversed and the exact solution equals the initial state."""
    return Workload(f"deform3d_{n}", 3, (n, n, n), 2, "deform3d", [3.0], dt, steps, fields=deform3d_fields(n))


# ---------------------------------------------------------------------------------------------
# Cosine hill (Sec. 3.1, eq. alpha) and the Table 1 grid
# ---------------------------------------------------------------------------------------------
def cosine_hill(n: Sequence[int], lo, hi, centre, radius) -> np.ndarray:
    x, y = node_coords(tuple(n), lo, hi)
    r = np.hypot(x - centre[0], y - centre[1])
    return np.where(r <= radius, 0.5 * (1.0 + np.cos(np.pi * r / radius)), 0.0)


def table1_grid():
    """The grid on which Table 1's exact moments are reproduced: [0,2]^2, 50 x 50 nodes at
    x_i = 0.04 i, the cosine hill scaled by 2 (centre (0.5, 1.0), radius 0.2)."""
    n, lo, hi = (50, 50), (0.0, 0.0), (2.0, 2.0)
    return n, lo, hi, cosine_hill(n, lo, hi, (0.5, 1.0), 0.2)


# ---------------------------------------------------------------------------------------------
# Random Fourier velocities (batched grids and served jobs)
# ---------------------------------------------------------------------------------------------
def _wavevector(rng, dim):
    vals = np.array([-4, -3, -2, -1, 1, 2, 3, 4], dtype=np.float64)
    return rng.choice(vals, size=dim)


def fourier2d_params(rng, nmodes: int = 8) -> List[float]:
    p = [float(nmodes)]
    for _ in range(nmodes):
        k = _wavevector(rng, 2)
        a, b = rng.standard_normal(2)
        p += [k[0], k[1], float(a), float(b)]
    return p


def fourier3d_params(rng, nmodes: int = 8) -> List[float]:
    p = [float(nmodes)]
    for _ in range(nmodes):
        k = _wavevector(rng, 3)
        a = rng.standard_normal(3)
        b = rng.standard_normal(3)
        p += list(k) + list(map(float, a)) + list(map(float, b))
    return p


def fourier_speed_bound(params: Sequence[float], dim: int) -> float:
    """Upper bound of |u| for a Fourier velocity (sum of mode amplitudes); sets dt from a CFL."""
    nm = int(params[0])
    w = 4 if dim == 2 else 9
    s = 0.0
    for q in range(nm):
        m = np.asarray(params[1 + w * q: 1 + w * (q + 1)])
        if dim == 2:
            s += 2.0 * math.pi * float(np.hypot(m[0], m[1])) * float(np.hypot(m[2], m[3]))
        else:
            k, a, b = m[:3], m[3:6], m[6:9]
            s += 2.0 * math.pi * float(np.linalg.norm(k)) * (float(np.linalg.norm(a)) + float(np.linalg.norm(b)))
    return s


def fourier2d_max_speed(params: Sequence[float], n: int) -> float:
    """Largest speed |u| of a 2-D Fourier velocity over the nodes of an n x n grid of the unit
    square (u = d psi/dy, v = -d psi/dx of psi = sum a cos(2 pi k.x) + b sin(2 pi k.x))."""
    x, y = node_coords((n, n))
    u = np.zeros_like(x)
    v = np.zeros_like(x)
    nm = int(params[0])
    for q in range(nm):
        kx, ky, a, b = params[1 + 4 * q: 5 + 4 * q]
        th = 2.0 * math.pi * (kx * x + ky * y)
        dpsi = 2.0 * math.pi * (b * np.cos(th) - a * np.sin(th))
        u += ky * dpsi
        v -= kx * dpsi
    return float(np.sqrt(u * u + v * v).max())


def gaussian_and_step_2d(n: int) -> np.ndarray:
    x, y = node_coords((n, n))
    g = np.exp(-(_min_image(x - 0.3) ** 2 + _min_image(y - 0.3) ** 2) / (2 * 0.1 ** 2))
    s = (np.hypot(_min_image(x - 0.65), _min_image(y - 0.65)) < 0.2).astype(np.float64)
    return np.stack([g, s])


def batched_grids(count: int = 512, seed: int = 0, steps: int = 50, cfl: float = 4.0,
                  side_lo: int = 32, side_hi: int = 512, with_fields: bool = True) -> List[Workload]:
    """Independent 2-D periodic grids with sides log-uniform in [side_lo, side_hi], each with a
    steady divergence-free velocity from a random streamfunction of 8 Fourier modes
    (wavenumbers 1-4, N(0,1) amplitudes), a Gaussian and a step field; dt = cfl*dx/max|u|, the
    largest speed taken over the grid's nodes."""
    rng = np.random.default_rng(seed)
    sides = np.round(np.exp(rng.uniform(math.log(side_lo), math.log(side_hi), size=count))).astype(int)
    out = []
    for g, nside in enumerate(sides):
        r = np.random.default_rng([seed, g])
        p = fourier2d_params(r)
        vmax = fourier2d_max_speed(p, int(nside))
        dt = cfl / (nside * vmax)
        out.append(Workload(f"batch{g}_{nside}", 2, (int(nside), int(nside)), 2, "fourier2d", p, dt, steps,
                            fields=gaussian_and_step_2d(int(nside)) if with_fields else None))
    return out


# ---------------------------------------------------------------------------------------------
# Serving trace: Poisson arrivals of mixed 2-D / 3-D jobs
# ---------------------------------------------------------------------------------------------
@dataclass
class Job:
    job_id: int
    arrival_s: float
    workload: Workload
    dtype: str  # "f32" or "f64"


def job_fields(dim: int, n: int, nfields: int, seed: int) -> np.ndarray:
    """Initial fields of a served job: alternating Gaussians and balls at seeded centres."""
    rng = np.random.default_rng(seed)
    coords = node_coords((n,) * dim)
    planes = []
    for f in range(nfields):
        c = rng.uniform(0.2, 0.8, size=dim)
        r2 = sum(_min_image(coords[a] - c[a]) ** 2 for a in range(dim))
        if f % 2 == 0:
            planes.append(np.exp(-r2 / (2 * 0.1 ** 2)))
        else:
            planes.append((r2 < 0.15 ** 2).astype(np.float64))
    return np.stack(planes)


def job_fields_device(dim: int, n: int, nfields: int, seed: int, device="cuda", dtype=None):
    """job_fields evaluated with torch on `device` (same seeded centres and shapes), so that a server
    can create a large job's initial fields without stalling on the host."""
    import torch
    dtype = dtype or torch.float64
    rng = np.random.default_rng(seed)
    ax = torch.arange(n, device=device, dtype=torch.float64) / n
    coords = torch.meshgrid(*([ax] * dim), indexing="ij")  # (z, y, x) order: x is the last axis
    coords = list(reversed(coords))
    planes = []
    for f in range(nfields):
        c = rng.uniform(0.2, 0.8, size=dim)
        r2 = sum((coords[a] - c[a] - torch.round(coords[a] - c[a])) ** 2 for a in range(dim))
        planes.append(torch.exp(-r2 / (2 * 0.1 ** 2)) if f % 2 == 0 else (r2 < 0.15 ** 2).to(torch.float64))
    return torch.stack(planes).to(dtype)


def serving_trace(njobs: int = 2000, seed: int = 1, rate_hz: float = 200.0, frac_3d: float = 0.3,
                  frac_f64: float = 0.1, side2d=(64, 2048), side3d=(32, 192), steps=(10, 200),
                  cfl: float = 4.0) -> List[Job]:
    """Poisson stream of advection jobs: 2-D (side log-uniform in side2d) or 3-D (side3d),
    1-4 fields, a step count uniform in `steps`, random-Fourier divergence-free velocity, FP32 with
    a fraction frac_f64 asking for FP64.  Fields are generated on demand (job_fields)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for q in range(njobs):
        t += rng.exponential(1.0 / rate_hz)
        is3d = rng.uniform() < frac_3d
        lo, hi = side3d if is3d else side2d
        nside = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        nf = int(rng.integers(1, 5))
        ns = int(rng.integers(steps[0], steps[1] + 1))
        dtype = "f64" if rng.uniform() < frac_f64 else "f32"
        dim = 3 if is3d else 2
        p = fourier3d_params(rng) if is3d else fourier2d_params(rng)
        dt = cfl / (nside * fourier_speed_bound(p, dim))
        wl = Workload(f"job{q}", dim, (nside,) * dim, nf, "fourier3d" if is3d else "fourier2d", p, dt, ns)
        jobs.append(Job(q, t, wl, dtype))
    return jobs


# ---------------------------------------------------------------------------------------------
# Test inputs: smooth random displacements (in cell units) that do not fold the grid
# ---------------------------------------------------------------------------------------------
def smooth_displacement(n: Sequence[int], amplitude: float, seed: int, modes: int = 3,
                        shift: Sequence[float] | None = None) -> np.ndarray:
    """A periodic smooth displacement field of shape (*plane_shape, dim) in cell units: a uniform
    shift plus a few low Fourier modes whose largest gradient stays below `amplitude`."""
    rng = np.random.default_rng(seed)
    dim = len(n)
    coords = node_coords(tuple(n))
    shape = coords[0].shape
    D = np.zeros(shape + (dim,))
    for a in range(dim):
        acc = np.zeros(shape)
        for _ in range(modes):
            k = rng.integers(-2, 3, size=dim)
            if not np.any(k):
                k[0] = 1
            ph = rng.uniform(0, 2 * np.pi)
            amp = rng.uniform(0.5, 1.0)
            acc += amp * np.sin(2 * np.pi * sum(k[b] * coords[b] for b in range(dim)) + ph)
        # gradient in cells per cell of amp*sin(2 pi k.x): 2 pi |k| amp / n  -> scale to `amplitude`
        kmax = 2 * np.pi * 2.0 * math.sqrt(dim) * modes / min(n)
        D[..., a] = acc * (amplitude / kmax)
        if shift is not None:
            D[..., a] += shift[a]
    return D
