/*
 * sl.h -- C ABI of libsl.so, a GB300 (sm_103a) implementation of the forward semi-Lagrangian (FSL)
 * step of Becerra-Sagredo, Malaga & Mandujano, "Moments Preserving and high-resolution
 * Semi-Lagrangian Advection Scheme" (arXiv:1410.2817).
 *
 * The library solves the transport system Dh_f/Dt = 0 (Sec. 2, eq. momento with S = 0) for
 * `nfields` scalar fields carried by a moving material grid whose nodes follow a given velocity
 * u(x, t) (eq. vel).  One step:
 *   1. flags    -- jump criterion of Sec. 2.3 on the fields at the start of the step;
 *   2. advect   -- every Lagrangian node is moved from its reference position by one classical
 *                  RK4 step of eq. (vel);
 *   3. remap    -- every reference node is located in the deformed grid (Sec. 2.2 element search),
 *                  the multilinear element map (eq. mapping1, Z~0 geometry) is inverted by Newton's
 *                  method, the interpolation order is lowered near flagged nodes (Sec. 2.3) and the
 *                  tensor-product cardinal Z-spline sum (eq. multiZ, Appendix) gives the new value;
 *   4. reset    -- the remapped values become the fields on the reference mesh (Sec. 2).
 *
 * Conventions shared by every entry point
 *   - Grid: periodic box [lo, hi) per axis with n[a] nodes; node i sits at lo + i*(hi-lo)/n.
 *     A field plane is n[0]*n[1](*n[2]) contiguous values of the grid's dtype, x fastest
 *     (index = ix + n0*(iy + n1*iz)).  Field planes are caller-owned DEVICE memory.
 *   - Displacements D are stored in cell units (displacement / dx per axis).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is asynchronous on
 *     that stream unless its comment says "synchronises".
 *   - Errors: invalid arguments return SL_ERR_ARG before any work is queued; a failed CUDA call or
 *     launch returns SL_ERR_CUDA (text via sl_last_error()).  Kernels never trap: a target whose
 *     element search or Newton inversion fails keeps its old value and is counted in the grid's
 *     diagnostics (read with sl_get_diagnostics); with SL_FAIL_ERROR, sl_step additionally
 *     synchronises at its end and returns SL_ERR_LOCATE / SL_ERR_NEWTON / SL_ERR_FOLD.
 *   - Threading: one grid is used by one stream at a time.
 *   - The library allocates no device memory: every device buffer is either the caller's field
 *     planes or the caller-supplied workspace given to sl_create_grid.
 */
#ifndef SL_H
#define SL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SL_OK = 0,
    SL_ERR_ARG = 1,         /* invalid argument: NULL pointer, bad size, enum or alignment      */
    SL_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed                       */
    SL_ERR_NOMEM = 3,       /* workspace smaller than sl_grid_workspace_bytes()                  */
    SL_ERR_BUDGET = 4,      /* a batch does not fit the memory it was given                      */
    SL_ERR_LOCATE = 5,      /* some target's element search gave up after walk_max hops           */
    SL_ERR_NEWTON = 6,      /* some target's Newton inversion did not converge                    */
    SL_ERR_FOLD = 7,        /* some target met a folded element (det J <= 0)                      */
    SL_ERR_UNSUPPORTED = 8  /* valid but unimplemented combination of options                    */
} sl_status;

enum { SL_F64 = 0, SL_F32 = 1 };                       /* dtype of field planes and of D          */
enum {                                                 /* trajectory integrator (eq. vel)         */
    SL_RK4 = 0,             /* classical 4-stage Runge-Kutta                                        */
    SL_WRK3 = 1             /* Williamson's low-storage 3-stage, third-order Runge-Kutta (Sec. 2,
                               the paper's integrator): A = (0, -5/9, -153/128),
                               B = (1/3, 15/16, 8/15), stage times t, t + h/3, t + 3h/4            */
};
#define SL_MAX_SUBSTEPS 16                             /* trajectory sub-steps per remap (max)     */
enum {                                                 /* velocity u(x, t) of eq. (vel)           */
    SL_VEL_UNIFORM = 0,     /* params (u, v[, w])                                                   */
    SL_VEL_SOLID_BODY = 1,  /* params (Omega, cx, cy): u = Omega (cy - y, x - cx)      (Sec. 3.1) */
    SL_VEL_SWIRL2D = 2,     /* params (T): u = sin^2(pi x) sin(2pi y) cos(pi t/T),
                                           v = -sin^2(pi y) sin(2pi x) cos(pi t/T)               */
    SL_VEL_DEFORM3D = 3,    /* params (T): u = 2 sin^2(pi x) sin(2pi y) sin(2pi z) cos(pi t/T),
                                           v, w the cyclic permutations with amplitude -1        */
    SL_VEL_FOURIER2D = 4,   /* params (q, [kx ky a b] * q): u = d psi/dy, v = -d psi/dx with
                                           psi = sum a cos(2pi k.x) + b sin(2pi k.x), q <= 16    */
    SL_VEL_FOURIER3D = 5,   /* params (q, [k(3) a(3) b(3)] * q): u = curl of
                                           A = sum a cos(2pi k.x) + b sin(2pi k.x), q <= 8       */
    SL_VEL_CARRIED = 6,     /* params () or (f_x, f_y[, f_z]): the velocity is transported by the
                               nodes as fields f_a (default the first dim fields; Sec. 3.2, Burgers:
                               Du/Dt = 0, so each node moves on the straight line X + t u(X) and
                               every integrator gives D = dt u / dx).  The trajectories need the
                               fields: sl_step reads them at the start of each step, and
                               sl_advect_nodes_carried replaces sl_advect_nodes.  On the 2-D
                               tiled path (not the pipelined configuration 5) each remap launch
                               also writes the next step's D from its remapped velocity; not
                               batched.                                                         */
    SL_VEL_NLSW = 7         /* params (f0) or (f0, nu >= 0): the non-dimensional shallow-water system
                               of Sec. 3.3, eq. (nlsw), on a 2-D grid whose fields 0, 1, 2 are h,
                               u1, u2 (further fields are passive):
                                 Dh/Dt = -(1 + h) div u,
                                 Du/Dt = -grad h - f (-u2, u1) + nu div[(1 + h)(grad u + grad u^T)],
                                 f = f0 x2 (x2 the node's current position).
                               Each sl_step step runs the three stages of the low-storage RK3
                               (integrator must be SL_WRK3) on the nodes -- sources by differences
                               on the node lattice (second order for max_order <= 1, fourth order
                               for 2: the Z-spline derivative at the nodes), turned physical
                               through the Jacobian of the node positions; with nu > 0 a stress
                               pass precedes each stage -- then remaps once.  The workspace holds
                               13 extra planes.  sl_advect_nodes does not apply; not batched.   */
};
enum { SL_NEWTON_F64 = 0, SL_NEWTON_MIXED = 1 };       /* precision of the element-map inversion  */
enum { SL_FAIL_KEEP = 0, SL_FAIL_ERROR = 1 };          /* what a failed target reports             */
enum { SL_START_BACKWARD = 0, SL_START_PAPER = 1 };    /* first element of the search              */
enum { SL_KERNEL_AUTO = 0, SL_KERNEL_GENERIC = 1, SL_KERNEL_TILED = 2 };

typedef struct sl_grid sl_grid; /* opaque; host object that borrows the device workspace */

typedef struct {
    int dim;                        /* 2 or 3                                                       */
    int64_t n[3];                   /* nodes per axis (n[2] ignored in 2-D); each >= 4               */
    double lo[3], hi[3];            /* periodic box                                                  */
    int nfields;                    /* 1..8 fields advected together                                 */
    int dtype;                      /* SL_F64 or SL_F32                                              */
    int max_order;                  /* m_max of the Z-spline: 0 (linear), 1 (cubic) or 2 (quintic;
                                       tiled in 2-D FP32, plain kernels in 3-D and FP64)            */
    double limiter_threshold;       /* 0.25 in the paper (Sec. 2.3); < 0 disables the limiter        */
    int integrator;                 /* SL_RK4 or SL_WRK3                                             */
    int velocity_kind;              /* SL_VEL_*                                                      */
    const double *velocity_params;  /* host array, copied by sl_create_grid                          */
    int n_velocity_params;
    int newton_mode;                /* SL_NEWTON_F64 (any dtype) or SL_NEWTON_MIXED (SL_F32 only).
                                       SL_F32 with SL_NEWTON_F64 inverts every target in FP64: on
                                       the blocked kernel in 3-D, on the plain kernels in 2-D   */
    int newton_max_iter;            /* <= 0 selects 8                                                */
    int walk_max;                   /* <= 0 selects 64                                               */
    int fail_policy;                /* SL_FAIL_KEEP or SL_FAIL_ERROR                                  */
    int walk_start;                 /* SL_START_BACKWARD (from j - D_j) or SL_START_PAPER (Sec. 2.2) */
    int kernel;                     /* SL_KERNEL_AUTO, SL_KERNEL_GENERIC or SL_KERNEL_TILED           */
    int tile_config;                /* 2-D FP32 tiles: 0 default (7 where it applies, else 1);
                                       6: 64x32 and 7: 32x32 tiles of the persistent kernel whose
                                       windows are copied by TMA boxes (one CTA per SM with 6, two
                                       with 7; up to 3 fields, max_order <= 1, an analytic velocity,
                                       even n[0], 16-byte aligned planes, else 1);
                                       1: 32x32, 2: 32x16, 3: 64x16, 4: 32x16 compiled for 4 CTAs
                                       per SM, 5: 32x32 pipelined (persistent, one CTA per SM
                                       staging the next tiles while it computes; 1 above 4
                                       fields) -- the shared-memory tile kernels with per-element
                                       copies.  Batches take their own tile configuration (0..5).
                                       3-D FP32 grids: 1 runs the blocked kernel, which gathers
                                       every value through L1; any other value runs plain remaps
                                       on the staged kernel (the field values of each 16x4x4
                                       target block's stencils copied to shared memory during the
                                       element search: TMA boxes inside the grid, per-element
                                       copies across the seam) where it applies -- up to 2
                                       fields, newton_mode other than SL_NEWTON_F64 -- and fused
                                       steps on the blocked kernel.  Both give identical results. */
    int trajectory_substeps;        /* integrator steps per remap (Sec. 2: the Lagrangian grid may
                                       move for several time steps before the fields are
                                       interpolated back): each step of length dt integrates the
                                       trajectories with this many sub-steps of dt / substeps, then
                                       remaps once.  <= 0 selects 1; at most SL_MAX_SUBSTEPS.   */
} sl_grid_desc;

/* Counters accumulated on the device since creation or the last sl_reset_diagnostics. */
typedef struct {
    uint64_t targets;               /* target-node remaps performed                                  */
    uint64_t fail_locate;           /* element search gave up                                        */
    uint64_t fail_newton;           /* Newton hit its iteration cap inside the element               */
    uint64_t fail_fold;             /* det J <= 0                                                    */
    uint64_t hops_sum, hops_max;    /* element-search hops (Newton solves) per target                */
    uint64_t iters_sum, iters_max;  /* Newton iterations per target                                  */
    uint64_t newton_f64;            /* (mixed mode) targets re-solved in FP64                        */
    uint64_t order_hist[3];         /* field-targets interpolated with order 0, 1, 2                 */
    uint64_t tiles_fallback;        /* tiles whose stencil window did not fit shared memory          */
    uint64_t kernel_launches;       /* kernels this grid's calls have launched (host-side count)    */
    uint64_t timeouts;              /* bounded waits for shared-memory copies that ran out (the CTA
                                       stopped; its targets are left unwritten) -- expected 0      */
} sl_diag;

/* Remap debug outputs (device pointers, each may be NULL). */
typedef struct {
    int64_t *cell;                  /* [N] wrapped linear index of the element's lower corner, -1 = failed */
    double *xi;                     /* [N*dim] local coordinates in the element (always FP64)        */
    uint8_t *order;                 /* [nfields*N] order used per field (255 = failed target)        */
    uint8_t *status;                /* [N] 0 ok, 1 locate, 2 newton, 3 fold                          */
} sl_remap_debug;

/* Bytes of device workspace a grid needs (two displacement buffers, flags, counters and their
 * per-SM copies, reduction scratch; for the swirl and the deformation flow, sin(pi x) and
 * cos(pi x) at the node coordinates).  Returns 0 for an invalid descriptor. */
size_t sl_grid_workspace_bytes(const sl_grid_desc *desc);

/* Create a grid (Sec. 2: reference mesh plus Lagrangian grid).  `dev_workspace` is caller-owned
 * device memory of at least sl_grid_workspace_bytes(desc) bytes, 256-byte aligned; the grid
 * borrows it until sl_destroy_grid.  Zeroes the counters and the displacement and fills the sin/cos
 * tables (synchronises). */
sl_status sl_create_grid(const sl_grid_desc *desc, void *dev_workspace, size_t ws_bytes, sl_grid **out);
sl_status sl_destroy_grid(sl_grid *grid);

/* eq. (vel): move every Lagrangian node from its reference position over [t, t+dt] with the grid's
 * integrator (trajectory_substeps steps of RK4 or of the low-storage RK3) in the grid's analytic
 * velocity; writes the grid's current displacement D (cell units).  SL_ERR_ARG for a carried
 * velocity (it needs the fields: sl_advect_nodes_carried). */
sl_status sl_advect_nodes(sl_grid *grid, double t, double dt, void *stream);

/* Sec. 3.2: trajectories of a grid whose velocity is carried (SL_VEL_CARRIED): every node moves
 * over dt with the velocity it holds in the field planes `fields` (nfields device pointers, the
 * grid's dtype; only the velocity components are read): D_i = dt u_i / dx in cell units, written
 * to the grid's current displacement.  SL_ERR_ARG for any other velocity kind. */
sl_status sl_advect_nodes_carried(sl_grid *grid, const void *const *fields, double dt, void *stream);

/* Sec. 2 reset / Sec. 2.2-2.3 / eq. (multiZ): with the current D, compute the jump flags of `in`,
 * locate every reference node, invert the element map, choose the order and interpolate.
 * `in`, `out`: host arrays of nfields device pointers; in and out must not overlap. */
sl_status sl_remap_fields(sl_grid *grid, const void *const *in, void *const *out, void *stream);

/* Same as sl_remap_fields, additionally writing per-target diagnostics (any pointer may be NULL). */
sl_status sl_remap_fields_debug(sl_grid *grid, const void *const *in, void *const *out,
                                const sl_remap_debug *dbg, void *stream);

/* nsteps full steps (flags, advect, remap, reset) starting at time t0.  `fields`: nfields device
 * planes, updated in place; `scratch`: nfields device planes of the same size used as the other
 * half of a ping-pong pair (contents undefined afterwards).  On the fused FP32 path the grid's
 * current D afterwards holds the displacement of the step that follows (t0 + nsteps*dt), and a
 * next call starting there with the same dt does not integrate it again. */
sl_status sl_step(sl_grid *grid, void *const *fields, void *const *scratch, double t0, double dt, int nsteps,
                  void *stream);

/* The same steps out of place: `in` (nfields device planes, read only) is advanced nsteps steps
 * and the result written to `out`; `scratch` (nfields planes) is the other half of the ping-pong
 * for nsteps > 1 and may be NULL for nsteps <= 1.  in, out and scratch must not overlap.  One step
 * on the fused FP32 path is one launch, with no copy back (a shallow-water grid copies `in` to
 * `out` first and advances it in place).  The carried displacement and SL_FAIL_ERROR behave as
 * in sl_step. */
sl_status sl_step_out(sl_grid *grid, const void *const *in, void *const *out, void *const *scratch, double t0, double dt,
                      int nsteps, void *stream);

/* Sec. 3.1: discrete moments of one field plane about the box centre c:
 * m_0 = sum h,  m_p = sum_i h_i sum_a (x_a^i - c_a)^p for 1 <= p <= pmax (<= 7), accumulated in
 * FP64 in a fixed order.  Writes pmax+1 doubles to host_out (synchronises). */
sl_status sl_moments(sl_grid *grid, const void *field, int pmax, double *host_out, void *stream);

/* Discrete moments (as sl_moments) of one field plane, for callers that cannot allocate device
 * memory: a host program whose allocator owns all device memory and forbids other allocations,
 * code on a real-time path where cudaMalloc/cudaFree would synchronise the device, or a caller
 * that only holds the field plane it was handed.  It needs no grid and no workspace and
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).  The paper has no
 * counterpart: this is a calling convenience.
 *   dim, n, lo, hi, dtype: the grid of `field` (as in sl_grid_desc); field: device plane.
 *   pmax: 0..7; host_out: pmax+1 doubles.  Synchronises `stream`.
 * Its scratch is a fixed file-scope device array of 512 x 8 + 8 doubles (about 33 KB) that every
 * GPU loading the library holds until the process exits.  pmax above 7 (the moments a scratch
 * row holds) or more than 2^31 - 1 nodes returns SL_ERR_ARG.  Every call on a device shares the
 * array and leaves its contents behind; each call overwrites everything it reads, so nothing
 * needs clearing, but calls whose kernels overlap on the GPU (different streams, no ordering)
 * race on it and must be serialised by the caller.  The array's device address is looked up
 * (cudaGetSymbolAddress, with the device current) on every call made outside stream capture, so
 * a reset of the device's primary context between calls is harmless; a call made while `stream`
 * is being captured reuses the address the last uncaptured call on that device found, so make at
 * least one call on each device before capturing one (otherwise SL_ERR_CUDA).  A rejected call
 * leaves its reason in sl_last_error(). */
sl_status sl_moments_noalloc(int dim, const int64_t n[3], const double lo[3], const double hi[3], int dtype,
                             const void *field, int pmax, double *host_out, void *stream);

/* ---- Batches: many independent 2-D FP32 grids advanced together ---------------------------
 * A batch advances count grids (created with sl_create_grid, 2-D, SL_F32 with SL_NEWTON_MIXED, the
 * same nfields <= 4, backward walk start, an analytic velocity with any integrator and sub-step count; either all of
 * max_order <= 1 or all quintic, max_order 2, whose tiles are 32 x 32 whatever tile_config) by the
 * same number of steps with one persistent launch per step over a work-list of (grid, tile)
 * items: each item is the single-grid tiled step of that tile (Sec. 2.1-2.3, eq. multiZ, eq. vel).  Grids keep their own workspaces (displacements and
 * counters).  The batch's device state (grid table, work-list, per-step work counters, grid
 * times) lives in a caller-owned workspace of sl_batch_workspace_bytes() bytes (256-byte
 * aligned); the library allocates no device memory. */
typedef struct sl_batch sl_batch;

/* Workspace bytes of a batch of these grids with tile configuration tile_config (0..5, as in
 * sl_grid_desc); 0 if a grid is not eligible. */
size_t sl_batch_workspace_bytes(sl_grid *const *grids, int count, int tile_config);

/* fields[q], scratch[q]: host arrays of nfields device planes of grid q (the planes are
 * borrowed; scratch contents are undefined after a step).  t0[q], dt[q]: grid q's time and step.
 * Copies the grid table to the device (synchronises).  Returns SL_ERR_UNSUPPORTED for
 * ineligible grids and SL_ERR_NOMEM for a short workspace. */
sl_status sl_batch_create(sl_grid *const *grids, int count, void *const *const *fields, void *const *const *scratch,
                          const double *t0, const double *dt, int tile_config, void *dev_workspace, size_t ws_bytes,
                          sl_batch **out);

/* nsteps full steps of every grid (fields updated in place; each grid's time advances by
 * nsteps*dt on the device).  use_graph != 0: the launch sequence of this step count is captured
 * once into a CUDA graph and replayed (needs a non-NULL stream; make the first such call outside
 * any other capture).  Calls on one batch must not overlap. */
sl_status sl_batch_step(sl_batch *batch, int nsteps, int use_graph, void *stream);

/* Work items per step, kernels launched so far, and the first grid's time (host mirror). */
sl_status sl_batch_info(const sl_batch *batch, int *nitems, unsigned long long *launches, double *t_first);
sl_status sl_batch_destroy(sl_batch *batch);

/* Jump flags of Sec. 2.3 for `fields` into flags_out (device, N bytes; bit f for field f). */
sl_status sl_compute_flags(sl_grid *grid, const void *const *fields, uint8_t *flags_out, void *stream);

/* Copy a displacement (device memory, grid dtype, `stride` values per node >= dim, cell units)
 * into / out of the grid's current D. */
sl_status sl_set_displacement(sl_grid *grid, const void *D, int64_t stride, void *stream);
sl_status sl_get_displacement(sl_grid *grid, void *D_out, int64_t stride, void *stream);

/* Read (synchronises) or zero the device counters. */
sl_status sl_get_diagnostics(sl_grid *grid, sl_diag *out, void *stream);
sl_status sl_reset_diagnostics(sl_grid *grid, void *stream);

const char *sl_status_string(sl_status status);
/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char *sl_last_error(void);
/* Version string of the library build. */
const char *sl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SL_H */
