// sl_api.cu -- the extern "C" entry points declared in include/sl.h: argument checks, carving of
// the caller's workspace, and dispatch to the kernels.  The library never allocates device memory.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "sl_internal.h"

static thread_local char g_last_error[512];

static sl_status fail_cuda(cudaError_t e, const char *where)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return SL_ERR_CUDA;
}

static sl_status fail_arg(const char *why)
{
    snprintf(g_last_error, sizeof(g_last_error), "invalid argument: %s", why);
    return SL_ERR_ARG;
}

#define SL_CUDA(call, where)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return fail_cuda(e_, where);   \
    } while (0)

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------------------------------------
// descriptor validation
// ------------------------------------------------------------------------------------------------
static const char *check_desc(const sl_grid_desc *d)
{
    if (!d) return "descriptor is NULL";
    if (d->dim != 2 && d->dim != 3) return "dim must be 2 or 3";
    long long N = 1;
    for (int a = 0; a < d->dim; ++a) {
        if (d->n[a] < 4 || d->n[a] > (1 << 20)) return "each n[a] must be in [4, 2^20]";
        if (!(d->hi[a] > d->lo[a])) return "hi must exceed lo on every axis";
        N *= d->n[a];
    }
    if (N > (1LL << 31) - 1) return "too many nodes (limit 2^31 - 1)";
    if (d->nfields < 1 || d->nfields > SL_MAX_FIELDS) return "nfields must be in [1, 8]";
    if (d->dtype != SL_F64 && d->dtype != SL_F32) return "dtype must be SL_F64 or SL_F32";
    if (d->max_order < 0 || d->max_order > 2) return "max_order must be 0, 1 or 2";
    if (d->integrator != SL_RK4 && d->integrator != SL_WRK3) return "integrator must be SL_RK4 or SL_WRK3";
    if (d->trajectory_substeps > SL_MAX_SUBSTEPS) return "trajectory_substeps must be <= SL_MAX_SUBSTEPS";
    if (d->newton_mode != SL_NEWTON_F64 && d->newton_mode != SL_NEWTON_MIXED) return "bad newton_mode";
    if (d->newton_mode == SL_NEWTON_MIXED && d->dtype != SL_F32) return "SL_NEWTON_MIXED needs dtype SL_F32";
    if (d->fail_policy != SL_FAIL_KEEP && d->fail_policy != SL_FAIL_ERROR) return "bad fail_policy";
    if (d->walk_start != SL_START_BACKWARD && d->walk_start != SL_START_PAPER) return "bad walk_start";
    if (d->kernel < SL_KERNEL_AUTO || d->kernel > SL_KERNEL_TILED) return "bad kernel";
    if (d->tile_config < 0 || d->tile_config > 7) return "tile_config must be in [0, 7]";
    if (d->newton_max_iter > 64 || d->walk_max > 4096) return "newton_max_iter <= 64 and walk_max <= 4096";
    const int np = d->n_velocity_params;
    if (np < 0 || np > SL_MAX_VEL_PARAMS) return "n_velocity_params out of range";
    if (np > 0 && !d->velocity_params) return "velocity_params is NULL";
    const double *p = d->velocity_params;
    switch (d->velocity_kind) {
    case SL_VEL_UNIFORM:
        if (np < d->dim) return "uniform velocity needs dim parameters";
        break;
    case SL_VEL_SOLID_BODY:
        if (d->dim != 2 || np < 3) return "solid-body rotation is 2-D with 3 parameters";
        break;
    case SL_VEL_SWIRL2D:
        if (d->dim != 2 || np < 1 || !(p[0] != 0.0)) return "swirl is 2-D with a nonzero period";
        break;
    case SL_VEL_DEFORM3D:
        if (d->dim != 3 || np < 1 || !(p[0] != 0.0)) return "3-D deformation is 3-D with a nonzero period";
        break;
    case SL_VEL_FOURIER2D: {
        if (d->dim != 2 || np < 1) return "fourier2d is 2-D";
        const int q = (int)p[0];
        if ((double)q != p[0] || q < 1 || q > 16 || np < 1 + 4 * q) return "fourier2d needs 1..16 modes of 4 values";
        break;
    }
    case SL_VEL_FOURIER3D: {
        if (d->dim != 3 || np < 1) return "fourier3d is 3-D";
        const int q = (int)p[0];
        if ((double)q != p[0] || q < 1 || q > 8 || np < 1 + 9 * q) return "fourier3d needs 1..8 modes of 9 values";
        break;
    }
    case SL_VEL_CARRIED: {
        if (np != 0 && np != d->dim) return "carried velocity takes no parameter or one field index per axis";
        if (np == 0 && d->nfields < d->dim) return "carried velocity needs dim fields";
        for (int a = 0; a < np; ++a) {
            // range first: the integer test converts to int only once p[a] is known to fit
            if (!isfinite(p[a]) || p[a] < 0 || p[a] >= d->nfields || p[a] != floor(p[a]))
                return "carried velocity field indices must be integers in [0, nfields)";
            for (int b = 0; b < a; ++b)
                if (p[b] == p[a]) return "carried velocity field indices must be distinct";
        }
        break;
    }
    case SL_VEL_NLSW:
        if (d->dim != 2 || d->nfields < 3) return "nlsw is 2-D with at least 3 fields (h, u1, u2)";
        if (np != 1 && np != 2) return "nlsw takes f0 and optionally the viscosity nu";
        if (np == 2 && !(p[1] >= 0.0)) return "nlsw viscosity must be >= 0";
        if (d->integrator != SL_WRK3 || d->trajectory_substeps > 1)
            return "nlsw integrates with SL_WRK3, one step per remap";
        break;
    default:
        return "unknown velocity_kind";
    }
    for (int q = 0; q < np; ++q)
        if (!isfinite(p[q])) return "velocity parameters must be finite";
    return nullptr;
}

struct Layout {
    size_t counters, stripes, trig, partials, moment_out, flags, flags2, D0, D1, rk, total;
};

static Layout layout_of(const sl_grid_desc *d)
{
    Layout L;
    long long N = 1;
    for (int a = 0; a < d->dim; ++a) N *= d->n[a];
    const size_t ts = d->dtype == SL_F64 ? 8 : 4;
    const size_t ds = d->dim == 2 ? 2 : 4;
    size_t off = 0;
    L.counters = off;
    off += align256(sizeof(DevCounters));
    L.stripes = off;
    off += align256(sizeof(DevCounters) * SL_COUNTER_STRIPES);
    L.trig = off;
    if (d->velocity_kind == SL_VEL_SWIRL2D || d->velocity_kind == SL_VEL_DEFORM3D) {
        long long nt = 0;
        for (int a = 0; a < d->dim; ++a) nt += d->n[a];
        off += align256((size_t)nt * 2 * ts);
    }
    L.partials = off;
    off += align256(sizeof(double) * 8 * SL_MOMENT_BLOCKS);
    L.moment_out = off;
    off += align256(sizeof(double) * 8);
    L.flags = off;
    off += align256((size_t)N);
    L.flags2 = off;
    off += align256((size_t)N);
    L.D0 = off;
    off += align256((size_t)N * ds * ts);
    L.D1 = off;
    off += align256((size_t)N * ds * ts);
    // shallow water: two sets of RK3 registers of h, u1, u2 and of the displacement, and the
    // viscous stress (13 planes)
    L.rk = off;
    if (d->velocity_kind == SL_VEL_NLSW) off += align256((size_t)N * 13 * ts);
    L.total = off;
    return L;
}

extern "C" size_t sl_grid_workspace_bytes(const sl_grid_desc *desc)
{
    if (check_desc(desc)) return 0;
    return layout_of(desc).total;
}

extern "C" sl_status sl_create_grid(const sl_grid_desc *desc, void *dev_workspace, size_t ws_bytes, sl_grid **out)
{
    if (!out) return fail_arg("out is NULL");
    *out = nullptr;
    if (const char *why = check_desc(desc)) return fail_arg(why);
    if (!dev_workspace) return fail_arg("workspace is NULL");
    if (((uintptr_t)dev_workspace & 255u) != 0) return fail_arg("workspace must be 256-byte aligned");
    const Layout L = layout_of(desc);
    if (ws_bytes < L.total) {
        snprintf(g_last_error, sizeof(g_last_error), "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
        return SL_ERR_NOMEM;
    }
    sl_grid *g = (sl_grid *)calloc(1, sizeof(sl_grid));
    if (!g) return fail_arg("host allocation of the grid object failed");
    g->desc = *desc;
    memset(g->vel_params, 0, sizeof(g->vel_params));
    for (int q = 0; q < desc->n_velocity_params; ++q) g->vel_params[q] = desc->velocity_params[q];
    g->desc.velocity_params = g->vel_params;
    if (g->desc.newton_max_iter <= 0) g->desc.newton_max_iter = 8;
    if (g->desc.walk_max <= 0) g->desc.walk_max = 64;
    g->dim = desc->dim;
    g->nfields = desc->nfields;
    g->dtype = desc->dtype;
    g->ds = desc->dim == 2 ? 2 : 4;
    g->tsize = desc->dtype == SL_F64 ? 8 : 4;
    g->N = 1;
    for (int a = 0; a < 3; ++a) {
        g->n[a] = a < desc->dim ? desc->n[a] : 1;
        g->N *= g->n[a];
        g->dx[a] = a < desc->dim ? (desc->hi[a] - desc->lo[a]) / (double)desc->n[a] : 1.0;
    }
    g->ws = (char *)dev_workspace;
    g->ws_bytes = ws_bytes;
    g->counters = (DevCounters *)(g->ws + L.counters);
    g->stripes = (DevCounters *)(g->ws + L.stripes);
    g->trig = nullptr;
    if (desc->velocity_kind == SL_VEL_SWIRL2D || desc->velocity_kind == SL_VEL_DEFORM3D) {
        g->trig = g->ws + L.trig;
        long long o = 0;
        for (int a = 0; a < 3; ++a) {
            g->trig_off[a] = o;
            if (a < desc->dim) o += 2 * desc->n[a];
        }
    }
    g->partials = (double *)(g->ws + L.partials);
    g->moment_out = (double *)(g->ws + L.moment_out);
    g->flags = (uint8_t *)(g->ws + L.flags);
    g->flags2 = (uint8_t *)(g->ws + L.flags2);
    g->D[0] = g->ws + L.D0;
    g->D[1] = g->ws + L.D1;
    g->dcur = 0;
    const int vk = desc->velocity_kind;
    g->steady = vk == SL_VEL_UNIFORM || vk == SL_VEL_SOLID_BODY || vk == SL_VEL_FOURIER2D || vk == SL_VEL_FOURIER3D;
    g->carried = vk == SL_VEL_CARRIED;
    g->nlsw = vk == SL_VEL_NLSW;
    g->rk = vk == SL_VEL_NLSW ? (void *)(g->ws + L.rk) : nullptr;
    for (int a = 0; a < 3; ++a)
        g->vel_field[a] = (g->carried && desc->n_velocity_params > a) ? (int)desc->velocity_params[a] : a;
    g->d_cached = 0;
    g->next_valid = 0;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->ws, 0, L.total, 0);
    if (e == cudaSuccess) e = launch_trig_tables(g, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        free(g);
        return fail_cuda(e, "sl_create_grid");
    }
    *out = g;
    return SL_OK;
}

extern "C" sl_status sl_destroy_grid(sl_grid *grid)
{
    if (!grid) return fail_arg("grid is NULL");
    free(grid);
    return SL_OK;
}

static sl_status check_planes(const sl_grid *g, const void *const *p, const char *what)
{
    if (!p) return fail_arg(what);
    for (int q = 0; q < g->nfields; ++q) {
        if (!p[q]) return fail_arg(what);
        if (((uintptr_t)p[q] % g->tsize) != 0) return fail_arg("field plane is not aligned to its dtype");
    }
    return SL_OK;
}

template <typename T>
static bool use_tiled(const sl_grid *g)
{
    if (g->desc.kernel == SL_KERNEL_GENERIC) return false;
    if (g->desc.kernel == SL_KERNEL_AUTO && g->dtype != SL_F32) return false;  // AUTO: tiled serves FP32
    return Launch<T>::tiled_supported(g);
}

// count launches: every launcher below starts exactly `k` kernels when it succeeds
static cudaError_t counted(sl_grid *g, cudaError_t e, int k)
{
    if (e == cudaSuccess) g->launches += (unsigned long long)k;
    return e;
}

extern "C" sl_status sl_advect_nodes(sl_grid *g, double t, double dt, void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (!isfinite(t) || !isfinite(dt)) return fail_arg("t and dt must be finite");
    if (g->carried) return fail_arg("a carried velocity needs the fields: call sl_advect_nodes_carried");
    if (g->nlsw) return fail_arg("shallow-water grids move their nodes inside sl_step");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = g->dtype == SL_F64 ? Launch<double>::advect(g, g->D[g->dcur], t, dt, s)
                                       : Launch<float>::advect(g, g->D[g->dcur], t, dt, s);
    e = counted(g, e, 1);
    g->d_cached = e == cudaSuccess && g->steady;
    g->d_cached_dt = dt;
    g->next_valid = 0;
    return e == cudaSuccess ? SL_OK : fail_cuda(e, "sl_advect_nodes");
}

extern "C" sl_status sl_advect_nodes_carried(sl_grid *g, const void *const *fields, double dt, void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (!g->carried) return fail_arg("the grid's velocity is not carried by its fields");
    if (sl_status st = check_planes(g, fields, "field planes")) return st;
    if (!isfinite(dt)) return fail_arg("dt must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = g->dtype == SL_F64 ? Launch<double>::advect_carried(g, fields, g->D[g->dcur], dt, s)
                                       : Launch<float>::advect_carried(g, fields, g->D[g->dcur], dt, s);
    e = counted(g, e, 1);
    g->d_cached = 0;
    g->next_valid = 0;
    return e == cudaSuccess ? SL_OK : fail_cuda(e, "sl_advect_nodes_carried");
}

template <typename T>
static cudaError_t remap_impl(sl_grid *g, const void *D, const void *const *in, void *const *out,
                              const sl_remap_debug *dbg, cudaStream_t s)
{
    if (!dbg && use_tiled<T>(g)) return counted(g, Launch<T>::remap_tiled(g, D, in, out, s), tiled_kernels_per_call(g));
    cudaError_t e = counted(g, Launch<T>::flags(g, in, g->flags, s), 1);
    if (e != cudaSuccess) return e;
    return counted(g, Launch<T>::remap_generic(g, D, g->flags, in, out, dbg, s), 1);
}

static sl_status remap_entry(sl_grid *g, const void *const *in, void *const *out, const sl_remap_debug *dbg,
                             void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (sl_status st = check_planes(g, in, "input planes")) return st;
    if (sl_status st = check_planes(g, (const void *const *)out, "output planes")) return st;
    for (int q = 0; q < g->nfields; ++q)
        for (int r = 0; r < g->nfields; ++r)
            if (in[q] == out[r]) return fail_arg("input and output planes must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    const void *D = g->D[g->dcur];
    cudaError_t e = g->dtype == SL_F64 ? remap_impl<double>(g, D, in, out, dbg, s)
                                       : remap_impl<float>(g, D, in, out, dbg, s);
    return e == cudaSuccess ? SL_OK : fail_cuda(e, "sl_remap_fields");
}

extern "C" sl_status sl_remap_fields(sl_grid *g, const void *const *in, void *const *out, void *stream)
{
    return remap_entry(g, in, out, nullptr, stream);
}

extern "C" sl_status sl_remap_fields_debug(sl_grid *g, const void *const *in, void *const *out,
                                           const sl_remap_debug *dbg, void *stream)
{
    if (!dbg) return fail_arg("debug block is NULL");
    return remap_entry(g, in, out, dbg, stream);
}

// the grid's counters: the main copy and the per-SM stripes, summed (maxima for the two maxima)
static sl_status read_counters(sl_grid *g, DevCounters *c, cudaStream_t s)
{
    static thread_local DevCounters st[SL_COUNTER_STRIPES];
    SL_CUDA(cudaMemcpyAsync(c, g->counters, sizeof(DevCounters), cudaMemcpyDeviceToHost, s), "read counters");
    SL_CUDA(cudaMemcpyAsync(st, g->stripes, sizeof(st), cudaMemcpyDeviceToHost, s), "read counters");
    SL_CUDA(cudaStreamSynchronize(s), "read counters");
    for (int k = 0; k < SL_COUNTER_STRIPES; ++k) {
        const DevCounters &d = st[k];
        c->targets += d.targets;
        c->fail_locate += d.fail_locate;
        c->fail_newton += d.fail_newton;
        c->fail_fold += d.fail_fold;
        c->hops_sum += d.hops_sum;
        c->hops_max = std::max(c->hops_max, d.hops_max);
        c->iters_sum += d.iters_sum;
        c->iters_max = std::max(c->iters_max, d.iters_max);
        c->newton_f64 += d.newton_f64;
        for (int q = 0; q < 3; ++q) c->order_hist[q] += d.order_hist[q];
        c->tiles_fallback += d.tiles_fallback;
        c->timeouts += d.timeouts;
    }
    return SL_OK;
}

// nsteps full steps.  Step k reads src_k and writes dst_k: src_0 = in, dst_0 = A, and the
// destinations alternate A, B, A, ... (src_{k+1} = dst_k), so the result ends in A after an odd
// number of steps and in B after an even one.  `in` is read only by the first step; B may equal
// `in` (sl_step's in-place ping-pong).  A shallow-water grid advances `in` in place through its
// stages and remap (A, B unused except as the stages' scratch: see below).
template <typename T>
static cudaError_t step_impl(sl_grid *g, const void *const *in, void *const *A, void *const *B, double t0, double dt,
                             int nsteps, cudaStream_t s)
{
    const void *cur[SL_MAX_FIELDS];
    void *nxt[SL_MAX_FIELDS];
    for (int q = 0; q < g->nfields; ++q) {
        cur[q] = in[q];
        nxt[q] = A[q];
    }
    // after a step: its destination is the next source, the other buffer the next destination
    // (B may be NULL for a single out-of-place step: nothing is written after the last step)
    auto advance = [&]() {
        const bool wasA = nxt[0] == A[0];
        for (int q = 0; q < g->nfields; ++q) {
            cur[q] = nxt[q];
            nxt[q] = wasA ? (B ? B[q] : nullptr) : A[q];
        }
    };
    cudaError_t e = cudaSuccess;
    if (g->nlsw) {
        // the three RK3 stages on the nodes (four launches; the node values end in A), then the
        // remap back into `in`'s planes: the result lands in `in` after every step (the caller
        // passes writable planes there)
        g->d_cached = 0;
        g->next_valid = 0;
        void *const *fields = (void *const *)in;
        for (int k = 0; k < nsteps; ++k) {
            e = counted(g, Launch<T>::nlsw_stages(g, in, A, g->D[g->dcur], g->D[g->dcur ^ 1], dt, s),
                        nlsw_kernels_per_step(g));
            if (e == cudaSuccess) e = remap_impl<T>(g, g->D[g->dcur], (const void *const *)A, fields, nullptr, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const bool carried = g->carried != 0;
    if (carried && use_tiled<T>(g) && (g->desc.max_order == 2 || g->desc.tile_config != 5)) {
        // a carried velocity (Sec. 3.2) is the fields' own: the first step's D comes from the
        // fields, each later one from the remapped velocity of the step before, written by the
        // remap launch itself (the 2-D tiled kernels except the pipelined configuration).  The
        // caller may change the fields between calls, so nothing is carried over to the next call.
        g->d_cached = 0;
        g->next_valid = 0;
        e = counted(g, Launch<T>::advect_carried(g, cur, g->D[g->dcur], dt, s), 1);
        if (e != cudaSuccess) return e;
        for (int k = 0; k < nsteps; ++k) {
            const double t = t0 + (double)k * dt;
            const int nx = g->dcur ^ 1;
            void *dnext = k + 1 < nsteps ? g->D[nx] : nullptr;
            e = counted(g, Launch<T>::step_fused(g, g->D[g->dcur], dnext, t + dt, dt, cur, nxt, s),
                        tiled_kernels_per_call(g));
            if (e != cudaSuccess) return e;
            if (dnext) g->dcur = nx;
            advance();
        }
        return cudaSuccess;
    }
    // otherwise a carried velocity is read from the fields at the start of each step by its own
    // launch before the remap
    const bool fused = use_tiled<T>(g) && !carried;
    // steady velocity: one integration serves every step (and later calls with the same dt)
    const bool reuse = g->steady != 0;
    if (reuse && !(g->d_cached && g->d_cached_dt == dt)) {
        e = counted(g, Launch<T>::advect(g, g->D[g->dcur], t0, dt, s), 1);
        if (e != cudaSuccess) return e;
        g->d_cached = 1;
        g->d_cached_dt = dt;
    }
    if (fused && !reuse) {
        // the velocity is given, so D of the next step does not depend on the fields: each fused
        // launch remaps with D[cur] and writes D[next] for its own nodes -- the last one too, for
        // the step after this call.  D of this call's first step was left by the previous call
        // when its velocity arguments are bit-identical; otherwise it is integrated here.
        const VelArgs<float> v0 = make_vel_args<float>(g, t0, dt);
        const bool have = g->next_valid && memcmp(&v0, &g->next_vel, sizeof(v0)) == 0;
        g->next_valid = 0;
        if (!have) {
            e = counted(g, Launch<T>::advect(g, g->D[g->dcur], t0, dt, s), 1);
            if (e != cudaSuccess) return e;
        }
        g->d_cached = 0;
    }
    for (int k = 0; k < nsteps; ++k) {
        const double t = t0 + (double)k * dt;
        if (fused) {
            const int nx = g->dcur ^ 1;
            void *dnext = !reuse ? g->D[nx] : nullptr;
            e = counted(g, Launch<T>::step_fused(g, g->D[g->dcur], dnext, t + dt, dt, cur, nxt, s),
                        tiled_kernels_per_call(g));
            if (e != cudaSuccess) return e;
            if (dnext) {
                g->dcur = nx;
                if (k + 1 == nsteps) {
                    g->next_vel = make_vel_args<float>(g, t + dt, dt);
                    g->next_valid = 1;
                }
            }
        } else if (carried) {
            e = counted(g, Launch<T>::advect_carried(g, cur, g->D[g->dcur], dt, s), 1);
            g->d_cached = 0;
            g->next_valid = 0;
            if (e == cudaSuccess) e = remap_impl<T>(g, g->D[g->dcur], cur, nxt, nullptr, s);
            if (e != cudaSuccess) return e;
        } else {
            e = counted(g, Launch<T>::flags(g, cur, g->flags, s), 1);
            if (e == cudaSuccess && !reuse) {
                e = counted(g, Launch<T>::advect(g, g->D[g->dcur], t, dt, s), 1);
                g->d_cached = 0;
                g->next_valid = 0;
            }
            if (e == cudaSuccess)
                e = counted(g, Launch<T>::remap_generic(g, g->D[g->dcur], g->flags, cur, nxt, nullptr, s), 1);
            if (e != cudaSuccess) return e;
        }
        advance();
    }
    return cudaSuccess;
}

static sl_status check_step_args(const sl_grid *g, int nsteps, double t0, double dt)
{
    if (nsteps < 0) return fail_arg("nsteps must be >= 0");
    if (!isfinite(t0) || !isfinite(dt)) return fail_arg("t0 and dt must be finite");
    return SL_OK;
}

static bool planes_overlap(const sl_grid *g, const void *const *a, const void *const *b)
{
    for (int q = 0; q < g->nfields; ++q)
        for (int r = 0; r < g->nfields; ++r)
            if (a[q] == b[r]) return true;
    return false;
}

// counters before the call (SL_FAIL_ERROR) and the failure status after it
static sl_status fail_policy_result(sl_grid *g, const DevCounters &before, cudaStream_t s)
{
    DevCounters after;
    if (sl_status st = read_counters(g, &after, s)) return st;
    if (after.fail_locate > before.fail_locate) return SL_ERR_LOCATE;
    if (after.fail_newton > before.fail_newton) return SL_ERR_NEWTON;
    if (after.fail_fold > before.fail_fold) return SL_ERR_FOLD;
    return SL_OK;
}

extern "C" sl_status sl_step(sl_grid *g, void *const *fields, void *const *scratch, double t0, double dt, int nsteps,
                             void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (sl_status st = check_planes(g, (const void *const *)fields, "field planes")) return st;
    if (sl_status st = check_planes(g, (const void *const *)scratch, "scratch planes")) return st;
    if (planes_overlap(g, (const void *const *)fields, (const void *const *)scratch))
        return fail_arg("field and scratch planes must not overlap");
    if (sl_status st = check_step_args(g, nsteps, t0, dt)) return st;
    if (nsteps == 0) return SL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevCounters before;
    if (g->desc.fail_policy == SL_FAIL_ERROR)
        if (sl_status st = read_counters(g, &before, s)) return st;
    // the ping-pong between scratch and the caller's planes: after an odd number of steps the
    // result sits in the scratch planes and is copied back in one launch (a shallow-water grid
    // ends every step in `fields` itself)
    cudaError_t e = g->dtype == SL_F64
                        ? step_impl<double>(g, (const void *const *)fields, scratch, fields, t0, dt, nsteps, s)
                        : step_impl<float>(g, (const void *const *)fields, scratch, fields, t0, dt, nsteps, s);
    if (e == cudaSuccess && !g->nlsw && nsteps % 2 == 1)
        e = counted(g, g->dtype == SL_F64 ? Launch<double>::copy_planes(g, (const void *const *)scratch, fields, s)
                                          : Launch<float>::copy_planes(g, (const void *const *)scratch, fields, s),
                    1);
    if (e != cudaSuccess) return fail_cuda(e, "sl_step");
    if (g->desc.fail_policy == SL_FAIL_ERROR) return fail_policy_result(g, before, s);
    return SL_OK;
}

extern "C" sl_status sl_step_out(sl_grid *g, const void *const *in, void *const *out, void *const *scratch, double t0,
                                 double dt, int nsteps, void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (sl_status st = check_planes(g, in, "input planes")) return st;
    if (sl_status st = check_planes(g, (const void *const *)out, "output planes")) return st;
    if (planes_overlap(g, in, (const void *const *)out)) return fail_arg("input and output planes must not overlap");
    const bool need_scratch = nsteps > 1 || g->nlsw;
    if (need_scratch) {
        if (sl_status st = check_planes(g, (const void *const *)scratch, "scratch planes")) return st;
        if (planes_overlap(g, in, (const void *const *)scratch) ||
            planes_overlap(g, (const void *const *)out, (const void *const *)scratch))
            return fail_arg("scratch planes must not overlap the input or output planes");
    }
    if (sl_status st = check_step_args(g, nsteps, t0, dt)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (nsteps == 0 || g->nlsw) {
        // nothing to advance, or a shallow-water grid (which advances its planes in place): the
        // input is copied to the output first
        e = counted(g, g->dtype == SL_F64 ? Launch<double>::copy_planes(g, in, out, s)
                                          : Launch<float>::copy_planes(g, in, out, s),
                    1);
        if (e != cudaSuccess) return fail_cuda(e, "sl_step_out");
        if (nsteps == 0) return SL_OK;
        return sl_step(g, out, scratch, t0, dt, nsteps, stream);
    }
    DevCounters before;
    if (g->desc.fail_policy == SL_FAIL_ERROR)
        if (sl_status st = read_counters(g, &before, s)) return st;
    // destinations alternate so that the last step writes `out`
    void *const *A = nsteps % 2 == 1 ? out : scratch;
    void *const *B = nsteps % 2 == 1 ? scratch : out;
    e = g->dtype == SL_F64 ? step_impl<double>(g, in, A, B, t0, dt, nsteps, s)
                           : step_impl<float>(g, in, A, B, t0, dt, nsteps, s);
    if (e != cudaSuccess) return fail_cuda(e, "sl_step_out");
    if (g->desc.fail_policy == SL_FAIL_ERROR) return fail_policy_result(g, before, s);
    return SL_OK;
}

extern "C" sl_status sl_moments(sl_grid *g, const void *field, int pmax, double *host_out, void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (!field || !host_out) return fail_arg("field or host_out is NULL");
    if (pmax < 0 || pmax > 7) return fail_arg("pmax must be in [0, 7]");
    if (((uintptr_t)field % g->tsize) != 0) return fail_arg("field is not aligned to its dtype");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = g->dtype == SL_F64 ? Launch<double>::moments(g, field, pmax, s)
                                       : Launch<float>::moments(g, field, pmax, s);
    e = counted(g, e, 2);
    if (e != cudaSuccess) return fail_cuda(e, "sl_moments");
    SL_CUDA(cudaMemcpyAsync(host_out, g->moment_out, sizeof(double) * (pmax + 1), cudaMemcpyDeviceToHost, s),
            "sl_moments");
    SL_CUDA(cudaStreamSynchronize(s), "sl_moments");
    return SL_OK;
}

extern "C" sl_status sl_compute_flags(sl_grid *g, const void *const *fields, uint8_t *flags_out, void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (sl_status st = check_planes(g, fields, "field planes")) return st;
    if (!flags_out) return fail_arg("flags_out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = g->dtype == SL_F64 ? Launch<double>::flags(g, fields, flags_out, s)
                                       : Launch<float>::flags(g, fields, flags_out, s);
    e = counted(g, e, 1);
    return e == cudaSuccess ? SL_OK : fail_cuda(e, "sl_compute_flags");
}

extern "C" sl_status sl_set_displacement(sl_grid *g, const void *D, int64_t stride, void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (!D) return fail_arg("D is NULL");
    if (stride < g->dim || stride > 64) return fail_arg("stride must be in [dim, 64]");
    if (((uintptr_t)D % g->tsize) != 0) return fail_arg("D is not aligned to its dtype");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = g->dtype == SL_F64 ? Launch<double>::copy_disp(g, D, stride, g->D[g->dcur], g->ds, s)
                                       : Launch<float>::copy_disp(g, D, stride, g->D[g->dcur], g->ds, s);
    e = counted(g, e, 1);
    g->d_cached = 0;  // a displacement set by the caller is not the velocity's
    g->next_valid = 0;
    return e == cudaSuccess ? SL_OK : fail_cuda(e, "sl_set_displacement");
}

extern "C" sl_status sl_get_displacement(sl_grid *g, void *D_out, int64_t stride, void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    if (!D_out) return fail_arg("D_out is NULL");
    if (stride < g->dim || stride > 64) return fail_arg("stride must be in [dim, 64]");
    if (((uintptr_t)D_out % g->tsize) != 0) return fail_arg("D_out is not aligned to its dtype");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = g->dtype == SL_F64 ? Launch<double>::copy_disp(g, g->D[g->dcur], g->ds, D_out, stride, s)
                                       : Launch<float>::copy_disp(g, g->D[g->dcur], g->ds, D_out, stride, s);
    e = counted(g, e, 1);
    return e == cudaSuccess ? SL_OK : fail_cuda(e, "sl_get_displacement");
}

extern "C" sl_status sl_get_diagnostics(sl_grid *g, sl_diag *out, void *stream)
{
    if (!g || !out) return fail_arg("grid or out is NULL");
    DevCounters c;
    if (sl_status st = read_counters(g, &c, (cudaStream_t)stream)) return st;
    out->targets = c.targets;
    out->fail_locate = c.fail_locate;
    out->fail_newton = c.fail_newton;
    out->fail_fold = c.fail_fold;
    out->hops_sum = c.hops_sum;
    out->hops_max = c.hops_max;
    out->iters_sum = c.iters_sum;
    out->iters_max = c.iters_max;
    out->newton_f64 = c.newton_f64;
    for (int q = 0; q < 3; ++q) out->order_hist[q] = c.order_hist[q];
    out->tiles_fallback = c.tiles_fallback;
    out->kernel_launches = g->launches;
    out->timeouts = c.timeouts;
    return SL_OK;
}

extern "C" sl_status sl_reset_diagnostics(sl_grid *g, void *stream)
{
    if (!g) return fail_arg("grid is NULL");
    SL_CUDA(cudaMemsetAsync(g->counters, 0, sizeof(DevCounters), (cudaStream_t)stream), "sl_reset_diagnostics");
    SL_CUDA(cudaMemsetAsync(g->stripes, 0, sizeof(DevCounters) * SL_COUNTER_STRIPES, (cudaStream_t)stream),
            "sl_reset_diagnostics");
    return SL_OK;
}

extern "C" const char *sl_status_string(sl_status st)
{
    switch (st) {
    case SL_OK: return "ok";
    case SL_ERR_ARG: return "invalid argument";
    case SL_ERR_CUDA: return "CUDA error";
    case SL_ERR_NOMEM: return "workspace too small";
    case SL_ERR_BUDGET: return "memory budget exceeded";
    case SL_ERR_LOCATE: return "element search gave up";
    case SL_ERR_NEWTON: return "Newton inversion did not converge";
    case SL_ERR_FOLD: return "folded element";
    case SL_ERR_UNSUPPORTED: return "unsupported option combination";
    }
    return "unknown status";
}

extern "C" const char *sl_last_error(void) { return g_last_error; }

void sl_record_error(const char *what, const char *why)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, why);
}

extern "C" const char *sl_version(void) { return "libsl 0.1 (sm_103a)"; }
