// sl_batch.cu -- many independent 2-D FP32 grids of uneven sizes advanced together: one persistent
// launch per step for all of them over a work-list of (grid, tile) items, optionally replayed as
// a CUDA graph.  Each item runs the same per-tile body as the single-grid kernels (sl_tile2d.cuh):
// window staging, jump flags, element search with Newton inversion, order choice and tensor
// Z-spline sum (Sec. 2.1-2.3, eq. multiZ), and the next step's RK4 trajectories (eq. vel).
//
// Device state lives in the caller's batch workspace: the grid table, the item -> grid map, one
// work counter per step of a call, and each grid's time.  The grids' own workspaces hold their
// displacement buffers and counters as for single-grid calls.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "sl_tile2d_z2.cuh"

namespace {

constexpr int SL_BATCH_MAX_STEPS = 256;  // steps per launch sequence (longer calls are chunked)

// One grid of a batch (device table entry).
struct BatchGrid {
    TileArgs base;                 // n0, n1, nfields, limiter, counters; pointers set per step
    VelArgs<float> vel;            // velocity; ct[] filled per step from the grid's time
    const float *fields[SL_MAX_FIELDS];
    float *scratch[SL_MAX_FIELDS];
    float *D[2];
    double dt, period;             // period > 0: time-dependent velocity cos(pi t / period)
    int dcur;                      // displacement buffer holding D at the call's first step
    int steady;                    // steady velocity: D of the first step serves every step
    int tiles_x, tile_base;
};

// cos(pi t / period) at the stage times of every trajectory sub-step of a step starting at t, by
// the single-grid host code's own function (stage_time_factors); zero for a steady flow
__device__ __forceinline__ void stage_factors(const BatchGrid &g, double t, float *ct)
{
    if (g.period > 0.0) {
        stage_time_factors<float>(t, g.dt, g.vel.substeps, g.vel.integrator, g.period, ct);
    } else {
        for (int q = 0; q < 3 * g.vel.substeps; ++q) ct[q] = 0.f;
    }
}

// copy one grid-table entry into shared memory (all threads), then sync
__device__ __forceinline__ void load_entry(const BatchGrid *table, int gid, BatchGrid *dst)
{
    const int *src = reinterpret_cast<const int *>(table + gid);
    int *d = reinterpret_cast<int *>(dst);
    for (int q = threadIdx.x; q < (int)(sizeof(BatchGrid) / sizeof(int)); q += blockDim.x) d[q] = __ldg(src + q);
    __syncthreads();
}

// next work item of this CTA (thread 0 takes it from the step's counter)
__device__ __forceinline__ int next_item(unsigned *counter, int *s_item)
{
    __syncthreads();
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *s_item;
}

template <class Cfg, int NF>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB)
    batch_step_kernel(const BatchGrid *__restrict__ table, const int *__restrict__ item_grid, int nitems,
                      unsigned *counter, const double *__restrict__ tgrid, int k, int last)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sBox[4];
    __shared__ int s_item;
    __shared__ __align__(16) BatchGrid sg;
    __shared__ TileArgs sa;
    __shared__ VelArgs<float> sv;
    const TileSmem<Cfg, NF> sm(smem);
    for (int item = next_item(counter, &s_item); item < nitems; item = next_item(counter, &s_item)) {
        const int gid = __ldg(item_grid + item);
        load_entry(table, gid, &sg);
        if (threadIdx.x == 0) {
            sa = sg.base;
            const bool even = (k & 1) == 0;
            for (int f = 0; f < NF; ++f) {
                sa.in[f] = even ? sg.fields[f] : sg.scratch[f];
                sa.out[f] = even ? sg.scratch[f] : const_cast<float *>(sg.fields[f]);
            }
            sa.D = sg.steady ? sg.D[sg.dcur] : sg.D[(sg.dcur + k) & 1];
            sa.D_next = (last || sg.steady) ? nullptr : sg.D[(sg.dcur + k + 1) & 1];
            sv = sg.vel;
            stage_factors(sg, tgrid[gid] + (double)(k + 1) * sg.dt, sv.ct);
        }
        __syncthreads();
        const int t = item - sg.tile_base;
        const int ty = t / sg.tiles_x, tx = t - ty * sg.tiles_x;
        LocalCounters cnt;
        cnt.clear();
        process_tile<Cfg, NF, true>(sa, sv, tx * Cfg::TX, ty * Cfg::TY, sm, sBox, cnt);
        flush_counters(cnt, sa.counters);
    }
}

// The same step for batches of quintic grids (32 x 32 tiles of the quintic tile body).
template <int NF>
__global__ void __launch_bounds__(CfgZ::NT, CfgZ::MINB)
    batch_step_z2_kernel(const BatchGrid *__restrict__ table, const int *__restrict__ item_grid, int nitems,
                         unsigned *counter, const double *__restrict__ tgrid, int k, int last)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sBox[4];
    __shared__ int s_item;
    __shared__ __align__(16) BatchGrid sg;
    __shared__ TileArgs sa;
    __shared__ VelArgs<float> sv;
    const TileSmemZ2<NF> sm(smem);
    for (int item = next_item(counter, &s_item); item < nitems; item = next_item(counter, &s_item)) {
        const int gid = __ldg(item_grid + item);
        load_entry(table, gid, &sg);
        if (threadIdx.x == 0) {
            sa = sg.base;
            const bool even = (k & 1) == 0;
            for (int f = 0; f < NF; ++f) {
                sa.in[f] = even ? sg.fields[f] : sg.scratch[f];
                sa.out[f] = even ? sg.scratch[f] : const_cast<float *>(sg.fields[f]);
            }
            sa.D = sg.steady ? sg.D[sg.dcur] : sg.D[(sg.dcur + k) & 1];
            sa.D_next = (last || sg.steady) ? nullptr : sg.D[(sg.dcur + k + 1) & 1];
            sv = sg.vel;
            stage_factors(sg, tgrid[gid] + (double)(k + 1) * sg.dt, sv.ct);
        }
        __syncthreads();
        const int t = item - sg.tile_base;
        const int ty = t / sg.tiles_x, tx = t - ty * sg.tiles_x;
        LocalCounters cnt;
        cnt.clear();
        process_tile_z2<NF, true>(sa, sv, tx * CfgZ::TX, ty * CfgZ::TY, sm, sBox, cnt);
        flush_counters(cnt, sa.counters);
    }
}

// RK4 displacements of every grid's nodes at the grid's time (before the first step of a call)
template <class Cfg>
__global__ void __launch_bounds__(Cfg::NT)
    batch_advect_kernel(const BatchGrid *__restrict__ table, const int *__restrict__ item_grid, int nitems,
                        unsigned *counter, const double *__restrict__ tgrid)
{
    __shared__ int s_item;
    __shared__ __align__(16) BatchGrid sg;
    __shared__ VelArgs<float> sv;
    for (int item = next_item(counter, &s_item); item < nitems; item = next_item(counter, &s_item)) {
        const int gid = __ldg(item_grid + item);
        load_entry(table, gid, &sg);
        if (threadIdx.x == 0) {
            sv = sg.vel;
            stage_factors(sg, tgrid[gid], sv.ct);
        }
        __syncthreads();
        const int t = item - sg.tile_base;
        const int ty = t / sg.tiles_x, tx = t - ty * sg.tiles_x;
        float2 *D = reinterpret_cast<float2 *>(sg.D[sg.dcur]);
        for (int q = threadIdx.x; q < Cfg::TX * Cfg::TY; q += Cfg::NT) {
            const int jx = tx * Cfg::TX + q % Cfg::TX, jy = ty * Cfg::TY + q / Cfg::TX;
            if (jx >= sg.base.n0 || jy >= sg.base.n1) continue;
            float X[3] = {node_position(sv.lo[0], jx, sv.dx[0]), node_position(sv.lo[1], jy, sv.dx[1]), 0.f}, d[3];
            trajectory_cells<float, 2>(sv, X, d);
            D[(long long)jy * sg.base.n0 + jx] = make_float2(d[0], d[1]);
        }
    }
}

// after a call: fields back into the caller's planes (odd step counts) and the grids' times
template <class Cfg>
__global__ void __launch_bounds__(Cfg::NT)
    batch_finish_kernel(const BatchGrid *__restrict__ table, const int *__restrict__ item_grid, int nitems,
                        unsigned *counter, double *tgrid, int ngrids, int nsteps)
{
    __shared__ int s_item;
    __shared__ __align__(16) BatchGrid sg;
    if (blockIdx.x == 0)
        for (int g = threadIdx.x; g < ngrids; g += blockDim.x) tgrid[g] += (double)nsteps * table[g].dt;
    if ((nsteps & 1) == 0) return;
    for (int item = next_item(counter, &s_item); item < nitems; item = next_item(counter, &s_item)) {
        const int gid = __ldg(item_grid + item);
        load_entry(table, gid, &sg);
        const int t = item - sg.tile_base;
        const int ty = t / sg.tiles_x, tx = t - ty * sg.tiles_x;
        for (int q = threadIdx.x; q < Cfg::TX * Cfg::TY; q += Cfg::NT) {
            const int jx = tx * Cfg::TX + q % Cfg::TX, jy = ty * Cfg::TY + q / Cfg::TX;
            if (jx >= sg.base.n0 || jy >= sg.base.n1) continue;
            const long long jj = (long long)jy * sg.base.n0 + jx;
            for (int f = 0; f < sg.base.nfields; ++f) const_cast<float *>(sg.fields[f])[jj] = sg.scratch[f][jj];
        }
    }
}

struct BatchLayout {
    size_t table, items, counters, tgrid, total;
};

BatchLayout batch_layout(int count, int nitems)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    BatchLayout L;
    size_t off = 0;
    L.table = off;
    off += al(sizeof(BatchGrid) * (size_t)count);
    L.items = off;
    off += al(sizeof(int) * (size_t)nitems);
    L.counters = off;
    off += al(sizeof(unsigned) * (SL_BATCH_MAX_STEPS + 2));
    L.tgrid = off;
    off += al(sizeof(double) * (size_t)count);
    L.total = off;
    return L;
}

template <class Cfg>
void tiles_of(const sl_grid *g, int *tx, int *ty)
{
    *tx = (int)((g->n[0] + Cfg::TX - 1) / Cfg::TX);
    *ty = (int)((g->n[1] + Cfg::TY - 1) / Cfg::TY);
}

void tile_counts(int cfg, const sl_grid *g, int *tx, int *ty)
{
    if (cfg == 2 || cfg == 4)
        tiles_of<CfgB>(g, tx, ty);
    else if (cfg == 3)
        tiles_of<CfgC>(g, tx, ty);
    else
        tiles_of<CfgA>(g, tx, ty);
}

}  // namespace

struct sl_batch {
    int count, nfields, cfg, nitems, num_sms;
    bool quintic;  // the grids take the quintic Z-spline (max_order 2)
    int device;
    std::vector<sl_grid *> grids;
    char *ws;
    BatchLayout L;
    BatchGrid *table;
    int *items;
    unsigned *counters;
    double *tgrid;
    std::vector<double> t_host, dt_host;
    std::vector<int> dcur0;           // displacement buffer each grid's advect writes at a call start
    unsigned long long launches = 0;  // kernels launched by this batch's calls
    // cached graphs: one per step count
    std::vector<int> graph_steps;
    std::vector<cudaGraphExec_t> graphs;
};

// the batch computes each step's RK4 stage factors on the device from the grid's time: one
// classical RK4 step per remap only
static bool batch_eligible(const sl_grid *g)
{
    return g && g->dim == 2 && g->dtype == SL_F32 && g->desc.newton_mode == SL_NEWTON_MIXED &&
           g->desc.walk_start == SL_START_BACKWARD && !g->carried && !g->nlsw;
}

// Tiles of quintic batches are the quintic kernel's 32 x 32 whatever the tile configuration.
static int batch_cfg(sl_grid *const *grids, int tile_config)
{
    return grids[0]->desc.max_order == 2 ? 1 : tile_config;
}

extern "C" size_t sl_batch_workspace_bytes(sl_grid *const *grids, int count, int tile_config)
{
    if (!grids || count < 1 || tile_config < 0 || tile_config > 5) return 0;
    long long nitems = 0;
    for (int q = 0; q < count; ++q) {
        if (!batch_eligible(grids[q])) return 0;
        if ((grids[q]->desc.max_order == 2) != (grids[0]->desc.max_order == 2)) return 0;
        int tx, ty;
        tile_counts(batch_cfg(grids, tile_config), grids[q], &tx, &ty);
        nitems += (long long)tx * ty;
    }
    if (nitems > (1LL << 30)) return 0;
    return batch_layout(count, (int)nitems).total;
}

extern "C" sl_status sl_batch_create(sl_grid *const *grids, int count, void *const *const *fields,
                                     void *const *const *scratch, const double *t0, const double *dt, int tile_config,
                                     void *dev_workspace, size_t ws_bytes, sl_batch **out)
{
    if (!out) return SL_ERR_ARG;
    *out = nullptr;
    if (!grids || count < 1 || !fields || !scratch || !t0 || !dt || !dev_workspace) return SL_ERR_ARG;
    if (tile_config < 0 || tile_config > 5) return SL_ERR_ARG;
    if (((uintptr_t)dev_workspace & 255u) != 0) return SL_ERR_ARG;
    const int nf = grids[0] ? grids[0]->nfields : 0;
    if (nf < 1 || nf > 4) return SL_ERR_UNSUPPORTED;
    for (int q = 0; q < count; ++q) {
        if (!batch_eligible(grids[q])) return SL_ERR_UNSUPPORTED;
        // one batch runs one tile kernel: cubic / linear grids, or quintic grids
        if ((grids[q]->desc.max_order == 2) != (grids[0]->desc.max_order == 2)) return SL_ERR_UNSUPPORTED;
        if (grids[q]->nfields != nf) return SL_ERR_UNSUPPORTED;
        if (!fields[q] || !scratch[q] || !isfinite(t0[q]) || !isfinite(dt[q])) return SL_ERR_ARG;
        for (int f = 0; f < nf; ++f)
            if (!fields[q][f] || !scratch[q][f] || fields[q][f] == scratch[q][f]) return SL_ERR_ARG;
    }
    const size_t need = sl_batch_workspace_bytes(grids, count, tile_config);
    if (need == 0) return SL_ERR_ARG;
    if (ws_bytes < need) return SL_ERR_NOMEM;
    sl_batch *b = new (std::nothrow) sl_batch();
    if (!b) return SL_ERR_ARG;
    b->count = count;
    b->nfields = nf;
    b->quintic = grids[0]->desc.max_order == 2;
    b->cfg = batch_cfg(grids, tile_config);
    b->grids.assign(grids, grids + count);
    std::vector<BatchGrid> table(count);
    std::vector<int> items;
    for (int q = 0; q < count; ++q) {
        sl_grid *g = grids[q];
        BatchGrid &e = table[q];
        memset(&e, 0, sizeof(e));
        e.base = make_tile_args(g, nullptr, nullptr, (const void *const *)fields[q], scratch[q]);
        e.vel = make_vel_args<float>(g, t0[q], dt[q]);
        for (int f = 0; f < nf; ++f) {
            e.fields[f] = (const float *)fields[q][f];
            e.scratch[f] = (float *)scratch[q][f];
        }
        e.D[0] = (float *)g->D[0];
        e.D[1] = (float *)g->D[1];
        e.dt = dt[q];
        e.period = (g->desc.velocity_kind == SL_VEL_SWIRL2D) ? g->vel_params[0] : 0.0;
        e.dcur = g->dcur;
        e.steady = g->steady;
        int tx, ty;
        tile_counts(b->cfg, g, &tx, &ty);
        e.tiles_x = tx;
        e.tile_base = (int)items.size();
        for (int t = 0; t < tx * ty; ++t) items.push_back(q);
    }
    b->nitems = (int)items.size();
    b->L = batch_layout(count, b->nitems);
    b->ws = (char *)dev_workspace;
    b->table = (BatchGrid *)(b->ws + b->L.table);
    b->items = (int *)(b->ws + b->L.items);
    b->counters = (unsigned *)(b->ws + b->L.counters);
    b->tgrid = (double *)(b->ws + b->L.tgrid);
    b->t_host.assign(t0, t0 + count);
    for (int q = 0; q < count; ++q) b->dcur0.push_back(grids[q]->dcur);
    b->dt_host.assign(dt, dt + count);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMemcpy(b->table, table.data(), sizeof(BatchGrid) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->items, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tgrid, t0, sizeof(double) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete b;
        return SL_ERR_CUDA;
    }
    *out = b;
    return SL_OK;
}

template <class Cfg, int NF>
static cudaError_t launch_batch_seq(sl_batch *b, int nsteps, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes<Cfg>(NF);
    static bool configured[64] = {};
    cudaError_t e = allow_smem(batch_step_kernel<Cfg, NF>, b->device, smem, configured);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step_kernel<Cfg, NF>, Cfg::NT, smem);
    if (e != cudaSuccess) return e;
    const int ctas = b->num_sms * (per_sm > 0 ? per_sm : 1);
    const int simple = b->num_sms * 8;
    e = cudaMemsetAsync(b->counters, 0, sizeof(unsigned) * (SL_BATCH_MAX_STEPS + 2), s);
    if (e != cudaSuccess) return e;
    batch_advect_kernel<Cfg><<<simple, Cfg::NT, 0, s>>>(b->table, b->items, b->nitems, b->counters + 0, b->tgrid);
    for (int k = 0; k < nsteps; ++k)
        batch_step_kernel<Cfg, NF><<<ctas, Cfg::NT, smem, s>>>(b->table, b->items, b->nitems, b->counters + 1 + k,
                                                               b->tgrid, k, k + 1 == nsteps);
    batch_finish_kernel<Cfg><<<simple, Cfg::NT, 0, s>>>(b->table, b->items, b->nitems,
                                                        b->counters + 1 + SL_BATCH_MAX_STEPS, b->tgrid, b->count,
                                                        nsteps);
    return cudaGetLastError();
}

static_assert(CfgZ::TX == CfgA::TX && CfgZ::TY == CfgA::TY, "quintic batches reuse the 32 x 32 tile geometry");

template <int NF>
static cudaError_t launch_batch_seq_z2(sl_batch *b, int nsteps, cudaStream_t s)
{
    const size_t smem = z2_smem_bytes(NF);
    static bool configured[64] = {};
    cudaError_t e = allow_smem(batch_step_z2_kernel<NF>, b->device, smem, configured);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step_z2_kernel<NF>, CfgZ::NT, smem);
    if (e != cudaSuccess) return e;
    const int ctas = b->num_sms * (per_sm > 0 ? per_sm : 1);
    const int simple = b->num_sms * 8;
    e = cudaMemsetAsync(b->counters, 0, sizeof(unsigned) * (SL_BATCH_MAX_STEPS + 2), s);
    if (e != cudaSuccess) return e;
    // the quintic tiles have the 32 x 32 geometry of CfgA, whose trajectory and finishing kernels serve
    batch_advect_kernel<CfgA><<<simple, CfgA::NT, 0, s>>>(b->table, b->items, b->nitems, b->counters + 0, b->tgrid);
    for (int k = 0; k < nsteps; ++k)
        batch_step_z2_kernel<NF><<<ctas, CfgZ::NT, smem, s>>>(b->table, b->items, b->nitems, b->counters + 1 + k,
                                                              b->tgrid, k, k + 1 == nsteps);
    batch_finish_kernel<CfgA><<<simple, CfgA::NT, 0, s>>>(b->table, b->items, b->nitems,
                                                          b->counters + 1 + SL_BATCH_MAX_STEPS, b->tgrid, b->count,
                                                          nsteps);
    return cudaGetLastError();
}

template <class Cfg>
static cudaError_t launch_batch_cfg(sl_batch *b, int nsteps, cudaStream_t s)
{
    switch (b->nfields) {
    case 1: return launch_batch_seq<Cfg, 1>(b, nsteps, s);
    case 2: return launch_batch_seq<Cfg, 2>(b, nsteps, s);
    case 3: return launch_batch_seq<Cfg, 3>(b, nsteps, s);
    default: return launch_batch_seq<Cfg, 4>(b, nsteps, s);
    }
}

static cudaError_t launch_batch(sl_batch *b, int nsteps, cudaStream_t s)
{
    if (b->quintic) {
        switch (b->nfields) {
        case 1: return launch_batch_seq_z2<1>(b, nsteps, s);
        case 2: return launch_batch_seq_z2<2>(b, nsteps, s);
        case 3: return launch_batch_seq_z2<3>(b, nsteps, s);
        default: return launch_batch_seq_z2<4>(b, nsteps, s);
        }
    }
    if (b->cfg == 2) return launch_batch_cfg<CfgB>(b, nsteps, s);
    if (b->cfg == 4) return launch_batch_cfg<CfgD>(b, nsteps, s);
    if (b->cfg == 3) return launch_batch_cfg<CfgC>(b, nsteps, s);
    return launch_batch_cfg<CfgA>(b, nsteps, s);
}

extern "C" sl_status sl_batch_step(sl_batch *b, int nsteps, int use_graph, void *stream)
{
    if (!b || nsteps < 0) return SL_ERR_ARG;
    if (nsteps == 0) return SL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (use_graph && s == nullptr) return SL_ERR_ARG;  // the legacy stream cannot be captured
    int done = 0;
    while (done < nsteps) {
        const int n = nsteps - done < SL_BATCH_MAX_STEPS ? nsteps - done : SL_BATCH_MAX_STEPS;
        // the D index each grid starts from must be in the table before the sequence runs
        cudaError_t e = cudaSuccess;
        if (!use_graph) {
            e = launch_batch(b, n, s);
        } else {
            cudaGraphExec_t exec = nullptr;
            for (size_t q = 0; q < b->graph_steps.size(); ++q)
                if (b->graph_steps[q] == n) exec = b->graphs[q];
            if (!exec) {
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t le = launch_batch(b, n, s);
                    e = cudaStreamEndCapture(s, &graph);
                    if (le != cudaSuccess) e = le;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                if (e == cudaSuccess) {
                    b->graph_steps.push_back(n);
                    b->graphs.push_back(exec);
                }
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        }
        if (e != cudaSuccess) return SL_ERR_CUDA;
        // every call integrates D afresh into the table's starting buffer, so the table (and any
        // captured graph) never changes; the grid objects point at the last step's D
        for (int q = 0; q < b->count; ++q) {
            b->grids[q]->dcur = b->grids[q]->steady ? b->dcur0[q] : (b->dcur0[q] + n - 1) & 1;
            b->grids[q]->d_cached = 0;
            b->t_host[q] += n * b->dt_host[q];
        }
        b->launches += (unsigned long long)(n + 2);
        done += n;
    }
    return SL_OK;
}

extern "C" sl_status sl_batch_info(const sl_batch *b, int *nitems, unsigned long long *launches, double *t_first)
{
    if (!b) return SL_ERR_ARG;
    if (nitems) *nitems = b->nitems;
    if (launches) *launches = b->launches;
    if (t_first) *t_first = b->t_host[0];
    return SL_OK;
}

extern "C" sl_status sl_batch_destroy(sl_batch *b)
{
    if (!b) return SL_ERR_ARG;
    for (cudaGraphExec_t g : b->graphs) cudaGraphExecDestroy(g);
    delete b;
    return SL_OK;
}
