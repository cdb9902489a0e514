// sl_kernels.cu -- the plain kernels of the FSL step (arXiv:1410.2817): one thread per node with
// gathers straight from global memory (read-only cache).  They serve every dtype and dimension;
// the FP64 instantiation is the single-grid FP64 path, and every kernel here can write per-target
// diagnostics for parity checks.
//
//   flags_kernel          Sec. 2.3 jump criterion (bit f of a byte per node)
//   advect_kernel         eq. (vel), one classical RK4 step per Lagrangian node
//   remap_generic_kernel  Sec. 2.2 element search + Newton inversion, Sec. 2.3 order reduction,
//                         eq. (multiZ) tensor Z-spline sum
//   moments_*             Sec. 3.1 discrete moments, FP64 accumulation in a fixed order
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "sl_internal.h"

// ------------------------------------------------------------------------------------------------
// argument builders
// ------------------------------------------------------------------------------------------------
template <typename T>
GridArgs<T> make_grid_args(const sl_grid *g)
{
    GridArgs<T> a;
    for (int q = 0; q < 3; ++q) a.n[q] = (int)(q < g->dim ? g->n[q] : 1);
    a.N = (long long)g->N;
    a.nfields = g->nfields;
    a.max_order = g->desc.max_order;
    a.threshold = (T)g->desc.limiter_threshold;
    a.newton_max_iter = g->desc.newton_max_iter;
    a.walk_max = g->desc.walk_max;
    a.walk_start = g->desc.walk_start;
    a.tol = sizeof(T) == 8 ? (T)1e-14 : (T)SL_NEWTON_TOL_F32;
    a.slack = sizeof(T) == 8 ? (T)1e-12 : (T)SL_SLACK_F32;
    return a;
}

template <typename T>
VelArgs<T> make_vel_args(const sl_grid *g, double t, double dt)
{
    VelArgs<T> v;
    memset(&v, 0, sizeof(v));
    v.kind = g->desc.velocity_kind;
    v.nmodes = (v.kind == SL_VEL_FOURIER2D || v.kind == SL_VEL_FOURIER3D) ? (int)g->vel_params[0] : 0;
    v.integrator = g->desc.integrator;
    v.substeps = g->desc.trajectory_substeps > 0 ? g->desc.trajectory_substeps : 1;
    for (int q = 0; q < SL_MAX_VEL_PARAMS; ++q) v.p[q] = (T)g->vel_params[q];
    if (v.kind == SL_VEL_SWIRL2D || v.kind == SL_VEL_DEFORM3D) {
        stage_time_factors<T>(t, dt, v.substeps, v.integrator, g->vel_params[0], v.ct);
    }
    for (int q = 0; q < 3; ++q) {
        v.lo[q] = (T)g->desc.lo[q];
        v.dx[q] = (T)g->dx[q];
        v.inv_dx[q] = (T)(1.0 / g->dx[q]);
    }
    v.dt = (T)dt;
    if (g->trig != nullptr && sizeof(T) == g->tsize)
        for (int q = 0; q < g->dim; ++q) v.sc[q] = (const T *)g->trig + g->trig_off[q];
    return v;
}

// sin(pi x), cos(pi x) at every node coordinate of every axis, computed by the kernels' own
// node_position and sincospi_t (so a table entry has the bits the kernels compute)
template <typename T>
__global__ void __launch_bounds__(256) trig_table_kernel(VelArgs<T> v, int dim, int n0, int n1, int n2, T *tab)
{
    const int n[3] = {n0, n1, n2};
    long long base = 0;
    for (int a = 0; a < dim; ++a) {
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n[a]; k += gridDim.x * blockDim.x) {
            T sn, cs;
            sincospi_t(node_position(v.lo[a], k, v.dx[a]), &sn, &cs);
            tab[base + 2 * k] = sn;
            tab[base + 2 * k + 1] = cs;
        }
        base += 2LL * n[a];
    }
}

cudaError_t launch_trig_tables(const sl_grid *g, cudaStream_t s)
{
    if (g->trig == nullptr) return cudaSuccess;
    const int n1 = g->dim > 1 ? (int)g->n[1] : 0, n2 = g->dim > 2 ? (int)g->n[2] : 0;
    if (g->dtype == SL_F64)
        trig_table_kernel<double><<<64, 256, 0, s>>>(make_vel_args<double>(g, 0.0, 1.0), g->dim, (int)g->n[0], n1, n2,
                                                     (double *)g->trig);
    else
        trig_table_kernel<float><<<64, 256, 0, s>>>(make_vel_args<float>(g, 0.0, 1.0), g->dim, (int)g->n[0], n1, n2,
                                                    (float *)g->trig);
    return cudaGetLastError();
}

// One block per `threads` nodes (the kernels also loop grid-stride, so any count is correct).
// Short-lived blocks let the block scheduler interleave work of higher-priority streams; the cap
// only guards the grid-size limit.
int grid_stride_blocks(const sl_grid *g, long long work, int threads)
{
    (void)g;
    long long b = (work + threads - 1) / threads;
    if (b > (1LL << 30)) b = 1LL << 30;
    if (b < 1) b = 1;
    return (int)b;
}

template GridArgs<double> make_grid_args<double>(const sl_grid *);
template GridArgs<float> make_grid_args<float>(const sl_grid *);
template VelArgs<double> make_vel_args<double>(const sl_grid *, double, double);
template VelArgs<float> make_vel_args<float>(const sl_grid *, double, double);

// ------------------------------------------------------------------------------------------------
// node index helpers
// ------------------------------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void node_coords(long long i, const int n[3], int k[3])
{
    k[0] = (int)(i % n[0]);
    long long r = i / n[0];
    k[1] = (int)(r % n[1]);
    k[2] = DIM == 3 ? (int)(r / n[1]) : 0;
}

template <int DIM>
__device__ __forceinline__ long long node_index(const int k[3], const int n[3])
{
    long long idx = wrap_idx(k[0], n[0]) + (long long)n[0] * wrap_idx(k[1], n[1]);
    if (DIM == 3) idx += (long long)n[0] * n[1] * wrap_idx(k[2], n[2]);
    return idx;
}

template <typename T>
struct FieldPtrs {
    const T *in[SL_MAX_FIELDS];
    T *out[SL_MAX_FIELDS];
};

// ------------------------------------------------------------------------------------------------
// Sec. 2.3: jump flags
// ------------------------------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(256) flags_kernel(GridArgs<T> g, FieldPtrs<T> f, uint8_t *__restrict__ flags)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned bits = 0;
        if (g.threshold >= T(0)) {
            int k[3];
            node_coords<DIM>(i, g.n, k);
            long long nb[3][2];
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                int kp[3] = {k[0], k[1], k[2]}, km[3] = {k[0], k[1], k[2]};
                kp[a] += 1;
                km[a] -= 1;
                nb[a][0] = node_index<DIM>(km, g.n);
                nb[a][1] = node_index<DIM>(kp, g.n);
            }
            for (int q = 0; q < g.nfields; ++q) {
                const T *h = f.in[q];
                const T h0 = __ldg(h + i);
                bool hit = false;
#pragma unroll
                for (int a = 0; a < DIM; ++a) hit |= jump_test<T>(__ldg(h + nb[a][0]), h0, __ldg(h + nb[a][1]), g.threshold);
                if (hit) bits |= 1u << q;
            }
        }
        flags[i] = (uint8_t)bits;
    }
}

// ------------------------------------------------------------------------------------------------
// eq. (vel): RK4 displacement of every Lagrangian node (cell units), stride ds values per node
// ------------------------------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(256) advect_kernel(GridArgs<T> g, VelArgs<T> v, T *__restrict__ D, int ds)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        int k[3];
        node_coords<DIM>(i, g.n, k);
        T X[3] = {T(0), T(0), T(0)}, d[3];
#pragma unroll
        for (int a = 0; a < DIM; ++a) X[a] = node_position(v.lo[a], k[a], v.dx[a]);
        trajectory_cells_node<T, DIM>(v, X, k, d);
#pragma unroll
        for (int a = 0; a < DIM; ++a) D[i * ds + a] = d[a];
        if (DIM == 3) D[i * ds + 3] = T(0);
    }
}

// ------------------------------------------------------------------------------------------------
// Sec. 3.2: the velocity carried by the nodes (Burgers, Du/Dt = 0) is constant along each
// trajectory, so every integrator moves node i by dt u_i: D_i = (dt / dx_a) u_a,i in cell units.
// ------------------------------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
    advect_carried_kernel(long long N, const T *__restrict__ u0, const T *__restrict__ u1, const T *__restrict__ u2,
                          T s0, T s1, T s2, T *__restrict__ D)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (DIM == 2) {
            using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
            T2 d;
            d.x = s0 * __ldg(u0 + i);
            d.y = s1 * __ldg(u1 + i);
            reinterpret_cast<T2 *>(D)[i] = d;
        } else {
            D[i * 4 + 0] = s0 * __ldg(u0 + i);
            D[i * 4 + 1] = s1 * __ldg(u1 + i);
            D[i * 4 + 2] = s2 * __ldg(u2 + i);
            D[i * 4 + 3] = T(0);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Sec. 2.2 element search with Newton inversion; the same walk as the paper's: invert, and while a
// local coordinate is out of range step into the neighbour it points to.
// ------------------------------------------------------------------------------------------------
template <typename TN>
struct WalkParams {
    TN tol, slack;
    int max_iter, walk_max;
};

// Start element (Sec. 2.2): the paper's "opposite the velocity" (the element having Lagrangian node
// j as a vertex on the side opposite its own displacement), or the backward estimate floor(j - D_j).
template <typename T, int DIM>
__device__ __forceinline__ void walk_start_cell(int mode, const int j[3], const T Dj[3], int c[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (mode == SL_START_PAPER) {
            c[a] = j[a] - (Dj[a] > T(0) ? 1 : 0);
        } else {
            // clamped so that a garbage displacement cannot overflow the walk's integer steps
            const T s = min_t(max_t(T(j[a]) - Dj[a], T(j[a]) - T(65536)), T(j[a]) + T(65536));
            c[a] = finite_t(s) ? (int)floor_t<T>(s) : j[a];
        }
    }
}

// Sec. 2.2 element search from element c: invert (Newton in precision TN) and, while a local
// coordinate is out of range, step into the neighbour it points to.  On return c is the last
// element tried and xi its local coordinates; *hops and *iters are incremented.
template <typename T, typename TN, int DIM>
__device__ __forceinline__ int walk_global(const WalkParams<TN> &w, const int n[3], const T *__restrict__ D, int ds,
                                           const int j[3], int c[3], TN xi[3], int *hops, int *iters,
                                           bool *degenerate = nullptr)
{
    CycleCheck cyc;
    cyc.start(c[0], c[1], c[2]);
    for (int hop = 0; hop < w.walk_max; ++hop) {
        TN P[8][3];
#pragma unroll
        for (int v = 0; v < (1 << DIM); ++v) {
            int k[3] = {c[0], c[1], c[2]};
#pragma unroll
            for (int a = 0; a < DIM; ++a) k[a] += (v >> a) & 1;
            const long long idx = node_index<DIM>(k, n);
#pragma unroll
            for (int a = 0; a < DIM; ++a) P[v][a] = TN(k[a] - j[a]) + (TN)__ldg(D + idx * ds + a);
        }
        int it = 0;
        const int st = newton_solve<TN, DIM>(P, w.max_iter, w.tol, xi, &it, degenerate);
        *hops += 1;
        *iters += it;
        bool finite = true, inside = true;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            if (!finite_t(xi[a])) finite = false;
            if (!(xi[a] >= -w.slack && xi[a] <= TN(1) + w.slack)) inside = false;
        }
        if (!finite) return st == ST_OK ? ST_NEWTON : st;
        if (inside) return st;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            if (xi[a] < -w.slack)
                c[a] -= 1;
            else if (xi[a] > TN(1) + w.slack)
                c[a] += 1;
        }
        if (cyc.step(c[0], c[1], c[2])) return ST_LOCATE;
    }
    return ST_LOCATE;
}

template <typename T>
struct RemapDebug {
    long long *cell;
    double *xi;
    uint8_t *order;
    uint8_t *status;
};

// NMODE: 0 = Newton in T; 1 = Newton in FP64 (FP32 data); 2 = FP32 Newton, FP64 re-solve of targets
// whose FP32 inversion failed or whose element is close to degenerate.
template <typename T, int DIM, int NMODE>
__global__ void __launch_bounds__(256)
    remap_generic_kernel(GridArgs<T> g, const T *__restrict__ D, int ds, const uint8_t *__restrict__ flags,
                         FieldPtrs<T> f, RemapDebug<T> dbg, DevCounters *counters)
{
    typedef typename std::conditional<NMODE == 1, double, T>::type TW;
    LocalCounters cnt;
    cnt.clear();
    WalkParams<TW> wp;
    wp.tol = NMODE == 1 ? TW(1e-14) : TW(g.tol);
    wp.slack = NMODE == 1 ? TW(1e-12) : TW(g.slack);
    wp.max_iter = g.newton_max_iter;
    wp.walk_max = g.walk_max;
    for (long long jj = blockIdx.x * (long long)blockDim.x + threadIdx.x; jj < g.N;
         jj += (long long)gridDim.x * blockDim.x) {
        int j[3], c[3];
        node_coords<DIM>(jj, g.n, j);
        T Dj[3] = {T(0), T(0), T(0)};
        TW xw[3] = {TW(0), TW(0), TW(0)};
#pragma unroll
        for (int a = 0; a < DIM; ++a) Dj[a] = __ldg(D + jj * ds + a);
        int hops = 0, iters = 0;
        walk_start_cell<T, DIM>(g.walk_start, j, Dj, c);
        bool degen = false;
        int st = walk_global<T, TW, DIM>(wp, g.n, D, ds, j, c, xw, &hops, &iters, &degen);
        T xi[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int a = 0; a < DIM; ++a) xi[a] = (T)xw[a];
        if (NMODE == 2) {
            const bool redo = st != ST_OK || degen;
            if (redo) {
                WalkParams<double> wd;
                wd.tol = 1e-14;
                wd.slack = 1e-12;
                wd.max_iter = g.newton_max_iter;
                wd.walk_max = g.walk_max;
                double xd[3] = {0.0, 0.0, 0.0};
                if (st == ST_LOCATE || st == ST_FOLD) walk_start_cell<T, DIM>(g.walk_start, j, Dj, c);
                st = walk_global<T, double, DIM>(wd, g.n, D, ds, j, c, xd, &hops, &iters);
#pragma unroll
                for (int a = 0; a < DIM; ++a) xi[a] = (T)xd[a];
                cnt.f64 += 1;
            }
        }
        cnt.targets += 1;
        cnt.hops += hops;
        cnt.hops_max = max(cnt.hops_max, (unsigned)hops);
        cnt.iters += iters;
        cnt.iters_max = max(cnt.iters_max, (unsigned)iters);
        if (dbg.status) dbg.status[jj] = (uint8_t)st;
        if (dbg.xi)
            for (int a = 0; a < DIM; ++a) dbg.xi[jj * DIM + a] = (double)xw[a];
        if (st != ST_OK) {
            cnt.fl += st == ST_LOCATE;
            cnt.fn += st == ST_NEWTON;
            cnt.ff += st == ST_FOLD;
            if (dbg.cell) dbg.cell[jj] = -1;
            for (int q = 0; q < g.nfields; ++q) {
                f.out[q][jj] = f.in[q][jj];
                if (dbg.order) dbg.order[(long long)q * g.N + jj] = 0xff;
            }
            continue;
        }
        if (dbg.cell) dbg.cell[jj] = node_index<DIM>(c, g.n);
        // wrapped node offsets of the cubic stencil c-1 .. c+2 along each axis (taps and flags)
        long long ox[4], oy[4], oz[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ox[k] = wrap_idx(c[0] - 1 + k, g.n[0]);
            oy[k] = (long long)wrap_idx(c[1] - 1 + k, g.n[1]) * g.n[0];
            oz[k] = DIM == 3 ? (long long)wrap_idx(c[2] - 1 + k, g.n[2]) * g.n[0] * g.n[1] : 0;
        }
        constexpr int KZ = DIM == 3 ? 4 : 1;
        // Sec. 2.3: OR of the flag bytes over the stencils of order 2 ([c-2, c+3]) and 1 ([c-1, c+2])
        unsigned box2 = 0, box1 = 0;
        if (g.max_order == 1) {
#pragma unroll
            for (int kz = 0; kz < KZ; ++kz)
#pragma unroll
                for (int ky = 0; ky < 4; ++ky)
#pragma unroll
                    for (int kx = 0; kx < 4; ++kx) box1 |= __ldg(flags + oz[kz] + oy[ky] + ox[kx]);
        } else if (g.max_order >= 2) {
            const int r = 2, w = 6;
            const int cnt_box = DIM == 3 ? w * w * w : w * w;
            for (int q = 0; q < cnt_box; ++q) {
                int o[3] = {q % w - r, (q / w) % w - r, DIM == 3 ? q / (w * w) - r : 0};
                int k[3] = {c[0] + o[0], c[1] + o[1], c[2] + o[2]};
                const unsigned fb = __ldg(flags + node_index<DIM>(k, g.n));
                box2 |= fb;
                bool inner = true;
#pragma unroll
                for (int a = 0; a < DIM; ++a) inner &= (o[a] >= -1 && o[a] <= 2);
                if (inner) box1 |= fb;
            }
        }
        // eq. (multiZ) weights of orders 1 (Z~1 at taps c-1 .. c+2, Appendix) and 0 (hat at c, c+1),
        // once per target
        T wc[3][4], wl[3][2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T x = a < DIM ? xi[a] : T(0), y = T(1) - x, x2 = x * x, y2 = y * y;
            wc[a][0] = T(-0.5) * x * y2;
            wc[a][1] = T(1) + x2 * (T(1.5) * x - T(2.5));
            wc[a][2] = T(1) + y2 * (T(1.5) * y - T(2.5));
            wc[a][3] = T(-0.5) * x2 * y;
            wl[a][0] = y;
            wl[a][1] = x;
        }
        for (int q = 0; q < g.nfields; ++q) {
            int m = g.max_order;
            if (m == 2 && ((box2 >> q) & 1u)) m = 1;
            if (m >= 1 && ((box1 >> q) & 1u)) m = 0;
            cnt.oh0 += m == 0;
            cnt.oh1 += m == 1;
            cnt.oh2 += m == 2;
            if (dbg.order) dbg.order[(long long)q * g.N + jj] = (uint8_t)m;
            const T *h = f.in[q];
            T sum = T(0);
            if (m == 1) {
#pragma unroll
                for (int kz = 0; kz < KZ; ++kz) {
                    T sy = T(0);
#pragma unroll
                    for (int ky = 0; ky < 4; ++ky) {
                        const T *row = h + oz[kz] + oy[ky];
                        T sx = T(0);
#pragma unroll
                        for (int kx = 0; kx < 4; ++kx) sx += wc[0][kx] * __ldg(row + ox[kx]);
                        sy += wc[1][ky] * sx;
                    }
                    sum += (DIM == 3 ? wc[2][kz] : T(1)) * sy;
                }
            } else if (m == 0) {
#pragma unroll
                for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz) {
                    T sy = T(0);
#pragma unroll
                    for (int ky = 0; ky < 2; ++ky) {
                        const T *row = h + oz[kz + 1] + oy[ky + 1];
                        sy += wl[1][ky] * (wl[0][0] * __ldg(row + ox[1]) + wl[0][1] * __ldg(row + ox[2]));
                    }
                    sum += (DIM == 3 ? wl[2][kz] : T(1)) * sy;
                }
            } else {
                T w[3][6];
#pragma unroll
                for (int a = 0; a < DIM; ++a) zs_weights<T>(m, xi[a], w[a]);
                const int wn = 2 * m + 2;
                const int wz = DIM == 3 ? wn : 1;
                for (int kz = 0; kz < wz; ++kz) {
                    for (int ky = 0; ky < wn; ++ky) {
                        for (int kx = 0; kx < wn; ++kx) {
                            int k[3] = {c[0] - m + kx, c[1] - m + ky, DIM == 3 ? c[2] - m + kz : 0};
                            T wt = w[0][kx] * w[1][ky];
                            if (DIM == 3) wt *= w[2][kz];
                            sum += __ldg(h + node_index<DIM>(k, g.n)) * wt;
                        }
                    }
                }
            }
            f.out[q][jj] = sum;
        }
    }
    // each warp adds into its SM's copy of the counters (the launch passes the per-SM copies)
    unsigned smid;
    asm("mov.u32 %0, %%smid;" : "=r"(smid));
    flush_counters_warp(cnt, counters + (smid % SL_COUNTER_STRIPES));
}

// ------------------------------------------------------------------------------------------------
// Sec. 3.1 moments: per-block partial sums (fixed grid, fixed tree order), then one final block
// ------------------------------------------------------------------------------------------------
struct MomentGeom {
    double lo[3], dx[3], cen[3];
};

template <typename T, int DIM>
__global__ void __launch_bounds__(256)
    moments_partial_kernel(GridArgs<T> g, MomentGeom mg, const T *__restrict__ h, int pmax, double *partials)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        int k[3];
        node_coords<DIM>(i, g.n, k);
        const double hv = (double)h[i];
        acc[0] += hv;
        double r[3];
#pragma unroll
        for (int a = 0; a < DIM; ++a) r[a] = mg.lo[a] + (double)k[a] * mg.dx[a] - mg.cen[a];
        double rp[3] = {1.0, 1.0, 1.0};
        for (int p = 1; p <= pmax; ++p) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                rp[a] *= r[a];
                s += rp[a];
            }
            acc[p] += hv * s;
        }
    }
    __shared__ double red[8][256];
    for (int p = 0; p <= pmax; ++p) red[p][threadIdx.x] = acc[p];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int p = 0; p <= pmax; ++p) red[p][threadIdx.x] += red[p][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int p = 0; p <= pmax; ++p) partials[blockIdx.x * 8 + p] = red[p][0];
}

__global__ void moments_final_kernel(const double *partials, int nblocks, int pmax, double *out)
{
    const int p = threadIdx.x;
    if (p > pmax) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[b * 8 + p];
    out[p] = s;
}

// ------------------------------------------------------------------------------------------------
// strided copy of displacements (set / get)
// ------------------------------------------------------------------------------------------------
// every field plane in one launch: 16-byte vector copies when all planes are 16-byte aligned
template <typename T, bool VEC>
__global__ void __launch_bounds__(256) copy_planes_kernel(long long N, int nf, FieldPtrs<T> f)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (VEC) {
        // every plane's vector at once: nf independent 16-byte loads in flight per thread; the
        // source (the scratch planes) is not read again before it is overwritten
        const long long nv = N * (long long)sizeof(T) / 16;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += stride) {
            float4 v[SL_MAX_FIELDS];
#pragma unroll
            for (int q = 0; q < SL_MAX_FIELDS; ++q)
                if (q < nf) v[q] = __ldcs(reinterpret_cast<const float4 *>(f.in[q]) + i);
#pragma unroll
            for (int q = 0; q < SL_MAX_FIELDS; ++q)
                if (q < nf) reinterpret_cast<float4 *>(f.out[q])[i] = v[q];
        }
    } else {
        for (int q = 0; q < nf; ++q)
            for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride)
                f.out[q][i] = f.in[q][i];
    }
}

template <typename T>
__global__ void copy_disp_kernel(long long N, int dim, const T *__restrict__ src, long long ss, T *__restrict__ dst,
                                 long long dsd)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < dim; ++a) dst[i * dsd + a] = src[i * ss + a];
        for (int a = dim; a < dsd; ++a) dst[i * dsd + a] = T(0);
    }
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
template <typename T>
static FieldPtrs<T> field_ptrs(const sl_grid *g, const void *const *in, void *const *out)
{
    FieldPtrs<T> f;
    memset(&f, 0, sizeof(f));
    for (int q = 0; q < g->nfields; ++q) {
        f.in[q] = in ? (const T *)in[q] : nullptr;
        f.out[q] = out ? (T *)out[q] : nullptr;
    }
    return f;
}

template <typename T>
cudaError_t Launch<T>::advect(const sl_grid *g, void *D, double t, double dt, cudaStream_t s)
{
    const GridArgs<T> ga = make_grid_args<T>(g);
    const VelArgs<T> va = make_vel_args<T>(g, t, dt);
    const int blocks = grid_stride_blocks(g, g->N, 256);
    if (g->dim == 2)
        advect_kernel<T, 2><<<blocks, 256, 0, s>>>(ga, va, (T *)D, g->ds);
    else
        advect_kernel<T, 3><<<blocks, 256, 0, s>>>(ga, va, (T *)D, g->ds);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::advect_carried(const sl_grid *g, const void *const *fields, void *D, double dt, cudaStream_t s)
{
    const T *u[3] = {nullptr, nullptr, nullptr};
    T sc[3] = {T(0), T(0), T(0)};
    for (int a = 0; a < g->dim; ++a) {
        u[a] = (const T *)fields[g->vel_field[a]];
        sc[a] = (T)(dt / g->dx[a]);
    }
    const int blocks = grid_stride_blocks(g, g->N, 256);
    if (g->dim == 2)
        advect_carried_kernel<T, 2><<<blocks, 256, 0, s>>>(g->N, u[0], u[1], u[1], sc[0], sc[1], sc[2], (T *)D);
    else
        advect_carried_kernel<T, 3><<<blocks, 256, 0, s>>>(g->N, u[0], u[1], u[2], sc[0], sc[1], sc[2], (T *)D);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::flags(const sl_grid *g, const void *const *in, uint8_t *flags, cudaStream_t s)
{
    const GridArgs<T> ga = make_grid_args<T>(g);
    const FieldPtrs<T> f = field_ptrs<T>(g, in, nullptr);
    const int blocks = grid_stride_blocks(g, g->N, 256);
    if (g->dim == 2)
        flags_kernel<T, 2><<<blocks, 256, 0, s>>>(ga, f, flags);
    else
        flags_kernel<T, 3><<<blocks, 256, 0, s>>>(ga, f, flags);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::remap_generic(const sl_grid *g, const void *D, const uint8_t *flags, const void *const *in,
                                     void *const *out, const sl_remap_debug *dbg, cudaStream_t s)
{
    const GridArgs<T> ga = make_grid_args<T>(g);
    const FieldPtrs<T> f = field_ptrs<T>(g, in, out);
    RemapDebug<T> d;
    d.cell = dbg ? (long long *)dbg->cell : nullptr;
    d.xi = dbg ? dbg->xi : nullptr;
    d.order = dbg ? dbg->order : nullptr;
    d.status = dbg ? dbg->status : nullptr;
    const int blocks = grid_stride_blocks(g, g->N, 256);
    const int nmode = sizeof(T) == 8 ? 0 : (g->desc.newton_mode == SL_NEWTON_F64 ? 1 : 2);
    if (g->dim == 2) {
        if (nmode == 0)
            remap_generic_kernel<T, 2, 0><<<blocks, 256, 0, s>>>(ga, (const T *)D, g->ds, flags, f, d, g->stripes);
        else if (nmode == 1)
            remap_generic_kernel<T, 2, 1><<<blocks, 256, 0, s>>>(ga, (const T *)D, g->ds, flags, f, d, g->stripes);
        else
            remap_generic_kernel<T, 2, 2><<<blocks, 256, 0, s>>>(ga, (const T *)D, g->ds, flags, f, d, g->stripes);
    } else {
        if (nmode == 0)
            remap_generic_kernel<T, 3, 0><<<blocks, 256, 0, s>>>(ga, (const T *)D, g->ds, flags, f, d, g->stripes);
        else if (nmode == 1)
            remap_generic_kernel<T, 3, 1><<<blocks, 256, 0, s>>>(ga, (const T *)D, g->ds, flags, f, d, g->stripes);
        else
            remap_generic_kernel<T, 3, 2><<<blocks, 256, 0, s>>>(ga, (const T *)D, g->ds, flags, f, d, g->stripes);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::moments(const sl_grid *g, const void *field, int pmax, cudaStream_t s)
{
    const GridArgs<T> ga = make_grid_args<T>(g);
    MomentGeom mg;
    for (int a = 0; a < 3; ++a) {
        mg.lo[a] = g->desc.lo[a];
        mg.dx[a] = g->dx[a];
        mg.cen[a] = 0.5 * (g->desc.lo[a] + g->desc.hi[a]);
    }
    if (g->dim == 2)
        moments_partial_kernel<T, 2><<<SL_MOMENT_BLOCKS, 256, 0, s>>>(ga, mg, (const T *)field, pmax, g->partials);
    else
        moments_partial_kernel<T, 3><<<SL_MOMENT_BLOCKS, 256, 0, s>>>(ga, mg, (const T *)field, pmax, g->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    moments_final_kernel<<<1, 32, 0, s>>>(g->partials, SL_MOMENT_BLOCKS, pmax, g->moment_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::copy_planes(const sl_grid *g, const void *const *src, void *const *dst, cudaStream_t s)
{
    FieldPtrs<T> f;
    memset(&f, 0, sizeof(f));
    bool vec = ((size_t)g->N * sizeof(T)) % 16 == 0;
    for (int q = 0; q < g->nfields; ++q) {
        f.in[q] = (const T *)src[q];
        f.out[q] = (T *)dst[q];
        vec = vec && ((uintptr_t)src[q] & 15u) == 0 && ((uintptr_t)dst[q] & 15u) == 0;
    }
    const long long work = vec ? (long long)g->N * (long long)sizeof(T) / 16 : (long long)g->N;
    const int blocks = (int)std::min<long long>(grid_stride_blocks(g, work, 256), (long long)g->num_sms * 8);
    if (vec)
        copy_planes_kernel<T, true><<<blocks, 256, 0, s>>>((long long)g->N, g->nfields, f);
    else
        copy_planes_kernel<T, false><<<blocks, 256, 0, s>>>((long long)g->N, g->nfields, f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::copy_disp(const sl_grid *g, const void *src, int64_t src_stride, void *dst, int64_t dst_stride,
                                 cudaStream_t s)
{
    const int blocks = grid_stride_blocks(g, g->N, 256);
    copy_disp_kernel<T><<<blocks, 256, 0, s>>>((long long)g->N, g->dim, (const T *)src, (long long)src_stride,
                                               (T *)dst, (long long)dst_stride);
    return cudaGetLastError();
}

template struct Launch<double>;
template struct Launch<float>;
