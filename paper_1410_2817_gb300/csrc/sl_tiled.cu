// sl_tiled.cu -- the FP32 production kernels of the FSL step (arXiv:1410.2817) for 2-D grids.
//
// One CTA owns a TX x TY tile of target (reference) nodes.  Its targets' departure points lie
// near j - D_j, so the CTA first takes the bounding box of the start elements floor(j - D_j),
// widens it by the walk slack, the cubic stencil (Sec. 2.1: nodes c-1 .. c+2) and the limiter's
// neighbours (Sec. 2.3), and stages that window -- displacements and field values -- in shared
// memory.  The jump flags and their OR over every element's 4x4 stencil are computed once per
// window node in shared memory, so each target's element search (Sec. 2.2), order choice
// (Sec. 2.3) and tensor Z-spline sum (eq. multiZ) read shared memory only.  A target whose walk
// leaves the window, or a tile whose window does not fit, falls back to global gathers (counted).
//
// Precision: FP32 data and FP32 Newton; targets whose FP32 inversion failed or that lie within
// FACE_MARGIN of an element face are re-solved in FP64 (the element choice there is sensitive to
// rounding).
//
// The fused variant also integrates the next step's trajectories (eq. vel) for the tile's own
// nodes: the velocity is given, so D(t + dt) does not depend on the fields being remapped.
#include <limits.h>
#include <math.h>
#include <string.h>

#include "sl_internal.h"

namespace {

constexpr int TX = 32;                 // tile width (targets), one warp per row
constexpr int TY = 16;                 // tile height
constexpr int NT = 256;                // threads per CTA
constexpr int ROWS = NT / TX;          // thread rows
constexpr int TPT = TY / ROWS;         // targets per thread
constexpr int HALO = 12;               // window capacity beyond the tile on each side
constexpr int WMAX = (TX + 2 * HALO) * (TY + 2 * HALO);
constexpr int WALK_SLACK = 1;          // elements the walk may step beyond the start-cell box
constexpr float FACE_MARGIN = 2e-5f;   // FP32 location trusted only this far from a face

struct TileArgs {
    int n0, n1;
    int nfields, max_order;
    float thr;
    int max_iter, walk_max;
    const float *D;
    float *D_next;
    const float *in[SL_MAX_FIELDS];
    float *out[SL_MAX_FIELDS];
    DevCounters *counters;
};

__device__ __forceinline__ int wrapi(int k, int n)
{
    int r = k % n;
    return r < 0 ? r + n : r;
}

// start element floor(j - D_j), clamped so that garbage displacements cannot overflow the walk
__device__ __forceinline__ int start_cell(int j, float d)
{
    const float s = fminf(fmaxf((float)j - d, (float)j - 65536.f), (float)j + 65536.f);
    return finite_t(s) ? (int)floorf(s) : j;
}

__device__ __forceinline__ long long gidx(int x, int y, int n0, int n1)
{
    return (long long)wrapi(y, n1) * n0 + wrapi(x, n0);
}

// window geometry of one CTA
struct Win {
    int lox, loy, wx, wy;
    __device__ __forceinline__ bool has(int x, int y) const
    {
        return (unsigned)(x - lox) < (unsigned)wx && (unsigned)(y - loy) < (unsigned)wy;
    }
    __device__ __forceinline__ int at(int x, int y) const { return (y - loy) * wx + (x - lox); }
};

// displacement of (unwrapped) node (x, y): shared memory when inside the window
__device__ __forceinline__ float2 disp(const TileArgs &a, const Win &w, const float2 *sD, bool staged, int x, int y)
{
    if (staged && w.has(x, y)) return sD[w.at(x, y)];
    return __ldg(reinterpret_cast<const float2 *>(a.D) + gidx(x, y, a.n0, a.n1));
}

// Sec. 2.2 element search from element (cx, cy) with Newton in precision TN.
template <typename TN>
__device__ __forceinline__ int walk2(const TileArgs &a, const Win &w, const float2 *sD, bool staged, int jx, int jy,
                                     int &cx, int &cy, TN xi[3], int &hops, int &iters)
{
    const TN tol = sizeof(TN) == 8 ? TN(1e-14) : TN(1e-5);
    const TN slack = sizeof(TN) == 8 ? TN(1e-12) : TN(1e-5);
    for (int hop = 0; hop < a.walk_max; ++hop) {
        TN P[8][3];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int kx = cx + (v & 1), ky = cy + (v >> 1);
            const float2 d = disp(a, w, sD, staged, kx, ky);
            P[v][0] = TN(kx - jx) + TN(d.x);
            P[v][1] = TN(ky - jy) + TN(d.y);
        }
        int it = 0;
        const int st = newton_solve2<TN>(P, a.max_iter, tol, xi, &it);
        hops += 1;
        iters += it;
        const bool finite = finite_t(xi[0]) && finite_t(xi[1]);
        if (!finite) return st == ST_OK ? ST_NEWTON : st;
        const bool inside = xi[0] >= -slack && xi[0] <= TN(1) + slack && xi[1] >= -slack && xi[1] <= TN(1) + slack;
        if (inside) return st;
        if (xi[0] < -slack)
            cx -= 1;
        else if (xi[0] > TN(1) + slack)
            cx += 1;
        if (xi[1] < -slack)
            cy -= 1;
        else if (xi[1] > TN(1) + slack)
            cy += 1;
    }
    return ST_LOCATE;
}

// Sec. 2.3 flags of one node from global memory (fallback path)
__device__ __forceinline__ unsigned node_flags_global(const TileArgs &a, int x, int y)
{
    if (a.thr < 0.f) return 0u;
    unsigned bits = 0;
    const long long c = gidx(x, y, a.n0, a.n1);
    const long long xm = gidx(x - 1, y, a.n0, a.n1), xp = gidx(x + 1, y, a.n0, a.n1);
    const long long ym = gidx(x, y - 1, a.n0, a.n1), yp = gidx(x, y + 1, a.n0, a.n1);
    for (int f = 0; f < a.nfields; ++f) {
        const float *h = a.in[f];
        const float h0 = __ldg(h + c);
        const bool hit = jump_test<float>(__ldg(h + xm), h0, __ldg(h + xp), a.thr) ||
                         jump_test<float>(__ldg(h + ym), h0, __ldg(h + yp), a.thr);
        bits |= hit ? (1u << f) : 0u;
    }
    return bits;
}

// Z~1 weights of taps c-1 .. c+2 at local coordinate x (Appendix), and Z~0 in the middle two
__device__ __forceinline__ void cubic_weights(float x, float w[4])
{
    const float y = 1.f - x, x2 = x * x, y2 = y * y;
    w[0] = -0.5f * x * y2;
    w[1] = fmaf(x2, fmaf(1.5f, x, -2.5f), 1.f);
    w[2] = fmaf(y2, fmaf(1.5f, y, -2.5f), 1.f);
    w[3] = -0.5f * x2 * y;
}

template <bool FUSED>
__global__ void __launch_bounds__(NT, 2) remap_tiled2d_kernel(const TileArgs a, const VelArgs<float> vn)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *sD = reinterpret_cast<float2 *>(smem);
    float *sH = reinterpret_cast<float *>(sD + WMAX);
    uint8_t *sF = reinterpret_cast<uint8_t *>(sH + a.nfields * WMAX);
    uint8_t *sR = sF + WMAX;
    uint8_t *sB = sR + WMAX;
    __shared__ int sBox[4];

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    if (threadIdx.x < 4) sBox[threadIdx.x] = (threadIdx.x < 2) ? INT_MAX : INT_MIN;

    // ---- phase 1: start elements floor(j - D_j) and their bounding box ----------------------
    int cx[TPT], cy[TPT];
    bool valid[TPT];
    int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN;
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
        valid[k] = jx < a.n0 && jy < a.n1;
        cx[k] = cy[k] = 0;
        if (valid[k]) {
            const float2 d = __ldg(reinterpret_cast<const float2 *>(a.D) + (long long)jy * a.n0 + jx);
            cx[k] = start_cell(jx, d.x);
            cy[k] = start_cell(jy, d.y);
            mnx = min(mnx, cx[k]);
            mny = min(mny, cy[k]);
            mxx = max(mxx, cx[k]);
            mxy = max(mxy, cy[k]);
        }
    }
    __syncthreads();
    mnx = __reduce_min_sync(0xffffffffu, mnx);
    mny = __reduce_min_sync(0xffffffffu, mny);
    mxx = __reduce_max_sync(0xffffffffu, mxx);
    mxy = __reduce_max_sync(0xffffffffu, mxy);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&sBox[0], mnx);
        atomicMin(&sBox[1], mny);
        atomicMax(&sBox[2], mxx);
        atomicMax(&sBox[3], mxy);
    }
    __syncthreads();
    Win w;
    const long long wxl = (long long)sBox[2] - sBox[0] + 2 * WALK_SLACK + 6;
    const long long wyl = (long long)sBox[3] - sBox[1] + 2 * WALK_SLACK + 6;
    const bool staged = wxl > 0 && wyl > 0 && wxl <= WMAX && wyl <= WMAX && wxl * wyl <= WMAX;
    w.lox = staged ? sBox[0] - WALK_SLACK - 2 : 0;
    w.loy = staged ? sBox[1] - WALK_SLACK - 2 : 0;
    w.wx = staged ? (int)wxl : 0;
    w.wy = staged ? (int)wyl : 0;
    const int nwin = w.wx * w.wy;

    // ---- phase 2: stage displacements and fields of the window ------------------------------
    for (int idx = threadIdx.x; idx < nwin; idx += NT) {
        const int wy = idx / w.wx, wx = idx - wy * w.wx;
        const long long gi = gidx(w.lox + wx, w.loy + wy, a.n0, a.n1);
        sD[idx] = __ldg(reinterpret_cast<const float2 *>(a.D) + gi);
        for (int f = 0; f < a.nfields; ++f) sH[f * WMAX + idx] = __ldg(a.in[f] + gi);
    }
    __syncthreads();

    // ---- phase 3: jump flags (Sec. 2.3) and their OR over each element's 4x4 stencil ---------
    for (int idx = threadIdx.x; idx < nwin; idx += NT) {
        const int wy = idx / w.wx, wx = idx - wy * w.wx;
        unsigned bits = 0;
        if (a.thr >= 0.f && wx >= 1 && wx < w.wx - 1 && wy >= 1 && wy < w.wy - 1) {
            for (int f = 0; f < a.nfields; ++f) {
                const float *h = sH + f * WMAX;
                const float h0 = h[idx];
                const bool hit = jump_test<float>(h[idx - 1], h0, h[idx + 1], a.thr) ||
                                 jump_test<float>(h[idx - w.wx], h0, h[idx + w.wx], a.thr);
                bits |= hit ? (1u << f) : 0u;
            }
        }
        sF[idx] = (uint8_t)bits;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nwin; idx += NT) {
        const int wy = idx / w.wx, wx = idx - wy * w.wx;
        uint8_t r = 0;
        if (wx >= 2 && wx < w.wx - 3) r = sF[idx - 1] | sF[idx] | sF[idx + 1] | sF[idx + 2];
        sR[idx] = r;
        (void)wy;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nwin; idx += NT) {
        const int wy = idx / w.wx;
        uint8_t b = 0;
        if (wy >= 2 && wy < w.wy - 3) b = sR[idx - w.wx] | sR[idx] | sR[idx + w.wx] | sR[idx + 2 * w.wx];
        sB[idx] = b;
    }
    __syncthreads();

    // ---- phase 4: per target: search, Newton, order, tensor Z-spline sum ---------------------
    LocalCounters cnt;
    cnt.clear();
    if (!staged && threadIdx.x == 0) cnt.fallback = 1;
#pragma unroll 1
    for (int k = 0; k < TPT; ++k) {
        if (!valid[k]) continue;
        const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
        const long long jj = (long long)jy * a.n0 + jx;
        int ex = cx[k], ey = cy[k], hops = 0, iters = 0;
        float xf[3] = {0.f, 0.f, 0.f};
        int st = walk2<float>(a, w, sD, staged, jx, jy, ex, ey, xf, hops, iters);
        float xi0 = xf[0], xi1 = xf[1];
        const bool redo = st != ST_OK || fabsf(xi0) < FACE_MARGIN || fabsf(1.f - xi0) < FACE_MARGIN ||
                          fabsf(xi1) < FACE_MARGIN || fabsf(1.f - xi1) < FACE_MARGIN;
        if (redo) {
            double xd[3] = {0.0, 0.0, 0.0};
            if (st == ST_LOCATE || st == ST_FOLD) {
                ex = cx[k];
                ey = cy[k];
            }
            st = walk2<double>(a, w, sD, staged, jx, jy, ex, ey, xd, hops, iters);
            xi0 = (float)xd[0];
            xi1 = (float)xd[1];
            cnt.f64 += 1;
        }
        cnt.targets += 1;
        cnt.hops += hops;
        cnt.hops_max = max(cnt.hops_max, (unsigned)hops);
        cnt.iters += iters;
        cnt.iters_max = max(cnt.iters_max, (unsigned)iters);
        if (st != ST_OK) {
            cnt.fl += st == ST_LOCATE;
            cnt.fn += st == ST_NEWTON;
            cnt.ff += st == ST_FOLD;
            for (int f = 0; f < a.nfields; ++f) a.out[f][jj] = __ldg(a.in[f] + jj);
        } else {
            // Sec. 2.3: the fields flagged anywhere in the element's 4x4 stencil drop to linear
            const bool fast = staged && ex - 2 >= w.lox && ex + 3 < w.lox + w.wx && ey - 2 >= w.loy &&
                              ey + 3 < w.loy + w.wy;
            unsigned bits = 0;
            if (a.max_order >= 1) {
                if (fast) {
                    bits = sB[w.at(ex, ey)];
                } else {
                    for (int q = 0; q < 16; ++q) bits |= node_flags_global(a, ex - 1 + (q & 3), ey - 1 + (q >> 2));
                }
            }
            float wc[2][4], wl[2][2];
            cubic_weights(xi0, wc[0]);
            cubic_weights(xi1, wc[1]);
            wl[0][0] = 1.f - xi0;
            wl[0][1] = xi0;
            wl[1][0] = 1.f - xi1;
            wl[1][1] = xi1;
            for (int f = 0; f < a.nfields; ++f) {
                const bool lin = a.max_order == 0 || ((bits >> f) & 1u);
                cnt.oh0 += lin;
                cnt.oh1 += !lin;
                float sum = 0.f;
                if (fast) {
                    const float *h = sH + f * WMAX;
                    if (lin) {
                        const int i0 = w.at(ex, ey);
                        const float r0 = fmaf(wl[0][1], h[i0 + 1], wl[0][0] * h[i0]);
                        const float r1 = fmaf(wl[0][1], h[i0 + w.wx + 1], wl[0][0] * h[i0 + w.wx]);
                        sum = fmaf(wl[1][1], r1, wl[1][0] * r0);
                    } else {
                        int i0 = w.at(ex - 1, ey - 1);
#pragma unroll
                        for (int ky = 0; ky < 4; ++ky) {
                            const float r = fmaf(wc[0][3], h[i0 + 3],
                                                 fmaf(wc[0][2], h[i0 + 2], fmaf(wc[0][1], h[i0 + 1], wc[0][0] * h[i0])));
                            sum = fmaf(wc[1][ky], r, sum);
                            i0 += w.wx;
                        }
                    }
                } else {
                    const float *h = a.in[f];
                    const int m = lin ? 0 : 1, wn = lin ? 2 : 4;
                    for (int ky = 0; ky < wn; ++ky) {
                        float r = 0.f;
                        for (int kx = 0; kx < wn; ++kx) {
                            const float wx_ = lin ? wl[0][kx] : wc[0][kx];
                            r = fmaf(wx_, __ldg(h + gidx(ex - m + kx, ey - m + ky, a.n0, a.n1)), r);
                        }
                        sum = fmaf(lin ? wl[1][ky] : wc[1][ky], r, sum);
                    }
                }
                a.out[f][jj] = sum;
            }
        }
        if (FUSED && a.D_next != nullptr) {
            float X[3] = {vn.lo[0] + (float)jx * vn.dx[0], vn.lo[1] + (float)jy * vn.dx[1], 0.f}, d[3];
            rk4_cells<float, 2>(vn, X, d);
            reinterpret_cast<float2 *>(a.D_next)[jj] = make_float2(d[0], d[1]);
        }
    }
    flush_counters(cnt, a.counters);
}

size_t tiled_smem_bytes(int nfields) { return (size_t)WMAX * (sizeof(float2) + sizeof(float) * nfields + 3); }

TileArgs make_tile_args(const sl_grid *g, const void *D, void *D_next, const void *const *in, void *const *out)
{
    TileArgs a;
    memset(&a, 0, sizeof(a));
    a.n0 = (int)g->n[0];
    a.n1 = (int)g->n[1];
    a.nfields = g->nfields;
    a.max_order = g->desc.max_order;
    a.thr = (float)g->desc.limiter_threshold;
    a.max_iter = g->desc.newton_max_iter;
    a.walk_max = g->desc.walk_max;
    a.D = (const float *)D;
    a.D_next = (float *)D_next;
    for (int f = 0; f < g->nfields; ++f) {
        a.in[f] = (const float *)in[f];
        a.out[f] = (float *)out[f];
    }
    a.counters = g->counters;
    return a;
}

template <bool FUSED>
cudaError_t launch_tiled(const sl_grid *g, const TileArgs &a, const VelArgs<float> &vn, cudaStream_t s)
{
    const size_t smem = tiled_smem_bytes(g->nfields);
    // the opt-in shared-memory limit is a per-device function attribute: set it once per device
    // to the largest size any field count needs
    static bool configured[2][64] = {};
    const int dev = g->device & 63;
    if (!configured[FUSED][dev]) {
        cudaError_t e = cudaFuncSetAttribute(remap_tiled2d_kernel<FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tiled_smem_bytes(SL_MAX_FIELDS));
        if (e != cudaSuccess) return e;
        configured[FUSED][dev] = true;
    }
    dim3 grid((unsigned)((g->n[0] + TX - 1) / TX), (unsigned)((g->n[1] + TY - 1) / TY));
    remap_tiled2d_kernel<FUSED><<<grid, NT, smem, s>>>(a, vn);
    return cudaGetLastError();
}

}  // namespace

// 2-D: one tiled launch; 3-D: flags + three box-OR passes + one blocked launch
int tiled_kernels_per_call(const sl_grid *g) { return g->dim == 2 ? 1 : 5; }

template <typename T>
bool Launch<T>::tiled_supported(const sl_grid *g)
{
    if (sizeof(T) != 4 || g->desc.max_order > 1 || g->desc.walk_start != SL_START_BACKWARD) return false;
    if (g->dim == 3) return true;
    return tiled_smem_bytes(g->nfields) <= 200 * 1024;
}

template <typename T>
cudaError_t Launch<T>::remap_tiled(const sl_grid *g, const void *D, const void *const *in, void *const *out,
                                   cudaStream_t s)
{
    if (!tiled_supported(g)) return cudaErrorNotSupported;
    if (g->dim == 3) {
        cudaError_t e = launch_box_flags3d(g, in, g->flags, g->flags2, s);
        if (e != cudaSuccess) return e;
        return launch_blocked3d(g, D, nullptr, g->flags2, 0.0, 0.0, false, in, out, s);
    }
    const TileArgs a = make_tile_args(g, D, nullptr, in, out);
    VelArgs<float> vn;
    memset(&vn, 0, sizeof(vn));
    return launch_tiled<false>(g, a, vn, s);
}

template <typename T>
cudaError_t Launch<T>::step_fused(const sl_grid *g, const void *D, void *D_next, double t_next, double dt,
                                  const void *const *in, void *const *out, cudaStream_t s)
{
    if (!tiled_supported(g)) return cudaErrorNotSupported;
    if (g->dim == 3) {
        cudaError_t e = launch_box_flags3d(g, in, g->flags, g->flags2, s);
        if (e != cudaSuccess) return e;
        return launch_blocked3d(g, D, D_next, g->flags2, t_next, dt, true, in, out, s);
    }
    const TileArgs a = make_tile_args(g, D, D_next, in, out);
    const VelArgs<float> vn = make_vel_args<float>(g, t_next, dt);
    return launch_tiled<true>(g, a, vn, s);
}

template bool Launch<double>::tiled_supported(const sl_grid *);
template bool Launch<float>::tiled_supported(const sl_grid *);
template cudaError_t Launch<double>::remap_tiled(const sl_grid *, const void *, const void *const *, void *const *,
                                                 cudaStream_t);
template cudaError_t Launch<float>::remap_tiled(const sl_grid *, const void *, const void *const *, void *const *,
                                                cudaStream_t);
template cudaError_t Launch<double>::step_fused(const sl_grid *, const void *, void *, double, double,
                                                const void *const *, void *const *, cudaStream_t);
template cudaError_t Launch<float>::step_fused(const sl_grid *, const void *, void *, double, double,
                                               const void *const *, void *const *, cudaStream_t);
