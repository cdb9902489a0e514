// sl_blocked3d.cu -- the FP32 production kernels of the FSL step (arXiv:1410.2817) for 3-D grids.
//
//   * box_flags: the jump flags of Sec. 2.3 are computed once per node and OR-ed over every
//     element's 4x4x4 stencil [c-1, c+2]^3 (separable: x, then y, then z), so choosing the order
//     of a target (Sec. 2.3) costs one byte load;
//   * remap_blocked3d_kernel: one thread per target; a CTA covers a 16x4x4 block of targets so
//     that the element search (Sec. 2.2, Newton in FP32 with FP64 re-solves near faces) and the
//     64-tap tricubic sums (eq. multiZ) of neighbouring targets hit the same L1 lines;
//   * remap_staged3d_kernel (plain remaps of up to 2 fields): the same blocks and element search,
//     with the field values of the block's stencils copied to shared memory (TMA boxes inside the
//     grid, per-element copies across the periodic seam) while the search runs, and the tap sums
//     read from there.
// Both share the element search, the refined start and the tap sums, so they give identical
// results.  The fused variants also integrate the next step's trajectories (eq. vel) for their
// own nodes.
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "sl_async.cuh"
#include "sl_internal.h"

namespace {

constexpr int BX = 16, BY = 4, BZ = 4, NT3 = BX * BY * BZ;

struct Geo3 {
    int n0, n1, n2;
};

__device__ __forceinline__ int wrap3(int k, int n) { return wrap_idx(k, n); }

__device__ __forceinline__ long long lin3(const Geo3 &g, int x, int y, int z)
{
    return ((long long)wrap3(z, g.n2) * g.n1 + wrap3(y, g.n1)) * g.n0 + wrap3(x, g.n0);
}

struct Fields3 {
    const float *in[SL_MAX_FIELDS];
    float *out[SL_MAX_FIELDS];
};

// ---- Sec. 2.3 flags and their OR over each element's stencil [c-1, c+2]^3 ------------------
// Two passes.  flags_x3d: a warp covers 32 consecutive nodes x0-1 .. x0+30 of one row, tests each
// node (6 neighbours per field, wrapped) and ORs the flags of x-1 .. x+2 with shuffles, writing
// the 29 nodes x0 .. x0+28.  box_yz3d: ORs those bytes over y-1 .. y+2 and z-1 .. z+2.  Blocks
// are 32 x 8 threads over (x, y) and loop over y and z, so no index is divided.
constexpr int FX = 29;  // nodes written per warp and row by flags_x3d

template <int NFM>
__global__ void __launch_bounds__(256)
    flags_x3d_kernel(Geo3 g, int nfields, float thr, Fields3 f, uint8_t *out, int zchunk)
{
    const int lane = threadIdx.x;
    const int x0 = blockIdx.x * FX;
    const int x = wrap_idx(x0 - 1 + lane, g.n0);  // rows shorter than a warp wrap more than once
    const int xm = wrap_near(x - 1, g.n0), xp = wrap_near(x + 1, g.n0);
    const long long plane = (long long)g.n0 * g.n1;
    const int zb = blockIdx.z * zchunk, ze = min(g.n2, zb + zchunk);
    for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < g.n1; y += gridDim.y * blockDim.y) {
        const long long yc = (long long)y * g.n0 + x, ym = (long long)wrap_near(y - 1, g.n1) * g.n0 + x,
                        yp = (long long)wrap_near(y + 1, g.n1) * g.n0 + x;
        const long long xl = (long long)y * g.n0 + xm, xr = (long long)y * g.n0 + xp;
        // a thread walks z through its chunk keeping the centre values of planes z-1 and z
        float cm[NFM], cc[NFM];
#pragma unroll
        for (int q = 0; q < NFM; ++q) {
            cm[q] = cc[q] = 0.f;
            if (q < nfields) {
                cm[q] = __ldg(f.in[q] + wrap_near(zb - 1, g.n2) * plane + yc);
                cc[q] = __ldg(f.in[q] + zb * plane + yc);
            }
        }
#pragma unroll 2
        for (int z = zb; z < ze; ++z) {
            const long long zc = z * plane, zp = wrap_near(z + 1, g.n2) * plane;
            unsigned bits = 0;
#pragma unroll
            for (int q = 0; q < NFM; ++q) {
                if (q < nfields) {
                    const float *h = f.in[q];
                    const float cp = __ldg(h + zp + yc);
                    const float l = __ldg(h + zc + xl), r = __ldg(h + zc + xr);
                    const float d = __ldg(h + zc + ym), u = __ldg(h + zc + yp);
                    const bool hit = jump_test<float>(l, cc[q], r, thr) | jump_test<float>(d, cc[q], u, thr) |
                                     jump_test<float>(cm[q], cc[q], cp, thr);
                    bits |= (hit && thr >= 0.f) ? (1u << q) : 0u;
                    cm[q] = cc[q];
                    cc[q] = cp;
                }
            }
            // lane l holds node x0 - 1 + l: the OR over x-1 .. x+2 for l = 1 .. 29
            const unsigned left = __shfl_up_sync(0xffffffffu, bits, 1);
            const unsigned r1 = __shfl_down_sync(0xffffffffu, bits, 1);
            const unsigned r2 = __shfl_down_sync(0xffffffffu, bits, 2);
            const int xo = x0 - 1 + lane;
            if (lane >= 1 && lane <= FX && xo < g.n0)
                out[zc + (long long)y * g.n0 + xo] = (uint8_t)(left | bits | r1 | r2);
        }
    }
}

// OR over y-1 .. y+2 and z-1 .. z+2; W = 4 handles 4 consecutive nodes per thread with 32-bit
// loads (rows of a multiple of 4 nodes), W = 1 one node with byte loads.
template <int W>
__global__ void __launch_bounds__(256) box_yz3d_kernel(Geo3 g, const uint8_t *__restrict__ in, uint8_t *out)
{
    typedef typename std::conditional<W == 4, unsigned, uint8_t>::type V;
    const int x = (blockIdx.x * 32 + threadIdx.x) * W;
    if (x >= g.n0) return;  // no barriers below
    const long long plane = (long long)g.n0 * g.n1;
    for (int z = blockIdx.z; z < g.n2; z += gridDim.z) {
        long long zo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) zo[k] = wrap_near(z - 1 + k, g.n2) * plane;
        for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < g.n1; y += gridDim.y * blockDim.y) {
            V r = 0;
#pragma unroll
            for (int ky = 0; ky < 4; ++ky) {
                const long long yo = (long long)wrap_near(y - 1 + ky, g.n1) * g.n0 + x;
#pragma unroll
                for (int kz = 0; kz < 4; ++kz) r |= __ldg(reinterpret_cast<const V *>(in + zo[kz] + yo));
            }
            *reinterpret_cast<V *>(out + z * plane + (long long)y * g.n0 + x) = r;
        }
    }
}

__device__ __forceinline__ void cubic_w(float x, float w[4])
{
    const float y = 1.f - x, x2 = x * x, y2 = y * y;
    w[0] = -0.5f * x * y2;
    w[1] = fmaf(x2, fmaf(1.5f, x, -2.5f), 1.f);
    w[2] = fmaf(y2, fmaf(1.5f, y, -2.5f), 1.f);
    w[3] = -0.5f * x2 * y;
}

// The 8 vertex displacements of element c (vertex v = x + 2 y + 4 z offsets) from global memory;
// D is padded to 4 floats per node.
struct GlobalD3 {
    Geo3 g;
    const float4 *D;
    __device__ __forceinline__ void load8(const int c[3], float4 d8[8]) const
    {
        // c[a] in [0, n[a] - 2] on every axis (a negative c fails the unsigned compare)
        if ((unsigned)c[0] < (unsigned)(g.n0 - 1) && (unsigned)c[1] < (unsigned)(g.n1 - 1) &&
            (unsigned)c[2] < (unsigned)(g.n2 - 1)) {
            // the element does not touch the periodic seam: vertices at fixed offsets
            const long long sy = g.n0, sz = (long long)g.n0 * g.n1;
            const float4 *b = D + ((long long)c[2] * g.n1 + c[1]) * g.n0 + c[0];
            d8[0] = __ldg(b);
            d8[1] = __ldg(b + 1);
            d8[2] = __ldg(b + sy);
            d8[3] = __ldg(b + sy + 1);
            d8[4] = __ldg(b + sz);
            d8[5] = __ldg(b + sz + 1);
            d8[6] = __ldg(b + sz + sy);
            d8[7] = __ldg(b + sz + sy + 1);
        } else {
#pragma unroll
            for (int v = 0; v < 8; ++v) d8[v] = __ldg(D + lin3(g, c[0] + (v & 1), c[1] + ((v >> 1) & 1), c[2] + (v >> 2)));
        }
    }
};

// Sec. 2.2 element search in 3-D from element c, Newton in precision TN; the vertices from `src`
// (GlobalD3, or a staged window with global reads where it ends).
template <typename TN, class Src>
__device__ __forceinline__ int walk3(const Src &src, int max_iter, int walk_max, const int j[3], int c[3], TN xi[3],
                                     int &hops, int &iters, bool *degen)
{
    const TN tol = sizeof(TN) == 8 ? TN(1e-14) : TN(SL_NEWTON_TOL_F32);
    const TN slack = sizeof(TN) == 8 ? TN(1e-12) : TN(SL_SLACK_F32);
    CycleCheck cyc;
    cyc.start(c[0], c[1], c[2]);
    for (int hop = 0; hop < walk_max; ++hop) {
        TN P[8][3];
        float4 d8[8];
        src.load8(c, d8);
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            P[v][0] = TN(c[0] + (v & 1) - j[0]) + TN(d8[v].x);
            P[v][1] = TN(c[1] + ((v >> 1) & 1) - j[1]) + TN(d8[v].y);
            P[v][2] = TN(c[2] + (v >> 2) - j[2]) + TN(d8[v].z);
        }
        int it = 0;
        const int st = newton_solve3<TN>(P, max_iter, tol, xi, &it, degen);
        hops += 1;
        iters += it;
        bool finite = true, inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            finite &= finite_t(xi[a]);
            inside &= xi[a] >= -slack && xi[a] <= TN(1) + slack;
        }
        if (!finite) return st == ST_OK ? ST_NEWTON : st;
        if (inside) return st;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (xi[a] < -slack)
                c[a] -= 1;
            else if (xi[a] > TN(1) + slack)
                c[a] += 1;
        }
        if (cyc.step(c[0], c[1], c[2])) return ST_LOCATE;
    }
    return ST_LOCATE;
}

// FP64 re-solve of a target whose FP32 inversion failed or whose element is nearly degenerate
// (rare: out of line, arguments and result by value, so that the main path keeps its element and
// coordinates in registers)
struct Resolve3 {
    int st, c0, c1, c2;
    float x0, x1, x2;
    int hops, iters;
};

__device__ __noinline__ Resolve3 resolve3_f64(const float4 *__restrict__ D, int n0, int n1, int n2, int max_iter,
                                              int walk_max, int j0, int j1, int j2, int st32, int cx, int cy, int cz,
                                              int sx, int sy, int sz)
{
    const Geo3 g = {n0, n1, n2};
    const int j[3] = {j0, j1, j2};
    int c[3] = {cx, cy, cz};
    if (st32 == ST_LOCATE || st32 == ST_FOLD) {
        c[0] = sx;
        c[1] = sy;
        c[2] = sz;
    }
    double xd[3] = {0.0, 0.0, 0.0};
    bool degd = false;
    int hops = 0, iters = 0;
    const GlobalD3 src = {g, D};
    const int st = walk3<double>(src, max_iter, walk_max, j, c, xd, hops, iters, &degd);
    Resolve3 r;
    r.st = st;
    r.c0 = c[0];
    r.c1 = c[1];
    r.c2 = c[2];
    r.x0 = (float)xd[0];
    r.x1 = (float)xd[1];
    r.x2 = (float)xd[2];
    r.hops = hops;
    r.iters = iters;
    return r;
}

struct Blocked3Args {
    Geo3 g;
    int nfields, max_order, max_iter, walk_max;
    const float4 *D;
    float4 *D_next;
    const uint8_t *box;   // OR of the flags over each element's 4x4x4 stencil
    Fields3 f;
    DevCounters *counters;  // the grid's SL_COUNTER_STRIPES per-SM copies of its counters
};

// The 4x4x4 stencil taps of element c from global memory: node offsets along each axis (direct when
// the stencil does not cross the periodic seam, wrapped otherwise; 32-bit: the blocked kernels
// take grids below 2^31 nodes), shared by all fields.  A tap source gives, for a pair of fields q,
// q + 1 (an odd last field pairs with itself), their planes (fields), a stencil row of them (row)
// and the row's 4 taps (tap).
struct GlobalTaps3 {
    const Fields3 &f;
    int nfields;
    int ox[4];
    unsigned oy[4], oz[4];
    struct Ptr2 {
        const float *a, *b;
    };
    __device__ __forceinline__ GlobalTaps3(const Geo3 &g, const Fields3 &f_, int nf, const int c[3]) : f(f_), nfields(nf)
    {
        const bool inner = (unsigned)(c[0] - 1) < (unsigned)(g.n0 - 3) && (unsigned)(c[1] - 1) < (unsigned)(g.n1 - 3) &&
                           (unsigned)(c[2] - 1) < (unsigned)(g.n2 - 3);
        const unsigned sy = (unsigned)g.n0, sz = (unsigned)g.n0 * (unsigned)g.n1;
        if (inner) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ox[k] = c[0] - 1 + k;
                oy[k] = (unsigned)(c[1] - 1 + k) * sy;
                oz[k] = (unsigned)(c[2] - 1 + k) * sz;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ox[k] = wrap3(c[0] - 1 + k, g.n0);
                oy[k] = (unsigned)wrap3(c[1] - 1 + k, g.n1) * sy;
                oz[k] = (unsigned)wrap3(c[2] - 1 + k, g.n2) * sz;
            }
        }
    }
    __device__ __forceinline__ Ptr2 fields(int q) const
    {
        const float *ha = f.in[q];
        return {ha, q + 1 < nfields ? f.in[q + 1] : ha};
    }
    __device__ __forceinline__ Ptr2 row(const Ptr2 &p, int kz, int ky) const
    {
        const unsigned o = oz[kz] + oy[ky];
        return {p.a + o, p.b + o};
    }
    __device__ __forceinline__ float2 tap(const Ptr2 &r, int kx) const
    {
        return make_float2(__ldg(r.a + ox[kx]), __ldg(r.b + ox[kx]));
    }
};

// eq. (multiZ) in 3-D for up to NFM fields: the 4x4x4 cubic (Z~1) sums and the trilinear (Z~0)
// sums over the element's 8 vertices in one pass, the taps from `tp` (GlobalTaps3 or the staged
// field window).  Fields run in pairs on packed FP32x2 FMAs (each lane rounds as fmaf does).
template <int NFM, class Taps>
__device__ __forceinline__ void tap_sums(const Taps &tp, int nfields, const float wc[3][4], const float xf[3],
                                         float cub[NFM], float lin[NFM])
{
    const float2 w0 = make_float2(wc[0][0], wc[0][0]), w1 = make_float2(wc[0][1], wc[0][1]);
    const float2 w2 = make_float2(wc[0][2], wc[0][2]), w3 = make_float2(wc[0][3], wc[0][3]);
    const float2 u0 = make_float2(1.f - xf[0], 1.f - xf[0]), u1 = make_float2(xf[0], xf[0]);
#pragma unroll
    for (int q = 0; q < NFM; q += 2) {
        if (q >= nfields) break;
        const auto fp = tp.fields(q);
        float2 cs = make_float2(0.f, 0.f), ls = cs;
#pragma unroll
        for (int kz = 0; kz < 4; ++kz) {
            float2 syc = make_float2(0.f, 0.f), syl = syc;
#pragma unroll
            for (int ky = 0; ky < 4; ++ky) {
                const auto row = tp.row(fp, kz, ky);
                const float2 t0 = tp.tap(row, 0), t1 = tp.tap(row, 1), t2 = tp.tap(row, 2), t3 = tp.tap(row, 3);
                float2 r = __fmul2_rn(w0, t0);
                r = __ffma2_rn(w1, t1, r);
                r = __ffma2_rn(w2, t2, r);
                r = __ffma2_rn(w3, t3, r);
                syc = __ffma2_rn(make_float2(wc[1][ky], wc[1][ky]), r, syc);
                if (ky == 1 || ky == 2) {
                    const float v = ky == 1 ? 1.f - xf[1] : xf[1];
                    syl = __ffma2_rn(make_float2(v, v), __ffma2_rn(u1, t2, __fmul2_rn(u0, t1)), syl);
                }
            }
            cs = __ffma2_rn(make_float2(wc[2][kz], wc[2][kz]), syc, cs);
            if (kz == 1 || kz == 2) {
                const float v = kz == 1 ? 1.f - xf[2] : xf[2];
                ls = __ffma2_rn(make_float2(v, v), syl, ls);
            }
        }
        cub[q] = cs.x;
        lin[q] = ls.x;
        if (q + 1 < NFM) {
            cub[q + 1] = cs.y;
            lin[q + 1] = ls.y;
        }
    }
}

// Start element of a target: one fixed-point step s <- j - D(s) from s0 = j - D_j, with D(s0)
// trilinear over the 8 nodes around s0 (the walk still decides); c keeps floor(s0) where the step
// is not finite or moves by 4 cells or more.
template <class Src>
__device__ __forceinline__ void refined_start3(const Src &src, const int j[3], const float s0[3], const int c0[3],
                                               int c[3])
{
    const float fx = s0[0] - (float)c0[0], fy = s0[1] - (float)c0[1], fz = s0[2] - (float)c0[2];
    float dd[3] = {0.f, 0.f, 0.f};
    float4 d8[8];
    src.load8(c0, d8);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const float4 d = d8[v];
        const float w = ((v & 1) ? fx : 1.f - fx) * (((v >> 1) & 1) ? fy : 1.f - fy) * ((v >> 2) ? fz : 1.f - fz);
        dd[0] = fmaf(w, d.x, dd[0]);
        dd[1] = fmaf(w, d.y, dd[1]);
        dd[2] = fmaf(w, d.z, dd[2]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        c[q] = c0[q];
        const float r = (float)j[q] - dd[q];
        if (finite_t(r) && fabsf(r - s0[q]) < 4.f) c[q] = (int)floorf(r);
    }
}

// s0 = j - D_j (clamped to 65536 cells; j where not finite) and its element
__device__ __forceinline__ void start_point3(const int j[3], const float4 dj, float s0[3], int c0[3])
{
    const float djv[3] = {dj.x, dj.y, dj.z};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float s = fminf(fmaxf((float)j[q] - djv[q], (float)j[q] - 65536.f), (float)j[q] + 65536.f);
        s0[q] = finite_t(s) ? s : (float)j[q];
        c0[q] = (int)floorf(s0[q]);
    }
}

// N64: every target's element search and Newton inversion in FP64 (SL_NEWTON_F64) from the refined
// start; otherwise in FP32 with an FP64 re-solve of failed or near-degenerate targets.
template <int NFM, bool FUSED, bool N64>
__global__ void __launch_bounds__(NT3, 4) remap_blocked3d_kernel(const Blocked3Args a, const VelArgs<float> vn)
{
    const Geo3 &g = a.g;
    const int jx = blockIdx.x * BX + threadIdx.x % BX;
    const int jy = blockIdx.y * BY + (threadIdx.x / BX) % BY;
    const int jz = blockIdx.z * BZ + threadIdx.x / (BX * BY);
    LocalCounters cnt;
    cnt.clear();
    if (jx < g.n0 && jy < g.n1 && jz < g.n2) {
        const long long jj = ((long long)jz * g.n1 + jy) * g.n0 + jx;
        const int j[3] = {jx, jy, jz};
        const GlobalD3 src = {g, a.D};
        int c[3], c0[3];
        float s0[3];
        start_point3(j, __ldg(a.D + jj), s0, c0);
        refined_start3(src, j, s0, c0, c);
        int hops = 0, iters = 0;
        float xf[3] = {0.f, 0.f, 0.f};
        bool degen = false;
        int st = ST_OK;
        if (!N64) st = walk3<float>(src, a.max_iter, a.walk_max, j, c, xf, hops, iters, &degen);
        if (N64 || st != ST_OK || degen) {
            const Resolve3 r = resolve3_f64(a.D, g.n0, g.n1, g.n2, a.max_iter, a.walk_max, j[0], j[1], j[2], st, c[0],
                                            c[1], c[2], c0[0], c0[1], c0[2]);
            st = r.st;
            c[0] = r.c0;
            c[1] = r.c1;
            c[2] = r.c2;
            xf[0] = r.x0;
            xf[1] = r.x1;
            xf[2] = r.x2;
            hops += r.hops;
            iters += r.iters;
            cnt.f64 += N64 ? 0 : 1;
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
            for (int q = 0; q < a.nfields; ++q) a.f.out[q][jj] = __ldg(a.f.in[q] + jj);
        } else {
            float wc[3][4];
#pragma unroll
            for (int q = 0; q < 3; ++q) cubic_w(xf[q], wc[q]);
            const GlobalTaps3 tp(g, a.f, a.nfields, c);
            unsigned bits = 0xffu;
            if (a.max_order >= 1) bits = __ldg(a.box + (tp.oz[1] + tp.oy[1] + (unsigned)tp.ox[1]));
            // one instance of the tap loop (a second one for stencils away from the x seam made
            // the kernel larger and measured slower)
            float cub[NFM], lin[NFM];
            tap_sums<NFM>(tp, a.nfields, wc, xf, cub, lin);
#pragma unroll
            for (int q = 0; q < NFM; ++q) {
                if (q >= a.nfields) break;
                const bool useL = ((bits >> q) & 1u) != 0u;
                cnt.oh0 += useL;
                cnt.oh1 += !useL;
                a.f.out[q][jj] = useL ? lin[q] : cub[q];
            }
        }
        if (FUSED && a.D_next != nullptr) {
            float X[3] = {node_position(vn.lo[0], jx, vn.dx[0]), node_position(vn.lo[1], jy, vn.dx[1]),
                          node_position(vn.lo[2], jz, vn.dx[2])};
            float d[3];
            trajectory_cells<float, 3>(vn, X, d);
            a.D_next[jj] = make_float4(d[0], d[1], d[2], 0.f);
        }
    }
    unsigned smid;
    asm("mov.u32 %0, %%smid;" : "=r"(smid));
    flush_counters_warp(cnt, a.counters + (smid % SL_COUNTER_STRIPES));
}

// ---- the staged kernel: each block's field values in shared memory ----------------------------
// The blocked kernel's 16x4x4 blocks and element search, with the 4x4x4 stencil taps (128 of the
// ~144 values a target reads) taken from shared memory.  The box of the block's start elements
// floor(j - D_j), widened by one element for the refined start and the walk (which end within one
// element of it for smooth flows) and by the stencil, is the block's field window.  Its copy --
// cp.async.bulk.tensor.3d boxes (one per field plane, issued by thread 0 on one mbarrier, no
// multicast) when the window lies inside the grid, per-element copies with periodic indices by
// every thread, tracked by a second mbarrier, when it crosses the seam -- runs while every target
// does its refined start, walk and Newton inversion on the displacements (through L1, as the
// blocked kernel).  Each target then waits for the copy and sums its taps from shared memory (from
// global memory where its stencil leaves the window; the whole block when its window exceeds the
// capacity).  Plain remaps only: a fused step's launch, which also integrates the next
// trajectories, measured faster on the blocked kernel.  On the deformation flows a block's window
// holds ~8 nodes per target and field, against the 64 tap values per field a target reads.
// window capacity in nodes per field plane (x a multiple of 4 nodes: the box copies' 16-byte rule)
constexpr int HWX = 28, HWY = 12, HWZ = 12;
constexpr int HPLANE = HWX * HWY * HWZ;  // floats per field window (a multiple of 32: planes stay 128-byte aligned)
static_assert(BX == 16 && BY == 4 && BZ == 4 && NT3 == 256 && (HWX * HWY) % 32 == 16, "staged 3-D thread layout");
constexpr size_t s3_smem(int nf) { return (size_t)nf * HPLANE * 4 + 128; }  // + room to align

struct Win3 {
    int hlo[3];       // origin of the field window (unwrapped node indices)
    int hext[3];      // its extent in nodes
    unsigned hlim[3]; // a stencil starting at node c - 1 lies inside when c - 1 - hlo < hlim
    int mode;         // 0: not staged, 1: box copies, 2: per-element copies
};

struct Maps3 {
    CUtensorMap f[2];  // field planes: FP32, dims (n0, n1, n2), box (HWX, HWY, HWZ)
};

struct Staged3Args {
    Blocked3Args b;
    int use_tma;                   // the tensor maps are valid
    unsigned long long *timeouts;  // counter of waits that ran out
};

// the field window of the start-element box [mn, mx] (thread 0): the stencils c-1 .. c+2 of the
// elements mn - 1 .. mx + 1
__device__ __forceinline__ void window3(Win3 &w, const int mn[3], const int mx[3], const Geo3 &g, bool tma)
{
    const int n[3] = {g.n0, g.n1, g.n2}, HW[3] = {HWX, HWY, HWZ};
    bool fits = true, inside = true;
    long long h0[3], he[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        h0[a] = (long long)mn[a] - 2;
        if (a == 0) h0[a] &= ~3LL;  // box copies start on a 16-byte boundary
        he[a] = (long long)mx[a] + 3 - h0[a] + 1;
        fits = fits && mn[a] <= mx[a] && he[a] <= HW[a] && h0[a] >= -(long long)n[a] && h0[a] + he[a] <= 2LL * n[a];
        inside = inside && h0[a] >= 0 && h0[a] + he[a] <= n[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w.hlo[a] = fits ? (int)h0[a] : 0;
        w.hext[a] = fits ? (int)he[a] : 0;
        w.hlim[a] = fits ? (unsigned)(he[a] - 3) : 0u;
    }
    w.mode = !fits ? 0 : (tma && inside) ? 1 : 2;
}

// stencil taps from the field windows (the tap source of tap_sums): s at the stencil's first node
// in plane 0; every tap at a fixed offset from it
template <int NF>
struct StagedTaps3 {
    const float *s;
    struct Ptr {
        const float *a;
    };
    static constexpr int DB = NF > 1 ? HPLANE : 0;  // plane of the pair's second field
    __device__ __forceinline__ Ptr fields(int q) const { return {s + q * HPLANE}; }
    __device__ __forceinline__ Ptr row(const Ptr &p, int kz, int ky) const { return {p.a + (kz * HWY + ky) * HWX}; }
    __device__ __forceinline__ float2 tap(const Ptr &r, int kx) const { return make_float2(r.a[kx], r.a[kx + DB]); }
};

// tap sums of a target whose stencil leaves the field window (rare: out of line)
struct Sums2 {
    float c0, c1, l0, l1;
};
__device__ __noinline__ Sums2 taps_global2(const Geo3 g, const float *h0, const float *h1, int nfields, int c0, int c1,
                                           int c2, float x0, float x1, float x2)
{
    const int c[3] = {c0, c1, c2};
    const float xf[3] = {x0, x1, x2};
    float wc[3][4];
#pragma unroll
    for (int q = 0; q < 3; ++q) cubic_w(xf[q], wc[q]);
    Fields3 f;
    f.in[0] = h0;
    f.in[1] = h1;
    const GlobalTaps3 tp(g, f, nfields, c);
    float cub[2], lin[2];
    tap_sums<2>(tp, nfields, wc, xf, cub, lin);
    return {cub[0], cub[1], lin[0], lin[1]};
}

// Box copies (thread 0): arm bar with every box's bytes and issue one box per field plane.
template <int NF>
__device__ __forceinline__ void stage3_boxes(const Maps3 &maps, const Win3 &w, float *sH, unsigned long long *bar)
{
    mbar_arrive_tx(bar, (unsigned)(NF * HPLANE * 4));
#pragma unroll
    for (int q = 0; q < NF; ++q) tma_load_3d(sH + q * HPLANE, &maps.f[q], w.hlo[0], w.hlo[1], w.hlo[2], bar);
}

// Per-element copies (every thread): warp w copies rows w, w + 8, .. of the window (a row is at
// most 28 nodes, a lane per node); the thread's copies then arrive on bar as they complete.
template <int NF>
__device__ __forceinline__ void stage3_elements(const Blocked3Args &a, const Win3 &w, float *sH, unsigned long long *bar)
{
    const Geo3 &g = a.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool on = lane < w.hext[0];
    const unsigned gx = on ? (unsigned)wrap_near(w.hlo[0] + lane, g.n0) : 0u;
    const int rows = w.hext[1] * w.hext[2];
    for (int r = warp; r < rows; r += NT3 / 32) {
        const int zz = r / w.hext[1], yy = r - zz * w.hext[1];
        const unsigned gi =
            ((unsigned)wrap_near(w.hlo[2] + zz, g.n2) * (unsigned)g.n1 + (unsigned)wrap_near(w.hlo[1] + yy, g.n1)) *
                (unsigned)g.n0 + gx;
        if (on) {
#pragma unroll
            for (int q = 0; q < NF; ++q) cp_async<4>(sH + q * HPLANE + (zz * HWY + yy) * HWX + lane, a.f.in[q] + gi);
        }
    }
    mbar_track_cp_async_noinc(bar);
}

template <int NF>
__global__ void __launch_bounds__(NT3, 4)
    remap_staged3d_kernel(const __grid_constant__ Staged3Args A, const __grid_constant__ Maps3 maps)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // box copies want 128-byte aligned destinations: the launch adds 128 bytes of room
    float *const sH = reinterpret_cast<float *>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
    __shared__ unsigned long long bar[2];  // 0: the box copies' bytes, 1: every thread's per-element copies
    __shared__ int box[6];
    __shared__ Win3 W;
    const Blocked3Args &a = A.b;
    const Geo3 &g = a.g;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], NT3);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        box[0] = box[1] = box[2] = INT_MAX;
        box[3] = box[4] = box[5] = INT_MIN;
    }
    // a warp takes 16 x of one row in two consecutive planes: its halves' shared-memory reads lie
    // a plane of the window apart (HWX HWY = 16 mod 32 banks), so they fall in distinct banks
    const int t = (int)threadIdx.x;
    const int jx = blockIdx.x * BX + (t & 15);
    const int jy = blockIdx.y * BY + ((t >> 5) & 3);
    const int jz = blockIdx.z * BZ + ((t >> 7) << 1) + ((t >> 4) & 1);
    const bool valid = jx < g.n0 && jy < g.n1 && jz < g.n2;
    const long long jj = ((long long)jz * g.n1 + jy) * g.n0 + jx;
    const int j[3] = {jx, jy, jz};
    int c0[3] = {jx, jy, jz};
    float s0[3] = {0.f, 0.f, 0.f};
    if (valid) start_point3(j, __ldg(a.D + jj), s0, c0);
    __syncthreads();  // the barriers and the box are initialised
    {
        int mn[3], mx[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            mn[q] = __reduce_min_sync(0xffffffffu, valid ? c0[q] : INT_MAX);
            mx[q] = __reduce_max_sync(0xffffffffu, valid ? c0[q] : INT_MIN);
        }
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                atomicMin(&box[q], mn[q]);
                atomicMax(&box[3 + q], mx[q]);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int mn[3] = {box[0], box[1], box[2]}, mx[3] = {box[3], box[4], box[5]};
        window3(W, mn, mx, g, A.use_tma != 0);
        if (W.mode == 1) stage3_boxes<NF>(maps, W, sH, &bar[0]);
    }
    __syncthreads();
    const int mode = W.mode;
    if (mode == 2) stage3_elements<NF>(a, W, sH, &bar[1]);
    LocalCounters cnt;
    cnt.clear();
    if (threadIdx.x == 0 && mode == 0) cnt.fallback += 1;
    // the element search while the window is copied (the blocked kernel's arithmetic)
    const GlobalD3 src = {g, a.D};
    int c[3] = {c0[0], c0[1], c0[2]};
    int st = ST_OK;
    float xf[3] = {0.f, 0.f, 0.f};
    if (valid) {
        refined_start3(src, j, s0, c0, c);
        int hops = 0, iters = 0;
        bool degen = false;
        st = walk3<float>(src, a.max_iter, a.walk_max, j, c, xf, hops, iters, &degen);
        if (st != ST_OK || degen) {
            const Resolve3 r = resolve3_f64(a.D, g.n0, g.n1, g.n2, a.max_iter, a.walk_max, j[0], j[1], j[2], st, c[0],
                                            c[1], c[2], c0[0], c0[1], c0[2]);
            st = r.st;
            c[0] = r.c0;
            c[1] = r.c1;
            c[2] = r.c2;
            xf[0] = r.x0;
            xf[1] = r.x1;
            xf[2] = r.x2;
            hops += r.hops;
            iters += r.iters;
            cnt.f64 += 1;
        }
        cnt.targets += 1;
        cnt.hops += hops;
        cnt.hops_max = max(cnt.hops_max, (unsigned)hops);
        cnt.iters += iters;
        cnt.iters_max = max(cnt.iters_max, (unsigned)iters);
    }
    // every thread waits for the copy (none may leave the block with a copy in flight); a wait
    // that runs out leaves the thread on global reads
    bool late = false;
    if (mode != 0) late = !mbar_wait(&bar[mode == 1 ? 0 : 1], 0u);
    if (late) atomicAdd(A.timeouts, 1ull);
    if (valid) {
        if (st != ST_OK) {
            cnt.fl += st == ST_LOCATE;
            cnt.fn += st == ST_NEWTON;
            cnt.ff += st == ST_FOLD;
#pragma unroll
            for (int q = 0; q < NF; ++q) a.f.out[q][jj] = __ldg(a.f.in[q] + jj);
        } else {
            const unsigned bits = a.max_order >= 1 ? (unsigned)__ldg(a.box + lin3(g, c[0], c[1], c[2])) : 0xffu;
            const unsigned r0 = (unsigned)(c[0] - 1 - W.hlo[0]), r1 = (unsigned)(c[1] - 1 - W.hlo[1]),
                           r2 = (unsigned)(c[2] - 1 - W.hlo[2]);
            float cub[2], lin[2];
            if (!late && r0 < W.hlim[0] && r1 < W.hlim[1] && r2 < W.hlim[2]) {
                float wc[3][4];
#pragma unroll
                for (int q = 0; q < 3; ++q) cubic_w(xf[q], wc[q]);
                const StagedTaps3<NF> tp = {sH + (r2 * HWY + r1) * HWX + r0};
                tap_sums<2>(tp, NF, wc, xf, cub, lin);
            } else {
                const Sums2 r = taps_global2(g, a.f.in[0], NF > 1 ? a.f.in[1] : a.f.in[0], NF, c[0], c[1], c[2], xf[0],
                                             xf[1], xf[2]);
                cub[0] = r.c0;
                cub[1] = r.c1;
                lin[0] = r.l0;
                lin[1] = r.l1;
            }
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                const bool useL = ((bits >> q) & 1u) != 0u;
                cnt.oh0 += useL;
                cnt.oh1 += !useL;
                a.f.out[q][jj] = useL ? lin[q] : cub[q];
            }
        }
    }
    unsigned smid;
    asm("mov.u32 %0, %%smid;" : "=r"(smid));
    flush_counters_warp(cnt, a.counters + (smid % SL_COUNTER_STRIPES));
}

}  // namespace

// box flags of a 3-D FP32 grid: flags ORed along x into `flags`, then over y and z into `tmp`
cudaError_t launch_box_flags3d(const sl_grid *g, const void *const *in, uint8_t *flags, uint8_t *tmp, cudaStream_t s)
{
    Geo3 geo = {(int)g->n[0], (int)g->n[1], (int)g->n[2]};
    Fields3 f;
    memset(&f, 0, sizeof(f));
    for (int q = 0; q < g->nfields; ++q) f.in[q] = (const float *)in[q];
    const dim3 block(32, 8);
    const unsigned gy = (unsigned)std::min<long long>((g->n[1] + 7) / 8, 65535);
    const unsigned gz = (unsigned)std::min<long long>(g->n[2], 65535);
    const int zchunk = (int)std::max<long long>(16, (g->n[2] + 65534) / 65535);
    const dim3 gridf((unsigned)((g->n[0] + FX - 1) / FX), gy, (unsigned)((g->n[2] + zchunk - 1) / zchunk));
    const float thr = (float)g->desc.limiter_threshold;
    if (g->nfields <= 2)
        flags_x3d_kernel<2><<<gridf, block, 0, s>>>(geo, g->nfields, thr, f, flags, zchunk);
    else if (g->nfields <= 4)
        flags_x3d_kernel<4><<<gridf, block, 0, s>>>(geo, g->nfields, thr, f, flags, zchunk);
    else
        flags_x3d_kernel<8><<<gridf, block, 0, s>>>(geo, g->nfields, thr, f, flags, zchunk);
    // the byte buffers start 256-byte aligned; rows of a multiple of 4 nodes keep 32-bit alignment
    if (g->n[0] % 4 == 0) {
        const dim3 gridb((unsigned)((g->n[0] / 4 + 31) / 32), gy, gz);
        box_yz3d_kernel<4><<<gridb, block, 0, s>>>(geo, flags, tmp);
    } else {
        const dim3 gridb((unsigned)((g->n[0] + 31) / 32), gy, gz);
        box_yz3d_kernel<1><<<gridb, block, 0, s>>>(geo, flags, tmp);
    }
    return cudaGetLastError();
}

template <bool N64>
static void launch_b3(int nfm, bool fused, dim3 grid, cudaStream_t s, const Blocked3Args &a, const VelArgs<float> &vn)
{
    if (fused) {
        if (nfm == 2) remap_blocked3d_kernel<2, true, N64><<<grid, NT3, 0, s>>>(a, vn);
        else if (nfm == 4) remap_blocked3d_kernel<4, true, N64><<<grid, NT3, 0, s>>>(a, vn);
        else remap_blocked3d_kernel<8, true, N64><<<grid, NT3, 0, s>>>(a, vn);
    } else {
        if (nfm == 2) remap_blocked3d_kernel<2, false, N64><<<grid, NT3, 0, s>>>(a, vn);
        else if (nfm == 4) remap_blocked3d_kernel<4, false, N64><<<grid, NT3, 0, s>>>(a, vn);
        else remap_blocked3d_kernel<8, false, N64><<<grid, NT3, 0, s>>>(a, vn);
    }
}

// The staged kernel serves plain remaps of FP32 grids with up to 2 fields whose targets invert in
// FP32 (FP64 re-solves only for failed or degenerate ones), unless tile configuration 1 asks for
// the L1 path.
static bool staged3d_supported(const sl_grid *g)
{
    return g->nfields <= 2 && g->desc.newton_mode != SL_NEWTON_F64 && g->desc.tile_config != 1;
}

template <int NF>
static cudaError_t launch_s3(const sl_grid *g, const Staged3Args &A, const Maps3 &maps, dim3 grid, cudaStream_t s)
{
    static bool configured[64] = {};
    if (!configured[g->device & 63]) {
        cudaError_t e = cudaFuncSetAttribute(remap_staged3d_kernel<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)s3_smem(NF));
        if (e != cudaSuccess) return e;
        configured[g->device & 63] = true;
    }
    remap_staged3d_kernel<NF><<<grid, NT3, s3_smem(NF), s>>>(A, maps);
    return cudaGetLastError();
}

static cudaError_t launch_staged3d(const sl_grid *g, const Blocked3Args &a, dim3 grid, cudaStream_t s)
{
    Staged3Args A;
    memset(&A, 0, sizeof(A));
    A.b = a;
    A.timeouts = &g->counters->timeouts;
    Maps3 maps;
    memset(&maps, 0, sizeof(maps));
    const unsigned long long n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    const unsigned long long dims[3] = {n0, n1, n2}, strides[2] = {4 * n0, 4 * n0 * n1};
    const unsigned boxd[3] = {HWX, HWY, HWZ};
    // (boxes no larger than the grid: smaller grids copy their windows element by element)
    bool tma = n0 >= HWX && n1 >= HWY && n2 >= HWZ;
    for (int q = 0; q < g->nfields; ++q) tma = tma && encode_tensor_f32(&maps.f[q], a.f.in[q], 3, dims, strides, boxd);
    A.use_tma = tma ? 1 : 0;
    return g->nfields == 1 ? launch_s3<1>(g, A, maps, grid, s) : launch_s3<2>(g, A, maps, grid, s);
}

cudaError_t launch_blocked3d(const sl_grid *g, const void *D, void *D_next, const uint8_t *box, double t_next,
                             double dt, bool fused, const void *const *in, void *const *out, cudaStream_t s)
{
    Blocked3Args a;
    memset(&a, 0, sizeof(a));
    a.g = {(int)g->n[0], (int)g->n[1], (int)g->n[2]};
    a.nfields = g->nfields;
    a.max_order = g->desc.max_order;
    a.max_iter = g->desc.newton_max_iter;
    a.walk_max = g->desc.walk_max;
    a.D = (const float4 *)D;
    a.D_next = (float4 *)D_next;
    a.box = box;
    for (int q = 0; q < g->nfields; ++q) {
        a.f.in[q] = (const float *)in[q];
        a.f.out[q] = (float *)out[q];
    }
    a.counters = g->stripes;  // per-SM copies: each warp adds its counters into its SM's copy
    dim3 grid((unsigned)((g->n[0] + BX - 1) / BX), (unsigned)((g->n[1] + BY - 1) / BY),
              (unsigned)((g->n[2] + BZ - 1) / BZ));
    VelArgs<float> vn;
    memset(&vn, 0, sizeof(vn));
    if (fused) vn = make_vel_args<float>(g, t_next, dt);
    // the staged kernel where it is the faster one: plain remaps (a fused step, whose launch also
    // integrates the next trajectories, measured faster on the blocked kernel)
    if (!fused && staged3d_supported(g)) return launch_staged3d(g, a, grid, s);
    const int nfm = g->nfields <= 2 ? 2 : g->nfields <= 4 ? 4 : 8;
    if (g->desc.newton_mode == SL_NEWTON_F64)
        launch_b3<true>(nfm, fused, grid, s, a, vn);
    else
        launch_b3<false>(nfm, fused, grid, s, a, vn);
    return cudaGetLastError();
}
