// sl_tile2d.cuh -- the per-tile body of the 2-D FP32 production kernels (single-grid and batched)
// of the FSL step (arXiv:1410.2817).
//
// One CTA owns a TX x TY tile of target (reference) nodes.  Its targets' departure points lie
// near j - D_j, so the CTA first takes the bounding box of the start elements floor(j - D_j),
// widens it by the walk slack, the cubic stencil (Sec. 2.1: nodes c-1 .. c+2) and the limiter's
// neighbours (Sec. 2.3), and stages that window -- displacements and field values -- in shared
// memory with asynchronous copies.  The jump flags and their OR over every element's 4x4 stencil
// are computed once per window node in shared memory, so each target's element search (Sec. 2.2),
// order choice (Sec. 2.3) and tensor Z-spline sum (eq. multiZ) read shared memory only.  A target
// whose walk leaves the window, or a tile whose window does not fit, falls back to global gathers.
//
// Precision: FP32 data and FP32 Newton; a target whose FP32 inversion failed, or whose element is
// close to degenerate, is re-solved in FP64.  Up to four fields are interleaved per window node
// (float4), so one 128-bit shared load serves every field of a stencil tap.
//
// The fused variant also integrates the next step's trajectories (eq. vel) for the tile's own
// nodes: the velocity is given, so D(t + dt) does not depend on the fields being remapped.
#pragma once

#include <algorithm>
#include <limits.h>
#include <math.h>
#include <string.h>

#include "sl_async.cuh"
#include "sl_internal.h"

namespace {

// Tile configuration: TX x TY targets per CTA of NT threads (TX a multiple of 32: one warp per
// row segment), window capacity (TX + 2 HALO) x (TY + 2 HALO) nodes in shared memory.
template <int TX_, int TY_, int NT_, int HALO_, int MINB_ = 3>
struct TileCfg {
    static constexpr int TX = TX_, TY = TY_, NT = NT_, HALO = HALO_;
    static constexpr int MINB = MINB_;     // CTAs per SM the register budget is compiled for
    static constexpr int ROWS = NT / TX;   // thread rows
    static constexpr int TPT = TY / ROWS;  // targets per thread
    static constexpr int WMAX = (TX + 2 * HALO) * (TY + 2 * HALO);
    static_assert(TX % 32 == 0 && NT % TX == 0 && TY % ROWS == 0, "bad tile configuration");
};
typedef TileCfg<32, 32, 256, 8> CfgA;  // default
typedef TileCfg<32, 16, 256, 8> CfgB;
typedef TileCfg<64, 16, 256, 8> CfgC;
typedef TileCfg<32, 16, 256, 8, 4> CfgD;  // 4 CTAs per SM: at most 64 registers per thread
typedef TileCfg<32, 32, 512, 8, 1> CfgP;  // pipelined, one CTA of 16 warps per SM

constexpr int WALK_SLACK = 1;          // elements the walk may step beyond the start-cell box

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
    DevCounters *stripes;  // the grid's per-SM copies of the counters (single grids; null in batches)
    // carried velocity (Sec. 3.2): D_next = dt u / dx from the remapped fields vf[0], vf[1]
    int carried, vf[2];
    float csc[2];
};

__device__ __forceinline__ long long gidx(int x, int y, int n0, int n1)
{
    return (long long)wrap_idx(y, n1) * n0 + wrap_idx(x, n0);
}

// row of flat index q in a region `width` wide: (q + 0.5) / width in FP32 is exact enough to
// floor correctly for q, width < 2^11 (the fractional part stays >= 0.5 / width)
__device__ __forceinline__ int row_of(int q, float inv_width) { return __float2int_rz(((float)q + 0.5f) * inv_width); }

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
__device__ __forceinline__ float2 disp(const TileArgs &a, const Win &w, const float2 *sD, int x, int y)
{
    if (w.has(x, y)) return sD[w.at(x, y)];
    return __ldg(reinterpret_cast<const float2 *>(a.D) + gidx(x, y, a.n0, a.n1));
}

// Sec. 2.2 element search from element (cx, cy) with Newton in precision TN (window wx = 0 when
// nothing is staged, so every vertex then comes from global memory).
template <typename TN>
__device__ __forceinline__ int walk2(const TileArgs &a, const Win &w, const float2 *sD, int jx, int jy, int &cx,
                                     int &cy, TN xi[3], int &hops, int &iters, bool &degen)
{
    const TN tol = sizeof(TN) == 8 ? TN(1e-14) : TN(SL_NEWTON_TOL_F32);
    const TN slack = sizeof(TN) == 8 ? TN(1e-12) : TN(SL_SLACK_F32);
    CycleCheck cyc;
    cyc.start(cx, cy, 0);
    for (int hop = 0; hop < a.walk_max; ++hop) {
        TN P[8][3];
        float2 d4[4];
        if (w.has(cx, cy) && w.has(cx + 1, cy + 1)) {
            const int i0 = w.at(cx, cy);
            d4[0] = sD[i0];
            d4[1] = sD[i0 + 1];
            d4[2] = sD[i0 + w.wx];
            d4[3] = sD[i0 + w.wx + 1];
        } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) d4[v] = disp(a, w, sD, cx + (v & 1), cy + (v >> 1));
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            P[v][0] = TN(cx + (v & 1) - jx) + TN(d4[v].x);
            P[v][1] = TN(cy + (v >> 1) - jy) + TN(d4[v].y);
        }
        int it = 0;
        const int st = newton_solve2<TN>(P, a.max_iter, tol, xi, &it, &degen);
        hops += 1;
        iters += it;
        if (!(finite_t(xi[0]) && finite_t(xi[1]))) return st == ST_OK ? ST_NEWTON : st;
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
        if (cyc.step(cx, cy, 0)) return ST_LOCATE;
    }
    return ST_LOCATE;
}

// Sec. 2.2 element search entirely in the staged window, FP32 Newton.  Returns false when an
// element leaves the window, Newton does not converge or the element is nearly degenerate: the
// target is then solved again on the general path (slow_target), which repeats this walk with
// global reads and re-solves in FP64.  The arithmetic is that of walk2<float>, so a target that
// succeeds here gets the same element and coordinates as on the general path.
__device__ __forceinline__ bool walk_window(const Win &w, const float2 *sD, int walk_max, int max_iter, int jx, int jy,
                                            int &ex, int &ey, float &xi0, float &xi1, int &hops, int &iters)
{
    const float slack = SL_SLACK_F32;
    CycleCheck cyc;
    cyc.start(ex, ey, 0);
    for (int hop = 0; hop < walk_max; ++hop) {
        if (!(w.has(ex, ey) && w.has(ex + 1, ey + 1))) return false;
        const int i0 = w.at(ex, ey);
        const float2 d0 = sD[i0], d1 = sD[i0 + 1], d2 = sD[i0 + w.wx], d3 = sD[i0 + w.wx + 1];
        const float rx0 = (float)(ex - jx), rx1 = (float)(ex + 1 - jx);
        const float ry0 = (float)(ey - jy), ry1 = (float)(ey + 1 - jy);
        float P[8][3];
        P[0][0] = rx0 + d0.x;
        P[0][1] = ry0 + d0.y;
        P[1][0] = rx1 + d1.x;
        P[1][1] = ry0 + d1.y;
        P[2][0] = rx0 + d2.x;
        P[2][1] = ry1 + d2.y;
        P[3][0] = rx1 + d3.x;
        P[3][1] = ry1 + d3.y;
        float xf[3];
        int it = 0;
        bool degen = false;
        const int st = newton_solve2<float>(P, max_iter, SL_NEWTON_TOL_F32, xf, &it, &degen);
        hops += 1;
        iters += it;
        if (st != ST_OK || degen) return false;  // converged implies finite coordinates
        const bool lo0 = xf[0] < -slack, hi0 = xf[0] > 1.f + slack;
        const bool lo1 = xf[1] < -slack, hi1 = xf[1] > 1.f + slack;
        if (!(lo0 || hi0 || lo1 || hi1)) {
            xi0 = xf[0];
            xi1 = xf[1];
            return true;
        }
        ex += lo0 ? -1 : (hi0 ? 1 : 0);
        ey += lo1 ? -1 : (hi1 ? 1 : 0);
        if (cyc.step(ex, ey, 0)) return false;
    }
    return false;
}

// Sec. 2.3 flags of one node from global memory (fallback path)
__device__ __forceinline__ unsigned node_flags_global(const TileArgs &a, int x, int y)
{
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

// order flags of element (ex, ey) from global memory: OR over its 4x4 stencil
__device__ __noinline__ unsigned box_flags_global(const TileArgs &a, int ex, int ey)
{
    unsigned bits = 0;
    for (int q = 0; q < 16; ++q) bits |= node_flags_global(a, ex - 1 + (q & 3), ey - 1 + (q >> 2));
    return bits;
}

// Z~1 weights of taps c-1 .. c+2 at local coordinate x (Appendix)
__device__ __forceinline__ void cubic_weights(float x, float w[4])
{
    const float y = 1.f - x, x2 = x * x, y2 = y * y;
    w[0] = -0.5f * x * y2;
    w[1] = fmaf(x2, fmaf(1.5f, x, -2.5f), 1.f);
    w[2] = fmaf(y2, fmaf(1.5f, y, -2.5f), 1.f);
    w[3] = -0.5f * x2 * y;
}

// eq. (multiZ) from global memory for a target whose stencil leaves the window
__device__ __noinline__ void interp_global(const TileArgs &a, long long jj, int ex, int ey, float xi0, float xi1,
                                           unsigned lin_mask)
{
    float wc[2][4];
    cubic_weights(xi0, wc[0]);
    cubic_weights(xi1, wc[1]);
    for (int f = 0; f < a.nfields; ++f) {
        const float *h = a.in[f];
        float cub = 0.f, lin = 0.f;
        for (int ky = 0; ky < 4; ++ky) {
            float r = 0.f;
            for (int kx = 0; kx < 4; ++kx) r = fmaf(wc[0][kx], __ldg(h + gidx(ex - 1 + kx, ey - 1 + ky, a.n0, a.n1)), r);
            cub = fmaf(wc[1][ky], r, cub);
        }
        for (int ky = 0; ky < 2; ++ky) {
            const float r = fmaf(xi0, __ldg(h + gidx(ex + 1, ey + ky, a.n0, a.n1)),
                                 (1.f - xi0) * __ldg(h + gidx(ex, ey + ky, a.n0, a.n1)));
            lin = fmaf(ky ? xi1 : 1.f - xi1, r, lin);
        }
        a.out[f][jj] = ((lin_mask >> f) & 1u) ? lin : cub;
    }
}

// jump bits (Sec. 2.3) of the first NC fields interleaved in a float4
template <int NC>
__device__ __forceinline__ unsigned jump4(const float4 &m, const float4 &c, const float4 &p, float thr)
{
    unsigned b = 0;
    b |= jump_test<float>(m.x, c.x, p.x, thr) ? 1u : 0u;
    if (NC > 1) b |= jump_test<float>(m.y, c.y, p.y, thr) ? 2u : 0u;
    if (NC > 2) b |= jump_test<float>(m.z, c.z, p.z, thr) ? 4u : 0u;
    if (NC > 3) b |= jump_test<float>(m.w, c.w, p.w, thr) ? 8u : 0u;
    return b;
}

__host__ __device__ constexpr int groups(int nf) { return (nf + 3) / 4; }
__host__ __device__ constexpr int in_group(int nf, int g) { return nf - 4 * g < 4 ? nf - 4 * g : 4; }

// eq. (multiZ) for the fields of group G (4 per float4) from the 4x4 taps starting at h: the cubic
// (Z~1) sum and the bilinear (Z~0) sum over the element's own 4 vertices; fields whose lin_mask bit
// is set take the bilinear value.  The sums run on field pairs with packed FP32x2 FMAs (each lane
// rounds as fmaf does); the pair holding only padding is skipped.
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

template <int NF, int G>
__device__ __forceinline__ void store_group(const TileArgs &a, long long jj, const float4 *h, int stride,
                                            const float wc[2][4], float xi0, float xi1, unsigned lin_mask)
{
    constexpr int NC = in_group(NF, G);
    constexpr bool HI = NC > 2;
    const float2 w0 = bcast2(wc[0][0]), w1 = bcast2(wc[0][1]), w2 = bcast2(wc[0][2]), w3 = bcast2(wc[0][3]);
    const float2 u0 = bcast2(1.f - xi0), u1 = bcast2(xi0);
    const float2 z = make_float2(0.f, 0.f);
    float2 cl = z, ch = z, ll = z, lh = z;
#pragma unroll
    for (int ky = 0; ky < 4; ++ky) {
        const float4 t0 = h[0], t1 = h[1], t2 = h[2], t3 = h[3];
        const float2 wy = bcast2(wc[1][ky]);
        float2 r = __fmul2_rn(w0, lo2(t0));
        r = __ffma2_rn(w1, lo2(t1), r);
        r = __ffma2_rn(w2, lo2(t2), r);
        r = __ffma2_rn(w3, lo2(t3), r);
        cl = __ffma2_rn(wy, r, cl);
        if (HI) {
            float2 q = __fmul2_rn(w0, hi2(t0));
            q = __ffma2_rn(w1, hi2(t1), q);
            q = __ffma2_rn(w2, hi2(t2), q);
            q = __ffma2_rn(w3, hi2(t3), q);
            ch = __ffma2_rn(wy, q, ch);
        }
        if (ky == 1 || ky == 2) {
            const float2 v = bcast2(ky == 1 ? 1.f - xi1 : xi1);
            ll = __ffma2_rn(v, __ffma2_rn(u1, lo2(t2), __fmul2_rn(u0, lo2(t1))), ll);
            if (HI) lh = __ffma2_rn(v, __ffma2_rn(u1, hi2(t2), __fmul2_rn(u0, hi2(t1))), lh);
        }
        h += stride;
    }
    const float cub[4] = {cl.x, cl.y, ch.x, ch.y}, lin[4] = {ll.x, ll.y, lh.x, lh.y};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int f = 4 * G + c;
        a.out[f][jj] = ((lin_mask >> f) & 1u) ? lin[c] : cub[c];
    }
}

// Words of one field's bit plane: rows x ceil(wx / 32) <= (WMAX + 31 WMAX / 8) / 32, because every
// staged window is at least 8 nodes wide and high.
__host__ __device__ constexpr int mask_words(int wmax) { return (wmax + 31 * (wmax / 8)) / 32 + 1; }

// Shared memory of one tile: displacements, fields (4 per float4), per field two bit planes of
// ceil(wx / 32) words per window row -- M, the jump flags of the interior nodes, and B, bit x of row
// y set when a flag lies among nodes x-1 .. x+2 of rows y-1 .. y+2 (element (x, y)'s stencil) --
// and the start points j - D_j of the tile's targets.
template <class Cfg, int NF>
struct TileSmem {
    static constexpr int WMAX = Cfg::WMAX, MW = mask_words(WMAX);
    float2 *D;
    float4 *H;
    unsigned *M, *B;
    float2 *S;
    __device__ __forceinline__ explicit TileSmem(unsigned char *base)
    {
        D = reinterpret_cast<float2 *>(base);
        H = reinterpret_cast<float4 *>(D + WMAX);
        S = reinterpret_cast<float2 *>(H + groups(NF) * WMAX);
        M = reinterpret_cast<unsigned *>(S + Cfg::TX * Cfg::TY);
        B = M + NF * MW;
    }
};

// Start element of target (jx, jy): one fixed-point step s <- j - D(s) from s0 = j - D_j, with D(s0)
// interpolated bilinearly in the staged window (the walk still decides); floor(s0) when not staged.
__device__ __forceinline__ void refined_start(const Win &w, const float2 *sD, bool staged, int jx, int jy, float2 s0,
                                              int &ex, int &ey)
{
    ex = (int)floorf(s0.x);
    ey = (int)floorf(s0.y);
    if (!staged) return;
    const int i0 = w.at(ex, ey);
    const float fx = s0.x - (float)ex, fy = s0.y - (float)ey;
    const float2 d00 = sD[i0], d10 = sD[i0 + 1], d01 = sD[i0 + w.wx], d11 = sD[i0 + w.wx + 1];
    const float bx = fmaf(fx, d10.x - d00.x, d00.x), by = fmaf(fx, d10.y - d00.y, d00.y);
    const float dx = fmaf(fy, fmaf(fx, d11.x - d01.x, d01.x) - bx, bx);
    const float dy = fmaf(fy, fmaf(fx, d11.y - d01.y, d01.y) - by, by);
    const float rx = (float)jx - dx, ry = (float)jy - dy;
    if (finite_t(rx) && finite_t(ry) && fabsf(rx - s0.x) < 4.f && fabsf(ry - s0.y) < 4.f) {
        ex = (int)floorf(rx);
        ey = (int)floorf(ry);
    }
}

// Result of one target on the general path (for the counters).
struct TargetOut {
    int st, hops, iters, f64, nlin;
};

// The general path of one target (rare: out of line so that the fast path carries none of its
// code or registers): the walk of walk2 from the refined start with global reads where the window
// ends, the FP64 re-solve of a failed or nearly degenerate FP32 inversion (from the first start
// element when the FP32 walk got lost or folded), then order and sum from shared memory when the
// element's stencil is staged and from global memory otherwise.  A target that still fails keeps
// its old values (the fail policy is applied by the host).
template <int NF>
__device__ __noinline__ TargetOut slow_target(const TileArgs &a, const Win w, const float2 *sD, const float4 *sH,
                                              int gstride, const unsigned *sB, bool limit, long long jj, int jx,
                                              int jy, int ex, int ey, int c0x, int c0y)
{
    TargetOut r = {ST_OK, 0, 0, 0, 0};
    float xf[3] = {0.f, 0.f, 0.f};
    bool degen = false;
    int st = walk2<float>(a, w, sD, jx, jy, ex, ey, xf, r.hops, r.iters, degen);
    float xi0 = xf[0], xi1 = xf[1];
    if (st != ST_OK || degen) {
        if (st == ST_LOCATE || st == ST_FOLD) {
            ex = c0x;
            ey = c0y;
        }
        double xd[3] = {0.0, 0.0, 0.0};
        bool dg = false;
        st = walk2<double>(a, w, sD, jx, jy, ex, ey, xd, r.hops, r.iters, dg);
        xi0 = (float)xd[0];
        xi1 = (float)xd[1];
        r.f64 = 1;
    }
    r.st = st;
    if (st != ST_OK) {
#pragma unroll
        for (int f = 0; f < NF; ++f) a.out[f][jj] = __ldg(a.in[f] + jj);
        return r;
    }
    const int rx = ex - w.lox, ry = ey - w.loy;
    const bool fast = rx >= 2 && rx <= w.wx - 4 && ry >= 2 && ry <= w.wy - 4;  // false when not staged
    unsigned lin_mask = a.max_order == 0 ? 0xffu : 0u;
    if (limit) {
        if (fast) {
            const int nwx = (w.wx + 31) >> 5;
            const unsigned *b = sB + ry * nwx + (rx >> 5);
            lin_mask = 0u;
#pragma unroll
            for (int f = 0; f < NF; ++f) lin_mask |= ((b[f * w.wy * nwx] >> (rx & 31)) & 1u) << f;
        } else {
            lin_mask = box_flags_global(a, ex, ey);
        }
    }
    r.nlin = __popc(lin_mask & ((1u << NF) - 1u));
    if (fast) {
        float wc[2][4];
        cubic_weights(xi0, wc[0]);
        cubic_weights(xi1, wc[1]);
        const int o = (ry - 1) * w.wx + (rx - 1);
        store_group<NF, 0>(a, jj, sH + o, w.wx, wc, xi0, xi1, lin_mask);
        if constexpr (groups(NF) > 1) store_group<NF, 1>(a, jj, sH + gstride + o, w.wx, wc, xi0, xi1, lin_mask);
    } else {
        interp_global(a, jj, ex, ey, xi0, xi1, lin_mask);
    }
    return r;
}

// Start point j - D_j of a target, clamped so that garbage displacements cannot overflow the walk.
__device__ __forceinline__ float2 start_point(int jx, int jy, float2 d)
{
    const float ux = fminf(fmaxf((float)jx - d.x, (float)jx - 65536.f), (float)jx + 65536.f);
    const float uy = fminf(fmaxf((float)jy - d.y, (float)jy - 65536.f), (float)jy + 65536.f);
    return make_float2(finite_t(ux) ? ux : (float)jx, finite_t(uy) ? uy : (float)jy);
}

// Window of a tile from the box [bx0, bx1] x [by0, by1] of its start elements: widened by the walk
// slack, the cubic stencil (c-1 .. c+2) and the limiter's neighbours (one more node each side).
// A window is staged when it fits WMAX nodes and lies within one period of the grid on each side
// (so that its nodes wrap with wrap_near); otherwise the tile runs on global memory.
template <int WMAX>
__device__ __forceinline__ Win window_of(int bx0, int by0, int bx1, int by1, int n0, int n1, bool &staged)
{
    const long long wxl = (long long)bx1 - bx0 + 2 * WALK_SLACK + 6;
    const long long wyl = (long long)by1 - by0 + 2 * WALK_SLACK + 6;
    const long long olx = (long long)bx0 - WALK_SLACK - 2, oly = (long long)by0 - WALK_SLACK - 2;
    staged = wxl > 0 && wyl > 0 && wxl <= WMAX && wyl <= WMAX && wxl * wyl <= WMAX && olx >= -n0 && oly >= -n1 &&
             olx + wxl <= 2LL * n0 && oly + wyl <= 2LL * n1;
    Win w;
    w.lox = staged ? (int)olx : 0;
    w.loy = staged ? (int)oly : 0;
    w.wx = staged ? (int)wxl : 0;
    w.wy = staged ? (int)wyl : 0;
    return w;
}

// Box of the CTA's start elements: warp reductions, then shared atomics into box (reset by the
// caller beforehand); returns after a barrier with the box read back.
__device__ __forceinline__ void reduce_box(int mnx, int mny, int mxx, int mxy, int *box, int &bx0, int &by0, int &bx1,
                                           int &by1)
{
    mnx = __reduce_min_sync(0xffffffffu, mnx);
    mny = __reduce_min_sync(0xffffffffu, mny);
    mxx = __reduce_max_sync(0xffffffffu, mxx);
    mxy = __reduce_max_sync(0xffffffffu, mxy);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&box[0], mnx);
        atomicMin(&box[1], mny);
        atomicMax(&box[2], mxx);
        atomicMax(&box[3], mxy);
    }
    __syncthreads();
    bx0 = box[0];
    by0 = box[1];
    bx1 = box[2];
    by1 = box[3];
}

// Issue the asynchronous copies of a staged window: displacements to sD, fields (4 per float4,
// group stride WMAX) to sH.  The caller waits for them (cp_async_wait_all + barrier).
template <class Cfg, int NF>
__device__ __forceinline__ void stage_window(const TileArgs &a, const Win &w, float2 *sD, float4 *sH)
{
    const int nwin = w.wx * w.wy;
    const float inv_wx = nwin > 0 ? 1.f / (float)w.wx : 0.f;
    for (int q = threadIdx.x; q < nwin; q += Cfg::NT) {
        const int wy = row_of(q, inv_wx), wx = q - wy * w.wx;
        const long long gi = (long long)wrap_near(w.loy + wy, a.n1) * a.n0 + wrap_near(w.lox + wx, a.n0);
        cp_async<8>(sD + q, reinterpret_cast<const float2 *>(a.D) + gi);
#pragma unroll
        for (int f = 0; f < NF; ++f)
            cp_async<4>(reinterpret_cast<float *>(sH + (f >> 2) * Cfg::WMAX + q) + (f & 3), a.in[f] + gi);
    }
}

// Clear the flag plane of a window before its flags are set.
template <class Cfg, int NF>
__device__ __forceinline__ void clear_flags(const TileArgs &a, const Win &w, unsigned *M)
{
    if (a.max_order >= 1 && a.thr >= 0.f) {
        const int nm = NF * w.wy * ((w.wx + 31) >> 5);
        for (int q = threadIdx.x; q < nm; q += Cfg::NT) M[q] = 0u;
    }
}

// Sec. 2.3: jump flags of the window's interior nodes (rows and columns 1 .. w-2) into the bit
// plane M (one bit per node and field, `plane` words per field, `nwx` words per row), set with a
// shared-memory atomic: flagged nodes are few.  M must be clear; the caller synchronises after.
template <class Cfg, int NF>
__device__ __forceinline__ void flag_window(const TileArgs &a, const Win &w, const float4 *sH, unsigned *sM, int nwx,
                                            int plane)
{
    constexpr int NT = Cfg::NT, WMAX = Cfg::WMAX;
    constexpr int NG = groups(NF);
    const int iw = w.wx - 2, ni = iw * (w.wy - 2);
    const float inv_iw = 1.f / (float)max(iw, 1);
    for (int q = threadIdx.x; q < ni; q += NT) {
        const int r = row_of(q, inv_iw), y = r + 1, x = q - r * iw + 1;
        const int idx = y * w.wx + x;
        unsigned bits = 0;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const float4 *h = sH + g * WMAX;
            const float4 c = h[idx];
            if (in_group(NF, g) == 4)
                bits |= (jump4<4>(h[idx - 1], c, h[idx + 1], a.thr) | jump4<4>(h[idx - w.wx], c, h[idx + w.wx], a.thr))
                        << (4 * g);
            else if (in_group(NF, g) == 3)
                bits |= (jump4<3>(h[idx - 1], c, h[idx + 1], a.thr) | jump4<3>(h[idx - w.wx], c, h[idx + w.wx], a.thr))
                        << (4 * g);
            else if (in_group(NF, g) == 2)
                bits |= (jump4<2>(h[idx - 1], c, h[idx + 1], a.thr) | jump4<2>(h[idx - w.wx], c, h[idx + w.wx], a.thr))
                        << (4 * g);
            else
                bits |= (jump4<1>(h[idx - 1], c, h[idx + 1], a.thr) | jump4<1>(h[idx - w.wx], c, h[idx + w.wx], a.thr))
                        << (4 * g);
        }
        if (bits) {
            unsigned *m = sM + y * nwx + (x >> 5);
            const unsigned bit = 1u << (x & 31);
#pragma unroll
            for (int f = 0; f < NF; ++f)
                if ((bits >> f) & 1u) atomicOr(m + f * plane, bit);
        }
    }
}

// Phases 3 and 4 of one tile whose window (sD, sH) and start points (sS) are in shared memory and
// whose flag plane M is clear: every thread of the CTA calls this; it synchronises the CTA.
template <class Cfg, int NF>
__device__ __forceinline__ void tile_compute(const TileArgs &a, int x0, int y0, const Win &w,
                                             bool staged, const float2 *sD, const float4 *sH, const float2 *sS,
                                             unsigned *sM, unsigned *sB, LocalCounters &cnt)
{
    constexpr int TX = Cfg::TX, NT = Cfg::NT, ROWS = Cfg::ROWS, TPT = Cfg::TPT, WMAX = Cfg::WMAX;
    constexpr int NG = groups(NF);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int n0 = a.n0, n1 = a.n1;
    const bool limit = a.max_order >= 1 && a.thr >= 0.f;
    // ---- phase 3: jump flags (Sec. 2.3) and their OR over each element's 4x4 stencil ---------
    // Flags of the interior nodes go to bit plane M (one bit per node and field, set with a
    // shared-memory atomic: flagged nodes are few); then B = M ORed over 4 rows and bits x-1 .. x+2.
    const int nwx = (w.wx + 31) >> 5, plane = w.wy * nwx;
    if (limit) {
        flag_window<Cfg, NF>(a, w, sH, sM, nwx, plane);
        __syncthreads();
        // rows 2 .. wy-4 (the elements whose stencil lies in the interior rows 1 .. wy-2)
        const int brows = w.wy - 5;
        const float inv_b = 1.f / (float)max(brows, 1);
        for (int q = threadIdx.x; q < NF * brows; q += NT) {
            const int f = row_of(q, inv_b), y = q - f * brows + 2;
            const unsigned *m = sM + f * plane + (y - 1) * nwx;
            unsigned *b = sB + f * plane + y * nwx;
            unsigned vp = 0u, vc = m[0] | m[nwx] | m[2 * nwx] | m[3 * nwx];
            for (int kw = 0; kw < nwx; ++kw) {
                const int k1 = kw + 1;
                const unsigned vq = k1 < nwx ? (m[k1] | m[nwx + k1] | m[2 * nwx + k1] | m[3 * nwx + k1]) : 0u;
                b[kw] = vc | __funnelshift_l(vp, vc, 1) | __funnelshift_r(vc, vq, 1) | __funnelshift_r(vc, vq, 2);
                vp = vc;
                vc = vq;
            }
        }
        __syncthreads();
    }

    // ---- phase 4: per target: search, Newton, order, tensor Z-spline sum ---------------------
    // Targets that leave the fast path are marked and finished after the loop, so that the loop
    // carries no call.
    if (!staged && threadIdx.x == 0) cnt.fallback += 1;
    unsigned slow = 0u;
#pragma unroll 1
    for (int k = 0; k < TPT; ++k) {
        const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
        if (jx >= n0 || jy >= n1) continue;
        const long long jj = (long long)jy * n0 + jx;
        int ex, ey;
        refined_start(w, sD, staged, jx, jy, sS[k * NT + threadIdx.x], ex, ey);
        int hops = 0, iters = 0;
        float xi0 = 0.f, xi1 = 0.f;
        bool ok = staged && walk_window(w, sD, a.walk_max, a.max_iter, jx, jy, ex, ey, xi0, xi1, hops, iters);
        const int rx = ex - w.lox, ry = ey - w.loy;
        ok = ok && rx >= 2 && rx <= w.wx - 4 && ry >= 2 && ry <= w.wy - 4;
        if (ok) {
            cnt.targets += 1;
            cnt.hops += hops;
            cnt.hops_max = max(cnt.hops_max, (unsigned)hops);
            cnt.iters += iters;
            cnt.iters_max = max(cnt.iters_max, (unsigned)iters);
            // Sec. 2.3: fields flagged anywhere in the element's 4x4 stencil drop to linear
            unsigned lin_mask = a.max_order == 0 ? 0xffu : 0u;
            if (limit) {
                const unsigned *b = sB + ry * nwx + (rx >> 5);
                lin_mask = 0u;
#pragma unroll
                for (int f = 0; f < NF; ++f) lin_mask |= ((b[f * plane] >> (rx & 31)) & 1u) << f;
            }
            const unsigned nlin = __popc(lin_mask & ((1u << NF) - 1u));
            cnt.oh0 += nlin;
            cnt.oh1 += NF - nlin;
            float wc[2][4];
            cubic_weights(xi0, wc[0]);
            cubic_weights(xi1, wc[1]);
            const int o = (ry - 1) * w.wx + (rx - 1);
            store_group<NF, 0>(a, jj, sH + o, w.wx, wc, xi0, xi1, lin_mask);
            if constexpr (NG > 1) store_group<NF, 1>(a, jj, sH + WMAX + o, w.wx, wc, xi0, xi1, lin_mask);
        } else {
            slow |= 1u << k;
        }
    }
#pragma unroll 1
    for (int k = 0; slow != 0u; ++k, slow >>= 1) {
        if (!(slow & 1u)) continue;
        const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
        const long long jj = (long long)jy * n0 + jx;
        const float2 s0 = sS[k * NT + threadIdx.x];
        int ex, ey;
        refined_start(w, sD, staged, jx, jy, s0, ex, ey);
        const TargetOut r = slow_target<NF>(a, w, sD, sH, WMAX, sB, limit, jj, jx, jy, ex, ey,
                                            (int)floorf(s0.x), (int)floorf(s0.y));
        cnt.targets += 1;
        cnt.hops += r.hops;
        cnt.hops_max = max(cnt.hops_max, (unsigned)r.hops);
        cnt.iters += r.iters;
        cnt.iters_max = max(cnt.iters_max, (unsigned)r.iters);
        cnt.f64 += r.f64;
        if (r.st != ST_OK) {
            cnt.fl += r.st == ST_LOCATE;
            cnt.fn += r.st == ST_NEWTON;
            cnt.ff += r.st == ST_FOLD;
        } else {
            cnt.oh0 += r.nlin;
            cnt.oh1 += NF - r.nlin;
        }
    }
}


// eq. (vel): the next step's trajectories of the tile's own nodes (fused steps).  They depend on
// the velocity only, so callers run them while the window copies are in flight.
template <class Cfg>
__device__ __forceinline__ void integrate_next(const TileArgs &a, const VelArgs<float> &vn, int x0, int y0)
{
    const int tx = threadIdx.x % Cfg::TX, ty = threadIdx.x / Cfg::TX;
#pragma unroll 1
    for (int k = 0; k < Cfg::TPT; ++k) {
        const int jx = x0 + tx, jy = y0 + ty + k * Cfg::ROWS;
        if (jx >= a.n0 || jy >= a.n1) continue;
        float X[3] = {node_position(vn.lo[0], jx, vn.dx[0]), node_position(vn.lo[1], jy, vn.dx[1]), 0.f}, d[3];
        trajectory_cells<float, 2>(vn, X, d);
        reinterpret_cast<float2 *>(a.D_next)[(long long)jy * a.n0 + jx] = make_float2(d[0], d[1]);
    }
}

// Sec. 3.2: the next step's displacements of a carried velocity are the remapped velocity of the
// tile's own targets, D = dt u / dx; each thread reads back the outputs it wrote itself.
template <class Cfg>
__device__ __forceinline__ void carried_next(const TileArgs &a, int x0, int y0)
{
    const int tx = threadIdx.x % Cfg::TX, ty = threadIdx.x / Cfg::TX;
#pragma unroll 1
    for (int k = 0; k < Cfg::TPT; ++k) {
        const int jx = x0 + tx, jy = y0 + ty + k * Cfg::ROWS;
        if (jx >= a.n0 || jy >= a.n1) continue;
        const long long jj = (long long)jy * a.n0 + jx;
        reinterpret_cast<float2 *>(a.D_next)[jj] =
            make_float2(a.csc[0] * a.out[a.vf[0]][jj], a.csc[1] * a.out[a.vf[1]][jj]);
    }
}

// One TX x TY tile of targets with origin (x0, y0), staged and computed in one pass: every thread
// of the CTA calls this; it synchronises the CTA.
template <class Cfg, int NF, bool FUSED>
__device__ __forceinline__ void process_tile(const TileArgs &a, const VelArgs<float> &vn, int x0, int y0,
                                             const TileSmem<Cfg, NF> &sm, int *sBox, LocalCounters &cnt)
{
    constexpr int TX = Cfg::TX, NT = Cfg::NT, ROWS = Cfg::ROWS, TPT = Cfg::TPT;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    if (threadIdx.x < 4) sBox[threadIdx.x] = (threadIdx.x < 2) ? INT_MAX : INT_MIN;

    // ---- phase 1: start elements floor(j - D_j) and their bounding box ----------------------
    int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN;
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
        float2 s0 = make_float2((float)jx, (float)jy);
        if (jx < a.n0 && jy < a.n1) {
            s0 = start_point(jx, jy, __ldg(reinterpret_cast<const float2 *>(a.D) + (long long)jy * a.n0 + jx));
            mnx = min(mnx, (int)floorf(s0.x));
            mny = min(mny, (int)floorf(s0.y));
            mxx = max(mxx, (int)floorf(s0.x));
            mxy = max(mxy, (int)floorf(s0.y));
        }
        sm.S[k * NT + threadIdx.x] = s0;
    }
    __syncthreads();
    int bx0, by0, bx1, by1;
    reduce_box(mnx, mny, mxx, mxy, sBox, bx0, by0, bx1, by1);
    bool staged;
    const Win w = window_of<Cfg::WMAX>(bx0, by0, bx1, by1, a.n0, a.n1, staged);

    // ---- phase 2: stage displacements and fields of the window (all copies in flight) -------
    stage_window<Cfg, NF>(a, w, sm.D, sm.H);
    clear_flags<Cfg, NF>(a, w, sm.M);
    if (FUSED && a.D_next != nullptr && !a.carried) integrate_next<Cfg>(a, vn, x0, y0);
    cp_async_wait_all();
    __syncthreads();
    tile_compute<Cfg, NF>(a, x0, y0, w, staged, sm.D, sm.H, sm.S, sm.M, sm.B, cnt);
    if (FUSED && a.D_next != nullptr && a.carried) carried_next<Cfg>(a, x0, y0);
}

// the counters of a one-tile CTA: each warp adds into its SM's copy, with no block barrier
__device__ __forceinline__ void flush_counters_sm(const LocalCounters &cnt, const TileArgs &a)
{
    if (a.stripes == nullptr) {
        flush_counters(cnt, a.counters);
        return;
    }
    unsigned smid;
    asm("mov.u32 %0, %%smid;" : "=r"(smid));
    flush_counters_warp(cnt, a.stripes + (smid % SL_COUNTER_STRIPES));
}

template <class Cfg, int NF, bool FUSED>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB) remap_tiled2d_kernel(const __grid_constant__ TileArgs a, const VelArgs<float> vn)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sBox[4];
    const TileSmem<Cfg, NF> sm(smem);
    LocalCounters cnt;
    cnt.clear();
    process_tile<Cfg, NF, FUSED>(a, vn, blockIdx.x * Cfg::TX, blockIdx.y * Cfg::TY, sm, sBox, cnt);
    flush_counters_sm(cnt, a);
}

// Pipelined persistent variant: each CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... and
// overlaps the memory traffic of the next tiles with the arithmetic of the current one.  While
// tile t is computed, the window of tile t + G is being copied into the other window slot and the
// displacements of tile t + 2G's targets into a third start-point slot, so that every copy has a
// whole tile of arithmetic to arrive in.
template <class Cfg, int NF, bool FUSED>
__global__ void __launch_bounds__(Cfg::NT, 1)
    remap_pipe2d_kernel(const __grid_constant__ TileArgs a, const VelArgs<float> vn, int tiles_x, int ntiles)
{
    constexpr int TX = Cfg::TX, TY = Cfg::TY, NT = Cfg::NT, ROWS = Cfg::ROWS, TPT = Cfg::TPT, WMAX = Cfg::WMAX;
    constexpr int NG = groups(NF), NTGT = TX * TY;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sBox[2][4];
    float2 *const sD = reinterpret_cast<float2 *>(smem);                 // 2 window slots
    float4 *const sH = reinterpret_cast<float4 *>(sD + 2 * WMAX);         // 2 window slots
    float2 *const sS = reinterpret_cast<float2 *>(sH + 2 * NG * WMAX);    // 3 start-point slots
    unsigned *const sM = reinterpret_cast<unsigned *>(sS + 3 * NTGT);
    unsigned *const sB = sM + NF * mask_words(WMAX);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX, G = (int)gridDim.x;
    LocalCounters cnt;
    cnt.clear();
    if (threadIdx.x < 8) sBox[threadIdx.x >> 2][threadIdx.x & 3] = (threadIdx.x & 3) < 2 ? INT_MAX : INT_MIN;

    // raw displacements of tile t's targets into start-point slot S (asynchronous)
    auto fetch_targets = [&](int t, float2 *S) {
        const int tr = t / tiles_x, x0 = (t - tr * tiles_x) * TX, y0 = tr * TY;
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
            if (jx < a.n0 && jy < a.n1)
                cp_async<8>(S + k * NT + threadIdx.x, reinterpret_cast<const float2 *>(a.D) + (long long)jy * a.n0 + jx);
        }
    };
    // start points of tile t (in place in S) and its window; box is reset, the other box gets
    // reset for the next call; contains a barrier
    auto window = [&](int t, float2 *S, int *box, int *other, bool &staged) -> Win {
        const int tr = t / tiles_x, x0 = (t - tr * tiles_x) * TX, y0 = tr * TY;
        int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN;
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
            if (jx < a.n0 && jy < a.n1) {
                const float2 s0 = start_point(jx, jy, S[k * NT + threadIdx.x]);
                S[k * NT + threadIdx.x] = s0;
                mnx = min(mnx, (int)floorf(s0.x));
                mny = min(mny, (int)floorf(s0.y));
                mxx = max(mxx, (int)floorf(s0.x));
                mxy = max(mxy, (int)floorf(s0.y));
            }
        }
        int bx0, by0, bx1, by1;
        reduce_box(mnx, mny, mxx, mxy, box, bx0, by0, bx1, by1);
        if (threadIdx.x < 4) other[threadIdx.x] = threadIdx.x < 2 ? INT_MAX : INT_MIN;
        return window_of<WMAX>(bx0, by0, bx1, by1, a.n0, a.n1, staged);
    };

    const int t0 = blockIdx.x;
    if (t0 < ntiles) {
        fetch_targets(t0, sS);
        if (t0 + G < ntiles) fetch_targets(t0 + G, sS + NTGT);
        cp_async_wait_all();
        __syncthreads();
        bool st_cur;
        Win w_cur = window(t0, sS, sBox[0], sBox[1], st_cur);
        stage_window<Cfg, NF>(a, w_cur, sD, sH);
        int s3 = 0;  // start-point slot of the current tile (i mod 3)
        for (int i = 0;; ++i) {
            const int t = t0 + i * G;
            if (t >= ntiles) break;
            const int tn = t + G, tnn = t + 2 * G, p = i & 1;
            const int s3n = s3 == 2 ? 0 : s3 + 1, s3nn = s3n == 2 ? 0 : s3n + 1;
            cp_async_wait_all();  // window of t, displacements of tn's targets
            __syncthreads();      // ... visible to all; tile t - G finished
            clear_flags<Cfg, NF>(a, w_cur, sM);
            bool st_nxt = false;
            Win w_nxt;
            w_nxt.lox = w_nxt.loy = w_nxt.wx = w_nxt.wy = 0;
            if (tn < ntiles) {
                w_nxt = window(tn, sS + s3n * NTGT, sBox[p ^ 1], sBox[p], st_nxt);
                stage_window<Cfg, NF>(a, w_nxt, sD + (p ^ 1) * WMAX, sH + (p ^ 1) * NG * WMAX);
                if (tnn < ntiles) fetch_targets(tnn, sS + s3nn * NTGT);
            } else {
                __syncthreads();
            }
            const int tr = t / tiles_x;
            if (FUSED && a.D_next != nullptr) integrate_next<Cfg>(a, vn, (t - tr * tiles_x) * TX, tr * TY);
            tile_compute<Cfg, NF>(a, (t - tr * tiles_x) * TX, tr * TY, w_cur, st_cur, sD + p * WMAX,
                                  sH + p * NG * WMAX, sS + s3 * NTGT, sM, sB, cnt);
            w_cur = w_nxt;
            st_cur = st_nxt;
            s3 = s3n;
        }
    }
    flush_counters(cnt, a.counters);
}

template <class Cfg>
__host__ size_t pipe_smem_bytes(int nfields)
{
    return 2 * (size_t)Cfg::WMAX * (sizeof(float2) + sizeof(float4) * (size_t)((nfields + 3) / 4)) +
           3 * sizeof(float2) * (size_t)(Cfg::TX * Cfg::TY) + 2 * sizeof(unsigned) * (size_t)nfields * (size_t)mask_words(Cfg::WMAX);
}

template <class Cfg>
__host__ size_t tile_smem_bytes(int nfields)
{
    return (size_t)Cfg::WMAX * (sizeof(float2) + sizeof(float4) * (size_t)((nfields + 3) / 4)) +
           sizeof(float2) * (size_t)(Cfg::TX * Cfg::TY) + 2 * sizeof(unsigned) * (size_t)nfields * (size_t)mask_words(Cfg::WMAX);
}

__host__ inline TileArgs make_tile_args(const sl_grid *g, const void *D, void *D_next, const void *const *in,
                                        void *const *out)
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
    a.stripes = g->stripes;
    return a;
}

// fused steps of a carried velocity take the next step's D from the remapped velocity fields
__host__ inline void set_carried(const sl_grid *g, double dt, TileArgs &a)
{
    if (!g->carried) return;
    a.carried = 1;
    for (int c = 0; c < 2; ++c) {
        a.vf[c] = g->vel_field[c];
        a.csc[c] = (float)(dt / g->dx[c]);
    }
}

// opt-in shared memory above 48 KB is a per-device function attribute: set it once per device
template <class K>
__host__ cudaError_t allow_smem(K kernel, int device, size_t bytes, bool *configured)
{
    if (!configured[device & 63]) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        configured[device & 63] = true;
    }
    return cudaSuccess;
}

template <class Cfg, int NF, bool FUSED>
__host__ cudaError_t launch_tiled_nf(const sl_grid *g, const TileArgs &a, const VelArgs<float> &vn, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes<Cfg>(NF);
    static bool configured[64] = {};
    cudaError_t e = allow_smem(remap_tiled2d_kernel<Cfg, NF, FUSED>, g->device, smem, configured);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g->n[0] + Cfg::TX - 1) / Cfg::TX), (unsigned)((g->n[1] + Cfg::TY - 1) / Cfg::TY));
    remap_tiled2d_kernel<Cfg, NF, FUSED><<<grid, Cfg::NT, smem, s>>>(a, vn);
    return cudaGetLastError();
}

template <class Cfg, bool FUSED>
__host__ cudaError_t launch_tiled_fused(const sl_grid *g, const TileArgs &a, const VelArgs<float> &vn, cudaStream_t s)
{
    switch (g->nfields) {
    case 1: return launch_tiled_nf<Cfg, 1, FUSED>(g, a, vn, s);
    case 2: return launch_tiled_nf<Cfg, 2, FUSED>(g, a, vn, s);
    case 3: return launch_tiled_nf<Cfg, 3, FUSED>(g, a, vn, s);
    case 4: return launch_tiled_nf<Cfg, 4, FUSED>(g, a, vn, s);
    case 5: return launch_tiled_nf<Cfg, 5, FUSED>(g, a, vn, s);
    case 6: return launch_tiled_nf<Cfg, 6, FUSED>(g, a, vn, s);
    case 7: return launch_tiled_nf<Cfg, 7, FUSED>(g, a, vn, s);
    default: return launch_tiled_nf<Cfg, 8, FUSED>(g, a, vn, s);
    }
}

template <class Cfg, int NF, bool FUSED>
__host__ cudaError_t launch_pipe_nf(const sl_grid *g, const TileArgs &a, const VelArgs<float> &vn, cudaStream_t s)
{
    const size_t smem = pipe_smem_bytes<Cfg>(NF);
    static bool configured[64] = {};
    static int per_sm[64] = {};
    cudaError_t e = allow_smem(remap_pipe2d_kernel<Cfg, NF, FUSED>, g->device, smem, configured);
    if (e != cudaSuccess) return e;
    if (per_sm[g->device & 63] == 0) {
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, remap_pipe2d_kernel<Cfg, NF, FUSED>, Cfg::NT, smem);
        if (e != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        per_sm[g->device & 63] = n;
    }
    const long long tiles_x = (g->n[0] + Cfg::TX - 1) / Cfg::TX, tiles_y = (g->n[1] + Cfg::TY - 1) / Cfg::TY;
    const long long ntiles = tiles_x * tiles_y;
    const long long ctas = std::min(ntiles, (long long)g->num_sms * per_sm[g->device & 63]);
    remap_pipe2d_kernel<Cfg, NF, FUSED><<<(unsigned)ctas, Cfg::NT, smem, s>>>(a, vn, (int)tiles_x, (int)ntiles);
    return cudaGetLastError();
}

// one pipelined remap (fused: also D(t_next)) of a 2-D FP32 grid with at most 4 fields
template <class Cfg>
__host__ cudaError_t launch_pipe_cfg(const sl_grid *g, const void *D, void *D_next, double t_next, double dt,
                                     bool fused, const void *const *in, void *const *out, cudaStream_t s)
{
    const TileArgs a = make_tile_args(g, D, D_next, in, out);
    VelArgs<float> vn;
    memset(&vn, 0, sizeof(vn));
    if (fused) vn = make_vel_args<float>(g, t_next, dt);
    switch (g->nfields) {
    case 1: return fused ? launch_pipe_nf<Cfg, 1, true>(g, a, vn, s) : launch_pipe_nf<Cfg, 1, false>(g, a, vn, s);
    case 2: return fused ? launch_pipe_nf<Cfg, 2, true>(g, a, vn, s) : launch_pipe_nf<Cfg, 2, false>(g, a, vn, s);
    case 3: return fused ? launch_pipe_nf<Cfg, 3, true>(g, a, vn, s) : launch_pipe_nf<Cfg, 3, false>(g, a, vn, s);
    case 4: return fused ? launch_pipe_nf<Cfg, 4, true>(g, a, vn, s) : launch_pipe_nf<Cfg, 4, false>(g, a, vn, s);
    default: return cudaErrorNotSupported;
    }
}

// one tiled remap (fused: also D(t_next) for the tile's nodes) of a 2-D FP32 grid
template <class Cfg>
__host__ cudaError_t launch_tiled_cfg(const sl_grid *g, const void *D, void *D_next, double t_next, double dt,
                                      bool fused, const void *const *in, void *const *out, cudaStream_t s)
{
    TileArgs a = make_tile_args(g, D, D_next, in, out);
    if (fused) {
        set_carried(g, dt, a);
        const VelArgs<float> vn = make_vel_args<float>(g, t_next, dt);
        return launch_tiled_fused<Cfg, true>(g, a, vn, s);
    }
    VelArgs<float> vn;
    memset(&vn, 0, sizeof(vn));
    return launch_tiled_fused<Cfg, false>(g, a, vn, s);
}

}  // namespace
