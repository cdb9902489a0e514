// sl_remap2d.cuh -- persistent 2-D FP32 remap of the FSL step (arXiv:1410.2817) with TMA-staged
// departure windows: each CTA walks through a static list of TX x TY tiles of target (reference)
// nodes (the last, partial round cut into half tiles, see item2).
//
// Per tile (Sec. 2.2, 2.3, eq. multiZ):
//   1. start points s = j - D_j of the tile's targets and the box of their elements floor(s);
//   2. the departure window -- that box widened by the walk slack, the cubic stencil (c-1 .. c+2)
//      and the limiter's neighbours -- is copied to shared memory: the displacement and the field
//      planes by cp.async.bulk.tensor box loads (one box per plane, one mbarrier, no multicast), or by
//      per-element asynchronous copies when the window crosses the periodic seam;
//   3. one pass over the window computes every node's jump flags (Sec. 2.3) and rewrites the
//      planar field values as float4 records (h0, h1, h2, flag bits), so that one 128-bit shared
//      load brings a stencil tap's three values and the flags its order test needs;
//   4. every target: refined start, element walk with FP32 Newton inversion (Sec. 2.2, eq.
//      mapping1), order from the OR of the 16 taps' flag bits, cubic and bilinear tensor sums
//      (eq. multiZ) on packed FP32x2 FMAs.  Consecutive lanes take consecutive targets of a row,
//      so that their shared-memory reads fall in distinct banks.
// The window of the CTA's next tile is copied while the current tile is computed (two window
// slots); the next tile's displacements are loaded into registers one tile ahead.  The fused
// variant also integrates the next step's trajectories of the tile's nodes (eq. vel; the swirl's
// two nodes of a thread at a time on packed FP32x2 arithmetic).  Targets the
// fast path cannot finish (walk leaves the window, FP32 Newton fails or meets a nearly degenerate
// element) take the general path of the shared tile body: walk with global reads, FP64 re-solve.
//
// Waits on an mbarrier are bounded in time; a wait that runs out is counted in the grid's
// timeout counter and the CTA stops (the host reports SL_ERR_CUDA).
#pragma once

#include "sl_async.cuh"
#include "sl_tile2d.cuh"

namespace {

// TX x TY targets per tile, NT threads (each a column of both halves of the tile row per pass), window capacity
// WX x WY nodes (WX a multiple of 4 for the TMA box, WY a multiple of the 8-row strip)
template <int TX_, int TY_, int NT_, int WX_, int WY_, int MINB_>
struct R2Cfg {
    static constexpr int TX = TX_, TY = TY_, NT = NT_, WX = WX_, WY = WY_, MINB = MINB_;
    static constexpr int PX = TX / 2;          // target pairs per tile row
    static constexpr int ROWS = NT / PX;       // tile rows per pass
    static constexpr int PPT = TY / ROWS;      // pairs per thread
    static constexpr int STRIP = 8;            // the window capacity's rows come in multiples of 8
    static constexpr int CH = 4;               // rows per work item of the flag pass
    static_assert(PX % 16 == 0 && NT % PX == 0 && TY % ROWS == 0, "bad remap2d tile");
    static_assert(WX % 4 == 0 && WY % STRIP == 0 && 2 * WX <= 256, "bad remap2d window");
    // dynamic shared memory (bytes): planar staging of 3 planes, two displacement windows, the
    // float4 records, two slots of start points
    static constexpr size_t STAGE = 3ull * WY * WX * 4, DWIN = 2ull * WY * WX * 8, REC = 1ull * WY * WX * 16;
    static constexpr size_t SPTS = 2ull * (TX * TY) * 8;
    static constexpr size_t SMEM = STAGE + DWIN + REC + SPTS + 128;  // + room to align the base
};
typedef R2Cfg<64, 32, 512, 88, 48, 1> R2Wide;    // one CTA of 16 warps per SM
typedef R2Cfg<32, 32, 256, 44, 48, 2> R2Square;  // two CTAs of 8 warps per SM

struct R2Maps {
    CUtensorMap f[3];  // field planes: FP32, dims (n0, n1), box (WX, WY)
    CUtensorMap D;     // displacement as FP32 pairs: dims (2 n0, n1), box (2 WX, WY)
};

// window of one tile: origin, extent, and how it is staged
struct Win2 {
    int lox, loy, wx, wy;
    int mode;  // 0: not staged (general path), 1: TMA boxes, 2: per-element copies
};

template <int WX>
__device__ __forceinline__ bool w2_has(const Win2 &w, int x, int y)
{
    return (unsigned)(x - w.lox) < (unsigned)w.wx && (unsigned)(y - w.loy) < (unsigned)w.wy;
}
template <int WX>
__device__ __forceinline__ int w2_at(const Win2 &w, int x, int y)
{
    return (y - w.loy) * WX + (x - w.lox);
}

struct R2Args {
    TileArgs t;        // grid, fields, displacement, counters (the shared tile body's arguments)
    int tiles_x, ntiles;
    int use_tma;       // the tensor maps are valid
    unsigned long long *timeouts;  // counter of waits that ran out
};

// ---- window of a tile from the box of its start elements --------------------------------------
template <class Cfg>
__device__ __forceinline__ Win2 window2(int bx0, int by0, int bx1, int by1, int n0, int n1, bool tma)
{
    Win2 w;
    // nodes x0 .. x1 the walk (slack 1), the stencil (c-1 .. c+2) and the limiter (one more on
    // each side) may touch; the origin is rounded down to a multiple of 4 for the box copies
    const long long x0 = (long long)bx0 - WALK_SLACK - 2, x1 = (long long)bx1 + WALK_SLACK + 3;
    const long long y0 = (long long)by0 - WALK_SLACK - 2, y1 = (long long)by1 + WALK_SLACK + 3;
    const long long lox = x0 & ~3LL;
    const long long wx = x1 - lox + 1, wy = y1 - y0 + 1;
    const bool fits = bx0 <= bx1 && by0 <= by1 && wx <= Cfg::WX && wy <= Cfg::WY && lox >= -n0 && y0 >= -n1 &&
                      lox + wx <= 2LL * n0 && y0 + wy <= 2LL * n1;
    w.lox = fits ? (int)lox : 0;
    w.loy = fits ? (int)y0 : 0;
    w.wx = fits ? (int)wx : 0;
    w.wy = fits ? (int)wy : 0;
    w.mode = !fits ? 0 : (tma && lox >= 0 && y0 >= 0 && lox + wx <= n0 && y0 + wy <= n1) ? 1 : 2;
    return w;
}

// ---- Sec. 2.2 element search with global reads where the window ends (general path) ----------
template <class Cfg, typename TN>
__device__ __forceinline__ int walk2w(const TileArgs &a, const Win2 &w, const float2 *sD, int jx, int jy, int &cx,
                                      int &cy, TN xi[3], int &hops, int &iters, bool &degen)
{
    const TN tol = sizeof(TN) == 8 ? TN(1e-14) : TN(SL_NEWTON_TOL_F32);
    const TN slack = sizeof(TN) == 8 ? TN(1e-12) : TN(SL_SLACK_F32);
    CycleCheck cyc;
    cyc.start(cx, cy, 0);
    for (int hop = 0; hop < a.walk_max; ++hop) {
        TN P[8][3];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int x = cx + (v & 1), y = cy + (v >> 1);
            const float2 d = (w.mode != 0 && w2_has<Cfg::WX>(w, x, y))
                                 ? sD[w2_at<Cfg::WX>(w, x, y)]
                                 : __ldg(reinterpret_cast<const float2 *>(a.D) + gidx(x, y, a.n0, a.n1));
            P[v][0] = TN(x - jx) + TN(d.x);
            P[v][1] = TN(y - jy) + TN(d.y);
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

// Start element of a target: one fixed-point step s <- j - D(s) from s0 = j - D_j with D(s0)
// bilinear in the staged window (the walk still decides); floor(s0) when not staged.
template <class Cfg>
__device__ __forceinline__ void refined_start2(const Win2 &w, const float2 *sD, int jx, int jy, float sx, float sy,
                                               int &ex, int &ey)
{
    ex = (int)floorf(sx);
    ey = (int)floorf(sy);
    if (w.mode == 0 || !(w2_has<Cfg::WX>(w, ex, ey) && w2_has<Cfg::WX>(w, ex + 1, ey + 1))) return;
    const int i0 = w2_at<Cfg::WX>(w, ex, ey);
    const float fx = sx - (float)ex, fy = sy - (float)ey;
    const float2 d00 = sD[i0], d10 = sD[i0 + 1], d01 = sD[i0 + Cfg::WX], d11 = sD[i0 + Cfg::WX + 1];
    const float bx = fmaf(fx, d10.x - d00.x, d00.x), by = fmaf(fx, d10.y - d00.y, d00.y);
    const float dx = fmaf(fy, fmaf(fx, d11.x - d01.x, d01.x) - bx, bx);
    const float dy = fmaf(fy, fmaf(fx, d11.y - d01.y, d01.y) - by, by);
    const float rx = (float)jx - dx, ry = (float)jy - dy;
    if (finite_t(rx) && finite_t(ry) && fabsf(rx - sx) < 4.f && fabsf(ry - sy) < 4.f) {
        ex = (int)floorf(rx);
        ey = (int)floorf(ry);
    }
}

// Sec. 2.2 element search inside the staged window, FP32 Newton (the arithmetic of walk2w<float>).
// False when the walk leaves the window, Newton fails or the element is nearly degenerate.
template <class Cfg>
__device__ __forceinline__ bool walk_fast2(const Win2 &w, const float2 *sD, int walk_max, int max_iter, int jx, int jy,
                                           int &ex, int &ey, float &xi0, float &xi1, int &hops, int &iters)
{
    const float slack = SL_SLACK_F32;
    CycleCheck cyc;
    cyc.start(ex, ey, 0);
    for (int hop = 0; hop < walk_max; ++hop) {
        if (!(w2_has<Cfg::WX>(w, ex, ey) && w2_has<Cfg::WX>(w, ex + 1, ey + 1))) return false;
        const int i0 = w2_at<Cfg::WX>(w, ex, ey);
        const float2 d0 = sD[i0], d1 = sD[i0 + 1], d2 = sD[i0 + Cfg::WX], d3 = sD[i0 + Cfg::WX + 1];
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
        if (st != ST_OK || degen) return false;
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

// eq. (multiZ) from the float4 records of the 4x4 stencil starting at r (pitch WX): the cubic sum
// of fields 0, 1 (packed pair) and 2 (the pair with the flag word, whose second lane is unused),
// the bilinear sum over the element's own vertices, and the OR of the 16 flag words.  Fields whose
// flag bit is set anywhere in the stencil take the bilinear value (Sec. 2.3; order 0 for every
// field when max_order is 0).
template <int WX, int NF>
__device__ __forceinline__ void stencil_sum(const float4 *r, float xi0, float xi1, bool limit, bool linear_only,
                                            float v[3], unsigned &nlin)
{
    float wc[2][4];
    cubic_weights(xi0, wc[0]);
    cubic_weights(xi1, wc[1]);
    const float2 w0 = bcast2(wc[0][0]), w1 = bcast2(wc[0][1]), w2 = bcast2(wc[0][2]), w3 = bcast2(wc[0][3]);
    const float2 u0 = bcast2(1.f - xi0), u1 = bcast2(xi0);
    const float2 z = make_float2(0.f, 0.f);
    float2 cl = z, ch = z, ll = z, lh = z;
    unsigned bits = 0u;
#pragma unroll
    for (int ky = 0; ky < 4; ++ky) {
        const float4 t0 = r[0], t1 = r[1], t2 = r[2], t3 = r[3];
        bits |= __float_as_uint(t0.w) | __float_as_uint(t1.w) | __float_as_uint(t2.w) | __float_as_uint(t3.w);
        const float2 wy = bcast2(wc[1][ky]);
        float2 q = __fmul2_rn(w0, lo2(t0));
        q = __ffma2_rn(w1, lo2(t1), q);
        q = __ffma2_rn(w2, lo2(t2), q);
        q = __ffma2_rn(w3, lo2(t3), q);
        cl = __ffma2_rn(wy, q, cl);
        if (NF > 2) {
            float2 p = __fmul2_rn(w0, hi2(t0));
            p = __ffma2_rn(w1, hi2(t1), p);
            p = __ffma2_rn(w2, hi2(t2), p);
            p = __ffma2_rn(w3, hi2(t3), p);
            ch = __ffma2_rn(wy, p, ch);
        }
        if (ky == 1 || ky == 2) {
            const float2 vy = bcast2(ky == 1 ? 1.f - xi1 : xi1);
            ll = __ffma2_rn(vy, __ffma2_rn(u1, lo2(t2), __fmul2_rn(u0, lo2(t1))), ll);
            if (NF > 2) lh = __ffma2_rn(vy, __ffma2_rn(u1, hi2(t2), __fmul2_rn(u0, hi2(t1))), lh);
        }
        r += WX;
    }
    const unsigned lin = linear_only ? 7u : (limit ? bits : 0u);
    v[0] = (lin & 1u) ? ll.x : cl.x;
    v[1] = (lin & 2u) ? ll.y : cl.y;
    v[2] = (lin & 4u) ? lh.x : ch.x;
    nlin = __popc(lin & ((1u << NF) - 1u));
}

// The general path of one target (rare, out of line): walk from the refined start with global
// reads where the window ends; on failure or a nearly degenerate element the FP64 re-solve from the
// first start element; then order and sum from the records when the stencil lies in the flagged
// part of the window, from global memory otherwise.  A target that still fails keeps its values.
template <class Cfg, int NF>
__device__ __noinline__ TargetOut slow_target2(const TileArgs &a, const Win2 w, const float2 *sD, const float4 *sR,
                                               bool limit, int jx, int jy, int ex, int ey, int c0x, int c0y)
{
    TargetOut r = {ST_OK, 0, 0, 0, 0};
    const long long jj = (long long)jy * a.n0 + jx;
    float xf[3] = {0.f, 0.f, 0.f};
    bool degen = false;
    int st = walk2w<Cfg, float>(a, w, sD, jx, jy, ex, ey, xf, r.hops, r.iters, degen);
    float xi0 = xf[0], xi1 = xf[1];
    if (st != ST_OK || degen) {
        if (st == ST_LOCATE || st == ST_FOLD) {
            ex = c0x;
            ey = c0y;
        }
        double xd[3] = {0.0, 0.0, 0.0};
        bool dg = false;
        st = walk2w<Cfg, double>(a, w, sD, jx, jy, ex, ey, xd, r.hops, r.iters, dg);
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
    const bool fast = w.mode != 0 && rx >= 2 && rx <= w.wx - 4 && ry >= 2 && ry <= w.wy - 4;
    if (fast) {
        float v[3];
        unsigned nlin;
        stencil_sum<Cfg::WX, NF>(sR + (ry - 1) * Cfg::WX + (rx - 1), xi0, xi1, limit, a.max_order == 0, v, nlin);
#pragma unroll
        for (int f = 0; f < NF; ++f) a.out[f][jj] = v[f];
        r.nlin = (int)nlin;
    } else {
        const unsigned lin_mask = a.max_order == 0 ? 0xffu : (limit ? box_flags_global(a, ex, ey) : 0u);
        r.nlin = __popc(lin_mask & ((1u << NF) - 1u));
        interp_global(a, jj, ex, ey, xi0, xi1, lin_mask);
    }
    return r;
}

// ---- the flag pass: planar staging -> float4 records with the flag bits -------------------------
// Sec. 2.3 jump test from the two one-sided differences dp = h+ - h, dm = h - h- of a node.
__device__ __forceinline__ bool jump_dd(float dp, float dm, float thr)
{
    return fabsf(dp - dm) > thr * fmaxf(fabsf(dp), fabsf(dm));
}

// Records are written for the window's interior nodes (1 .. wx-2, 1 .. wy-2), whose four
// neighbours are staged.  Consecutive threads take consecutive interior nodes of the window (row by
// row), so that every shared-memory read of a node and of its four neighbours, and every record
// written, falls in distinct banks; each node reads its five values per field and writes one
// 128-bit record.
template <class Cfg, int NF>
__device__ __forceinline__ void flag_pass(const Win2 &w, const float *stage, float4 *sR, float thr, bool limit)
{
    constexpr int WX = Cfg::WX, PLANE = WX * Cfg::WY;
    const int iw = w.wx - 2, ni = iw * (w.wy - 2);
    const float inv_iw = 1.f / (float)iw;
    for (int q = threadIdx.x; q < ni; q += Cfg::NT) {
        const int r = row_of(q, inv_iw);
        const int o = (r + 1) * WX + (q - r * iw) + 1;  // the node's offset in a plane
        float hv[3] = {0.f, 0.f, 0.f};
        unsigned bits = 0u;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float *p = stage + f * PLANE + o;
            const float c = p[0];
            hv[f] = c;
            // Sec. 2.3 along x and along y: flagged where |dp - dm| > thr max(|dp|, |dm|)
            if (limit && (jump_dd(p[1] - c, c - p[-1], thr) || jump_dd(p[WX] - c, c - p[-WX], thr))) bits |= 1u << f;
        }
        sR[o] = make_float4(hv[0], hv[1], hv[2], __uint_as_float(bits));
    }
}

// ---- staging of one window --------------------------------------------------------------------
// TMA: thread 0 arms the barrier with the bytes of every strip and issues the box copies.
// Per-element copies: every thread copies its share and makes the barrier track its copies; thread
// 0 adds the barrier's own arrival after a CTA barrier (mbar_finish).  Not staged: thread 0 arrives.
template <class Cfg, int NF>
__device__ __forceinline__ void stage_window2(const R2Args &A, const R2Maps &maps, const Win2 &w, float *stage,
                                              float2 *sD, unsigned long long *bar)
{
    constexpr int WX = Cfg::WX, PLANE = WX * Cfg::WY;
    if (w.mode == 1) {
        // one box of WX x WY per tensor, each issued by its own lane of warp 0 (lane 0 arms the
        // barrier first; the other lanes' copies follow after the warp's shuffle)
        const int lane = threadIdx.x;
        if (lane == 0) mbar_arrive_tx(bar, (unsigned)(Cfg::WY * WX * 4 * (NF + 2)));
        if (threadIdx.x < 32) __syncwarp();
        if (lane < NF)
            tma_load_2d(stage + lane * PLANE, &maps.f[lane], w.lox, w.loy, bar);
        else if (lane == NF)
            tma_load_2d(sD, &maps.D, 2 * w.lox, w.loy, bar);
    } else if (w.mode == 2) {
        const TileArgs &a = A.t;
        const int nwin = w.wx * w.wy;
        const float inv_wx = 1.f / (float)w.wx;
        for (int q = threadIdx.x; q < nwin; q += Cfg::NT) {
            const int yy = row_of(q, inv_wx), xx = q - yy * w.wx;
            const long long gi = (long long)wrap_near(w.loy + yy, a.n1) * a.n0 + wrap_near(w.lox + xx, a.n0);
            const int o = yy * WX + xx;
            cp_async<8>(sD + o, reinterpret_cast<const float2 *>(a.D) + gi);
#pragma unroll
            for (int f = 0; f < NF; ++f) cp_async<4>(stage + f * PLANE + o, a.in[f] + gi);
        }
        mbar_track_cp_async(bar);
    }
}
// the barrier's own arrival for windows not armed by the TMA path; after a CTA barrier that
// follows every thread's mbar_track_cp_async
__device__ __forceinline__ void mbar_finish(const Win2 &w, unsigned long long *bar)
{
    if (threadIdx.x == 0 && w.mode != 1) mbar_arrive(bar);
}

// Targets of a thread: column px of each half of the tile row (x0 + px and x0 + px + TX/2, so that
// consecutive lanes read consecutive shared-memory records), rows py + k ROWS.
template <class Cfg>
__device__ __forceinline__ int target_x(int x0, int h) { return x0 + (int)(threadIdx.x % Cfg::PX) + h * Cfg::PX; }
template <class Cfg>
__device__ __forceinline__ int target_y(int y0, int k) { return y0 + (int)(threadIdx.x / Cfg::PX) + k * Cfg::ROWS; }

// start points of tile t's targets from the displacements in registers, into slot S (float2 per
// target, index (2 k + h) NT + thread); their box
template <class Cfg>
__device__ __forceinline__ void start_points2(const TileArgs &a, int x0, int y0, int ylim, const float2 *dj, float2 *S,
                                              int &mnx, int &mny, int &mxx, int &mxy)
{
    mnx = mny = INT_MAX;
    mxx = mxy = INT_MIN;
#pragma unroll
    for (int k = 0; k < Cfg::PPT; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jx = target_x<Cfg>(x0, h), jy = target_y<Cfg>(y0, k);
            float2 s = make_float2((float)jx, (float)jy);
            if (jx < a.n0 && jy < ylim) {
                s = start_point(jx, jy, dj[2 * k + h]);
                mnx = min(mnx, (int)floorf(s.x));
                mny = min(mny, (int)floorf(s.y));
                mxx = max(mxx, (int)floorf(s.x));
                mxy = max(mxy, (int)floorf(s.y));
            }
            S[(2 * k + h) * Cfg::NT + threadIdx.x] = s;
        }
    }
}

// displacements of tile t's targets into registers
template <class Cfg>
__device__ __forceinline__ void load_dj(const TileArgs &a, int x0, int y0, int ylim, float2 *dj)
{
#pragma unroll
    for (int k = 0; k < Cfg::PPT; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jx = target_x<Cfg>(x0, h), jy = target_y<Cfg>(y0, k);
            dj[2 * k + h] = (jx < a.n0 && jy < ylim)
                                ? __ldg(reinterpret_cast<const float2 *>(a.D) + ((long long)jy * a.n0 + jx))
                                : make_float2(0.f, 0.f);
        }
    }
}

// box reduction of the CTA's start elements into the window of slot p (thread 0 writes it and
// resets the box); a CTA barrier inside
template <class Cfg>
__device__ __forceinline__ void reduce_window(const R2Args &A, int mnx, int mny, int mxx, int mxy, int *box, Win2 *W,
                                              int p)
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
    if (threadIdx.x == 0) {
        W[p] = window2<Cfg>(box[0], box[1], box[2], box[3], A.t.n0, A.t.n1, A.use_tma != 0);
        box[0] = box[1] = INT_MAX;
        box[2] = box[3] = INT_MIN;
    }
}

// The fast path of one target (Sec. 2.2, eq. mapping1, Sec. 2.3, eq. multiZ), without branches:
// the refined start (one fixed-point step s <- j - D(s), D bilinear in the staged window), the
// element's vertices relative to the target, Newton from the linear part's solution with one
// iteration, the element test and the stencil sum.  This is the first hop of walk_fast2 /
// walk2w<float> when Newton converges in one iteration, so a target gets the same element,
// coordinates and value on either path.  Every shared-memory index is clamped into its buffer, so
// the whole computation runs unconditionally (two targets interleave freely); the result is valid
// unless the element or its stencil leaves the staged window, the inversion needs more than one
// iteration, meets a non-positive or nearly degenerate Jacobian, or lands outside the element --
// such a target takes the general path.
template <class Cfg, int NF>
__device__ __forceinline__ bool fast_target(const Win2 &w, int base, const float2 *sD, const float4 *sR, int jx,
                                            int jy, float2 s, bool limit, bool lin_only, float v[3], unsigned &nlin)
{
    constexpr int WX = Cfg::WX;
    // refined start
    const float fsx = floorf(s.x), fsy = floorf(s.y);
    const int cx = (int)fsx, cy = (int)fsy;
    // (a staged window is at least 9 nodes wide and high, so the unsigned bounds below do not wrap;
    // an unstaged one has extent 0 and must be excluded first)
    const bool in0 = w.mode != 0 && (unsigned)(cx - w.lox) < (unsigned)(w.wx - 1) &&
                     (unsigned)(cy - w.loy) < (unsigned)(w.wy - 1);
    const int i0 = in0 ? cy * WX + cx - base : 0;
    const float fx = s.x - fsx, fy = s.y - fsy;
    const float2 q00 = sD[i0], q10 = sD[i0 + 1], q01 = sD[i0 + WX], q11 = sD[i0 + WX + 1];
    const float bx = fmaf(fx, q10.x - q00.x, q00.x), by = fmaf(fx, q10.y - q00.y, q00.y);
    const float dx = fmaf(fy, fmaf(fx, q11.x - q01.x, q01.x) - bx, bx);
    const float dy = fmaf(fy, fmaf(fx, q11.y - q01.y, q01.y) - by, by);
    const float rx = (float)jx - dx, ry = (float)jy - dy;
    const bool near = fabsf(rx - s.x) < 4.f && fabsf(ry - s.y) < 4.f;  // false for NaN
    const int ex = near ? (int)floorf(rx) : cx, ey = near ? (int)floorf(ry) : cy;
    // the element and its stencil (nodes ex-1 .. ex+2) in the flagged part of the window
    const bool in1 = in0 && (unsigned)(ex - w.lox - 2) <= (unsigned)(w.wx - 6) &&
                     (unsigned)(ey - w.loy - 2) <= (unsigned)(w.wy - 6);
    const int e0 = in1 ? ey * WX + ex - base : WX + 1;
    const float2 d0 = sD[e0], d1 = sD[e0 + 1], d2 = sD[e0 + WX], d3 = sD[e0 + WX + 1];
    const float rx0 = (float)(ex - jx), rx1 = (float)(ex + 1 - jx);
    const float ry0 = (float)(ey - jy), ry1 = (float)(ey + 1 - jy);
    const float p0x = rx0 + d0.x, p0y = ry0 + d0.y, p1x = rx1 + d1.x, p1y = ry0 + d1.y;
    const float p2x = rx0 + d2.x, p2y = ry1 + d2.y, p3x = rx1 + d3.x, p3y = ry1 + d3.y;
    // Newton (the arithmetic of newton_solve2<float>, one iteration)
    const float ax = p1x - p0x, ay = p1y - p0y, bxx = p2x - p0x, byy = p2y - p0y;
    const float exx = p3x - p1x - p2x + p0x, eyy = p3y - p1y - p2y + p0y;
    const float det0 = ax * byy - bxx * ay;
    const float inv0 = recip_t(det0);
    float xs = -(p0x * byy - p0y * bxx) * inv0;
    float xt = -(ax * p0y - ay * p0x) * inv0;
    const float j11 = ax + xt * exx, j21 = ay + xt * eyy;
    const float j12 = bxx + xs * exx, j22 = byy + xs * eyy;
    const float st = xs * xt;
    const float gx = p0x + xs * ax + xt * bxx + st * exx;
    const float gy = p0y + xs * ay + xt * byy + st * eyy;
    const float det = j11 * j22 - j12 * j21;
    const float inv = recip_t(det);
    const float u0 = (gx * j22 - gy * j12) * inv;
    const float u1 = (j11 * gy - j21 * gx) * inv;
    xs -= u0;
    xt -= u1;
    const bool conv = det0 > 0.f && det > 0.f && fmaxf(fabsf(u0), fabsf(u1)) <= SL_NEWTON_TOL_F32;
    const bool degen = det < SL_DEGENERATE * ((fabsf(j11) + fabsf(j21)) * (fabsf(j12) + fabsf(j22)));
    const float slack = SL_SLACK_F32;
    const bool inside = xs >= -slack && xs <= 1.f + slack && xt >= -slack && xt <= 1.f + slack;
    const bool ok = in1 && conv && !degen && inside;
    // records of the stencil (a block of the buffer's first rows when the target is not valid)
    const int t0 = in1 ? (ey - 1) * WX + (ex - 1) - base : 0;
    stencil_sum<WX, NF>(sR + t0, xs, xt, limit, lin_only, v, nlin);
    return ok;
}

// Phase 4 of one tile: every target of the thread; general-path targets after the loop.
template <class Cfg, int NF>
__device__ __forceinline__ void compute_tile2(const TileArgs &a, int x0, int y0, int ylim, const Win2 &w,
                                              const float2 *sD, const float4 *sR, const float2 *S, LocalCounters &cnt)
{
    const bool limit = a.max_order >= 1 && a.thr >= 0.f;
    const bool lin_only = a.max_order == 0;
    const int base = w.loy * Cfg::WX + w.lox;
    if (w.mode == 0 && threadIdx.x == 0) cnt.fallback += 1;
    unsigned slow = 0u, nfast = 0u, nlin_sum = 0u;
    // the two targets of a tile row (both halves) together: independent work to interleave
#pragma unroll 1
    for (int k = 0; k < Cfg::PPT; ++k) {
        const int jy = target_y<Cfg>(y0, k);
        const int jxa = target_x<Cfg>(x0, 0), jxb = target_x<Cfg>(x0, 1);
        const float2 sa = S[(2 * k) * Cfg::NT + threadIdx.x], sb = S[(2 * k + 1) * Cfg::NT + threadIdx.x];
        float va[3], vb[3];
        unsigned na = 0u, nb = 0u;
        const bool oka = fast_target<Cfg, NF>(w, base, sD, sR, jxa, jy, sa, limit, lin_only, va, na);
        const bool okb = fast_target<Cfg, NF>(w, base, sD, sR, jxb, jy, sb, limit, lin_only, vb, nb);
        const bool ina = jxa < a.n0 && jy < ylim, inb = jxb < a.n0 && jy < ylim;
        const bool fa = ina && oka && w.mode != 0, fb = inb && okb && w.mode != 0;
        const long long jj = (long long)jy * a.n0 + jxa;
        const int hb = Cfg::PX;  // the second target is PX columns to the right
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (fa) a.out[f][jj] = va[f];
            if (fb) a.out[f][jj + hb] = vb[f];
        }
        nfast += (fa ? 1u : 0u) + (fb ? 1u : 0u);
        nlin_sum += (fa ? na : 0u) + (fb ? nb : 0u);
        slow |= ((ina && !fa) ? 1u : 0u) << (2 * k);
        slow |= ((inb && !fb) ? 1u : 0u) << (2 * k + 1);
    }
    // fast targets: one hop, one Newton iteration each
    cnt.targets += nfast;
    cnt.hops += nfast;
    cnt.iters += nfast;
    cnt.hops_max = max(cnt.hops_max, nfast ? 1u : 0u);
    cnt.iters_max = max(cnt.iters_max, nfast ? 1u : 0u);
    cnt.oh0 += nlin_sum;
    cnt.oh1 += NF * nfast - nlin_sum;
#pragma unroll 1
    for (int q = 0; slow != 0u; ++q, slow >>= 1) {
        if (!(slow & 1u)) continue;
        const int jx = target_x<Cfg>(x0, q & 1), jy = target_y<Cfg>(y0, q >> 1);
        const float2 s = S[q * Cfg::NT + threadIdx.x];
        int ex, ey;
        refined_start2<Cfg>(w, sD, jx, jy, s.x, s.y, ex, ey);
        const TargetOut r = slow_target2<Cfg, NF>(a, w, sD, sR, limit, jx, jy, ex, ey, (int)floorf(s.x), (int)floorf(s.y));
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

// eq. (vel): the next step's trajectories of the tile's own nodes (fused steps; the velocity is
// given, so they do not depend on the fields being remapped)
template <class Cfg>
__device__ __forceinline__ void integrate_next2(const TileArgs &a, const VelArgs<float> &vn, int x0, int y0, int ylim)
{
    if (vn.kind == SL_VEL_SWIRL2D && vn.integrator == SL_RK4 && vn.substeps == 1) {
        // the swirl: a thread's two nodes of a tile row (PX columns apart) on packed FP32x2 arithmetic
        float2 *Dn = reinterpret_cast<float2 *>(a.D_next);
#pragma unroll 1
        for (int k = 0; k < Cfg::PPT; ++k) {
            const int jxa = target_x<Cfg>(x0, 0), jxb = target_x<Cfg>(x0, 1), jy = target_y<Cfg>(y0, k);
            const bool ina = jxa < a.n0 && jy < ylim, inb = jxb < a.n0 && jy < ylim;
            if (!ina && !inb) continue;
            const float Y = node_position(vn.lo[1], jy, vn.dx[1]);
            const float2 Xp = make_float2(node_position(vn.lo[0], jxa, vn.dx[0]), node_position(vn.lo[0], jxb, vn.dx[0]));
            // (sin, cos of pi x evaluated here: reading them from the grid's table measured slower)
            float2 Dx, Dy;
            rk4_swirl_pair(vn, Xp, make_float2(Y, Y), Dx, Dy);
            const long long jj = (long long)jy * a.n0 + jxa;
            if (ina) Dn[jj] = make_float2(Dx.x, Dy.x);
            if (inb) Dn[jj + Cfg::PX] = make_float2(Dx.y, Dy.y);
        }
        return;
    }
#pragma unroll 1
    for (int q = 0; q < 2 * Cfg::PPT; ++q) {
        const int jx = target_x<Cfg>(x0, q & 1), jy = target_y<Cfg>(y0, q >> 1);
        if (jx >= a.n0 || jy >= ylim) continue;
        float X[3] = {node_position(vn.lo[0], jx, vn.dx[0]), node_position(vn.lo[1], jy, vn.dx[1]), 0.f}, d[3];
        trajectory_cells<float, 2>(vn, X, d);
        reinterpret_cast<float2 *>(a.D_next)[(long long)jy * a.n0 + jx] = make_float2(d[0], d[1]);
    }
}

// The i-th work item of CTA b: the tile's target columns x0 .. x0 + TX - 1 and rows y0 .. ylim - 1
// (ylim <= y0: no item).  Items 0 .. R-1 are the tiles b, b + G, .. (R = ntiles / G full rounds).
// The last, partial round's rem tiles are cut into 2 rem half tiles (the two row passes of a tile)
// for the CTAs 0 .. 2 rem - 1 when there are enough CTAs, so that no CTA has a whole extra tile.
struct Item2 {
    int x0, y0, ylim;
};
template <class Cfg>
__device__ __forceinline__ Item2 item2(const R2Args &A, int b, int i)
{
    const int G = (int)gridDim.x, R = A.ntiles / G, rem = A.ntiles - R * G;
    const bool split = Cfg::PPT == 2 && rem > 0 && 2 * rem <= G;
    Item2 it = {0, 0, 0};
    int t = -1, half = -1;
    if (i < R)
        t = b + i * G;
    else if (i == R && split && b < 2 * rem)
        t = R * G + (b >> 1), half = b & 1;
    else if (i == R && !split && b < rem)
        t = R * G + b;
    if (t < 0) return it;
    const int tr = t / A.tiles_x;
    it.x0 = (t - tr * A.tiles_x) * Cfg::TX;
    it.y0 = tr * Cfg::TY;
    it.ylim = min(A.t.n1, it.y0 + Cfg::TY);
    if (half >= 0) {
        // rows y0 + half ROWS .. : target_y gives the first pass exactly these rows, the second
        // pass rows at or beyond ylim
        it.y0 += half * Cfg::ROWS;
        it.ylim = min(A.t.n1, it.y0 + Cfg::ROWS);
    }
    return it;
}
__device__ __forceinline__ bool item_valid(const Item2 &it) { return it.ylim > it.y0; }

template <class Cfg, int NF, bool FUSED>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB)
    remap2d_tma_kernel(const __grid_constant__ R2Args A, const __grid_constant__ R2Maps maps, const VelArgs<float> vn)
{
    constexpr int WX = Cfg::WX, WY = Cfg::WY, TX = Cfg::TX, TY = Cfg::TY, PPT = Cfg::PPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // box copies want 128-byte aligned destinations: the launch adds 128 bytes of room
    unsigned char *const smem =
        smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    float *const stage = reinterpret_cast<float *>(smem);
    float2 *const dwin = reinterpret_cast<float2 *>(smem + Cfg::STAGE);
    float4 *const rec = reinterpret_cast<float4 *>(smem + Cfg::STAGE + Cfg::DWIN);
    float2 *const spts = reinterpret_cast<float2 *>(smem + Cfg::STAGE + Cfg::DWIN + Cfg::REC);
    __shared__ unsigned long long bar[2];
    __shared__ int box[4];
    __shared__ Win2 W[2];
    __shared__ int abort_flag;
    const TileArgs &a = A.t;
    LocalCounters cnt;
    cnt.clear();
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        box[0] = box[1] = INT_MAX;
        box[2] = box[3] = INT_MIN;
        abort_flag = 0;
    }
    __syncthreads();
    unsigned phase = 0u;  // bit p: parity of slot p's next phase
    const int b = (int)blockIdx.x;
    Item2 cur = item2<Cfg>(A, b, 0);
    float2 dj[2 * PPT];
    if (item_valid(cur)) {
        // prologue: start points and window of the first item, displacements of the second
        load_dj<Cfg>(a, cur.x0, cur.y0, cur.ylim, dj);
        int mnx, mny, mxx, mxy;
        start_points2<Cfg>(a, cur.x0, cur.y0, cur.ylim, dj, spts, mnx, mny, mxx, mxy);
        reduce_window<Cfg>(A, mnx, mny, mxx, mxy, box, W, 0);
        __syncthreads();
        stage_window2<Cfg, NF>(A, maps, W[0], stage, dwin, &bar[0]);
        __syncthreads();
        mbar_finish(W[0], &bar[0]);
        const Item2 n1 = item2<Cfg>(A, b, 1);
        if (item_valid(n1)) load_dj<Cfg>(a, n1.x0, n1.y0, n1.ylim, dj);
    }
    for (int k = 0; item_valid(cur); ++k) {
        const int p = k & 1;
        const int x0 = cur.x0, y0 = cur.y0, ylim = cur.ylim;
        const Item2 nx = item2<Cfg>(A, b, k + 1);
        const bool has_next = item_valid(nx);
        // start points of the next item (its displacements are in registers) into the box
        if (has_next) {
            int mnx, mny, mxx, mxy;
            start_points2<Cfg>(a, nx.x0, nx.y0, nx.ylim, dj, spts + (p ^ 1) * 2 * PPT * Cfg::NT, mnx, mny, mxx,
                               mxy);
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
        }
        // this tile's window
        if (threadIdx.x == 0 && !mbar_wait(&bar[p], (phase >> p) & 1u)) {
            atomicAdd(A.timeouts, 1ull);
            abort_flag = 1;
        }
        __syncthreads();  // the box is complete, the window has landed
        if (abort_flag) break;
        // the phase has completed: every thread observes it once, which orders the copies' data
        // before its own reads
        (void)mbar_test(&bar[p], (phase >> p) & 1u);
        phase ^= 1u << p;
        if (threadIdx.x == 0 && has_next) {
            W[p ^ 1] = window2<Cfg>(box[0], box[1], box[2], box[3], a.n0, a.n1, A.use_tma != 0);
            box[0] = box[1] = INT_MAX;
            box[2] = box[3] = INT_MIN;
        }
        const Win2 w = W[p];
        if (w.mode != 0) flag_pass<Cfg, NF>(w, stage, rec, a.thr, a.max_order >= 1 && a.thr >= 0.f);
        fence_proxy_async();  // the staging planes' reads before the next box copies overwrite them
        __syncthreads();
        // the staging planes are free: copy the next item's window while this one is computed
        if (has_next) {
            stage_window2<Cfg, NF>(A, maps, W[p ^ 1], stage, dwin + (p ^ 1) * WX * WY, &bar[p ^ 1]);
            const Item2 n2 = item2<Cfg>(A, b, k + 2);
            if (item_valid(n2)) load_dj<Cfg>(a, n2.x0, n2.y0, n2.ylim, dj);
        }
        if (FUSED && a.D_next != nullptr) integrate_next2<Cfg>(a, vn, x0, y0, ylim);
        compute_tile2<Cfg, NF>(a, x0, y0, ylim, w, dwin + p * WX * WY, rec, spts + p * 2 * PPT * Cfg::NT, cnt);
        __syncthreads();
        if (has_next) mbar_finish(W[p ^ 1], &bar[p ^ 1]);
        cur = nx;
    }
    flush_counters(cnt, a.counters);
}

}  // namespace
