// sl_tile2d_z2.cuh -- the per-tile body of the 2-D FP32 kernels for the quintic Z-spline
// (m_max = 2: six taps per axis, Sec. 2.1 and the Appendix), with the order lowered 2 -> 1 -> 0
// near jumps (Sec. 2.3); used by the single-grid kernels (sl_tiled_z2.cu) and the batches.
//
// The structure is that of the cubic kernels (sl_tile2d.cuh): a CTA stages the departure window of
// its 32 x 32 targets in shared memory, computes the jump flags once per window node, and every
// target walks, inverts and sums from shared memory.  What the quintic changes: the window is two
// nodes wider (stencil c-2 .. c+3), the flags are ORed over two boxes per element -- 6 x 6 (order 2
// allowed) and 4 x 4 (order 1 allowed) -- and the tensor sums run over 6 x 6 taps, with the cubic
// and bilinear sums added only for the targets whose fields need them.
#pragma once

#include "sl_tile2d.cuh"

namespace {

typedef TileCfg<32, 32, 256, 8, 3> CfgZ;  // 32x32 targets, window up to 2304 nodes, 3 CTAs per SM

// Window of a tile from the box of its start elements: the walk slack, the quintic stencil
// (c-2 .. c+3) and the limiter's neighbours (one more node each side).
template <int WMAX>
__device__ __forceinline__ Win window_of_z2(int bx0, int by0, int bx1, int by1, int n0, int n1, bool &staged)
{
    const long long wxl = (long long)bx1 - bx0 + 2 * WALK_SLACK + 8;
    const long long wyl = (long long)by1 - by0 + 2 * WALK_SLACK + 8;
    const long long olx = (long long)bx0 - WALK_SLACK - 3, oly = (long long)by0 - WALK_SLACK - 3;
    staged = wxl > 0 && wyl > 0 && wxl <= WMAX && wyl <= WMAX && wxl * wyl <= WMAX && olx >= -n0 && oly >= -n1 &&
             olx + wxl <= 2LL * n0 && oly + wyl <= 2LL * n1;
    Win w;
    w.lox = staged ? (int)olx : 0;
    w.loy = staged ? (int)oly : 0;
    w.wx = staged ? (int)wxl : 0;
    w.wy = staged ? (int)wyl : 0;
    return w;
}

// element (rx, ry) of the window whose 6 x 6 stencil lies in the flagged interior rows/columns
__device__ __forceinline__ bool z2_inside(const Win &w, int rx, int ry)
{
    return rx >= 3 && rx <= w.wx - 5 && ry >= 3 && ry <= w.wy - 5;
}

// Z~2 weights of taps c-2 .. c+3 at local coordinate x in [0, 1] (Appendix; each tap's piece in its
// own local variable, x or 1 - x)
__device__ __forceinline__ void quintic_weights(float x, float w[6])
{
    const float y = 1.f - x;
    w[0] = z2_outer(y);
    w[1] = z2_middle(x);
    w[2] = z2_inner(x);
    w[3] = z2_inner(y);
    w[4] = z2_middle(y);
    w[5] = z2_outer(x);
}

// Shared memory of one tile: as for the cubic tiles, with two box planes: B1 (bit x of row y set
// when a flag lies among nodes x-1 .. x+2 of rows y-1 .. y+2) and B2 (nodes x-2 .. x+3 of rows
// y-2 .. y+3).
template <int NF>
struct TileSmemZ2 {
    static constexpr int WMAX = CfgZ::WMAX, MW = mask_words(WMAX);
    float2 *D;
    float4 *H;
    float2 *S;
    unsigned *M, *B1, *B2;
    __device__ __forceinline__ explicit TileSmemZ2(unsigned char *base)
    {
        D = reinterpret_cast<float2 *>(base);
        H = reinterpret_cast<float4 *>(D + WMAX);
        S = reinterpret_cast<float2 *>(H + groups(NF) * WMAX);
        M = reinterpret_cast<unsigned *>(S + CfgZ::TX * CfgZ::TY);
        B1 = M + NF * MW;
        B2 = B1 + NF * MW;
    }
};

__host__ size_t z2_smem_bytes(int nfields)
{
    return (size_t)CfgZ::WMAX * (sizeof(float2) + sizeof(float4) * (size_t)((nfields + 3) / 4)) +
           sizeof(float2) * (size_t)(CfgZ::TX * CfgZ::TY) +
           3 * sizeof(unsigned) * (size_t)nfields * (size_t)mask_words(CfgZ::WMAX);
}

// eq. (multiZ) for the fields of group G from the 6 x 6 taps starting at h (node c-2, c-2): the
// quintic sum; the cubic sum over the inner 4 x 4 taps when a field of the group takes order 1
// (cub_mask), the bilinear sum over the element's 4 vertices when one takes order 0 (lin_mask).
// Field pairs run on packed FP32x2 FMAs.
template <int NF, int G>
__device__ __forceinline__ void store_group_z2(const TileArgs &a, long long jj, const float4 *h, int stride,
                                               const float wq[2][6], float xi0, float xi1, unsigned lin_mask,
                                               unsigned cub_mask)
{
    constexpr int NC = in_group(NF, G);
    constexpr bool HI = NC > 2;
    const unsigned gm = ((1u << NC) - 1u) << (4 * G);
    const bool need1 = (cub_mask & gm) != 0u, need0 = (lin_mask & gm) != 0u;
    float wc[2][4];
    if (need1) {
        cubic_weights(xi0, wc[0]);
        cubic_weights(xi1, wc[1]);
    }
    const float2 z = make_float2(0.f, 0.f);
    const float2 u0 = bcast2(1.f - xi0), u1 = bcast2(xi0);
    float2 ql = z, qh = z, cl = z, ch = z, ll = z, lh = z;
#pragma unroll
    for (int ky = 0; ky < 6; ++ky) {
        // one row: every tap feeds the quintic sum, taps 1..4 of rows 1..4 the cubic one and taps
        // 2..3 of rows 2..3 the bilinear one
        const bool row1 = ky >= 1 && ky <= 4 && need1, row0 = (ky == 2 || ky == 3) && need0;
        float2 r = z, q = z, r1 = z, q1 = z, r0 = z, q0 = z;
#pragma unroll
        for (int kx = 0; kx < 6; ++kx) {
            const float4 t = h[kx];
            const float2 wx = bcast2(wq[0][kx]);
            r = __ffma2_rn(wx, lo2(t), r);
            if (HI) q = __ffma2_rn(wx, hi2(t), q);
            if (kx >= 1 && kx <= 4 && row1) {
                const float2 cx = bcast2(wc[0][kx - 1]);
                r1 = __ffma2_rn(cx, lo2(t), r1);
                if (HI) q1 = __ffma2_rn(cx, hi2(t), q1);
            }
            if ((kx == 2 || kx == 3) && row0) {
                const float2 lx = kx == 2 ? u0 : u1;
                r0 = __ffma2_rn(lx, lo2(t), r0);
                if (HI) q0 = __ffma2_rn(lx, hi2(t), q0);
            }
        }
        const float2 wy = bcast2(wq[1][ky]);
        ql = __ffma2_rn(wy, r, ql);
        if (HI) qh = __ffma2_rn(wy, q, qh);
        if (row1) {
            const float2 cy = bcast2(wc[1][ky - 1]);
            cl = __ffma2_rn(cy, r1, cl);
            if (HI) ch = __ffma2_rn(cy, q1, ch);
        }
        if (row0) {
            const float2 v = bcast2(ky == 2 ? 1.f - xi1 : xi1);
            ll = __ffma2_rn(v, r0, ll);
            if (HI) lh = __ffma2_rn(v, q0, lh);
        }
        h += stride;
    }
    const float qv[4] = {ql.x, ql.y, qh.x, qh.y}, cv[4] = {cl.x, cl.y, ch.x, ch.y}, lv[4] = {ll.x, ll.y, lh.x, lh.y};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int f = 4 * G + c;
        a.out[f][jj] = ((lin_mask >> f) & 1u) ? lv[c] : (((cub_mask >> f) & 1u) ? cv[c] : qv[c]);
    }
}

// order flags of element (ex, ey) from global memory: OR over its 6 x 6 stencil (b2) and over the
// inner 4 x 4 (b1)
__device__ __noinline__ uint2 box_flags_global_z2(const TileArgs &a, int ex, int ey)
{
    unsigned b1 = 0u, b2 = 0u;
    for (int q = 0; q < 36; ++q) {
        const int ox = q % 6 - 2, oy = q / 6 - 2;
        const unsigned fb = node_flags_global(a, ex + ox, ey + oy);
        b2 |= fb;
        if (ox >= -1 && ox <= 2 && oy >= -1 && oy <= 2) b1 |= fb;
    }
    return make_uint2(b1, b2);
}

// eq. (multiZ) from global memory for a target whose stencil leaves the window
__device__ __noinline__ void interp_global_z2(const TileArgs &a, long long jj, int ex, int ey, float xi0, float xi1,
                                              unsigned lin_mask, unsigned cub_mask)
{
    float wq[2][6], wc[2][4];
    quintic_weights(xi0, wq[0]);
    quintic_weights(xi1, wq[1]);
    cubic_weights(xi0, wc[0]);
    cubic_weights(xi1, wc[1]);
    for (int f = 0; f < a.nfields; ++f) {
        const float *h = a.in[f];
        float v;
        if ((lin_mask >> f) & 1u) {
            v = 0.f;
            for (int ky = 0; ky < 2; ++ky) {
                const float r = fmaf(xi0, __ldg(h + gidx(ex + 1, ey + ky, a.n0, a.n1)),
                                     (1.f - xi0) * __ldg(h + gidx(ex, ey + ky, a.n0, a.n1)));
                v = fmaf(ky ? xi1 : 1.f - xi1, r, v);
            }
        } else if ((cub_mask >> f) & 1u) {
            v = 0.f;
            for (int ky = 0; ky < 4; ++ky) {
                float r = 0.f;
                for (int kx = 0; kx < 4; ++kx) r = fmaf(wc[0][kx], __ldg(h + gidx(ex - 1 + kx, ey - 1 + ky, a.n0, a.n1)), r);
                v = fmaf(wc[1][ky], r, v);
            }
        } else {
            v = 0.f;
            for (int ky = 0; ky < 6; ++ky) {
                float r = 0.f;
                for (int kx = 0; kx < 6; ++kx) r = fmaf(wq[0][kx], __ldg(h + gidx(ex - 2 + kx, ey - 2 + ky, a.n0, a.n1)), r);
                v = fmaf(wq[1][ky], r, v);
            }
        }
        a.out[f][jj] = v;
    }
}

struct TargetOutZ2 {
    int st, hops, iters, f64, nlin, ncub;
};

// The general path of one target (out of line, rare): the walk with global reads where the window
// ends and the FP64 re-solve of a failed or nearly degenerate FP32 inversion (as for the cubic
// tiles), then orders and sums from shared memory when the element's stencil is staged and from
// global memory otherwise.  A target that still fails keeps its old values.
template <int NF>
__device__ __noinline__ TargetOutZ2 slow_target_z2(const TileArgs &a, const Win w, const float2 *sD, const float4 *sH,
                                                   const unsigned *sB1, const unsigned *sB2, bool limit, long long jj,
                                                   int jx, int jy, int ex, int ey, int c0x, int c0y)
{
    TargetOutZ2 r = {ST_OK, 0, 0, 0, 0, 0};
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
    const bool fast = z2_inside(w, rx, ry);  // false when not staged (w.wx = 0)
    unsigned b1 = 0u, b2 = 0u;
    if (limit) {
        if (fast) {
            const int nwx = (w.wx + 31) >> 5, plane = w.wy * nwx, o = ry * nwx + (rx >> 5);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                b1 |= ((sB1[f * plane + o] >> (rx & 31)) & 1u) << f;
                b2 |= ((sB2[f * plane + o] >> (rx & 31)) & 1u) << f;
            }
        } else {
            const uint2 b = box_flags_global_z2(a, ex, ey);
            b1 = b.x;
            b2 = b.y;
        }
    }
    const unsigned full = (1u << NF) - 1u, lin_mask = b1 & full, cub_mask = b2 & ~b1 & full;
    r.nlin = __popc(lin_mask);
    r.ncub = __popc(cub_mask);
    if (fast) {
        float wq[2][6];
        quintic_weights(xi0, wq[0]);
        quintic_weights(xi1, wq[1]);
        const int o = (ry - 2) * w.wx + (rx - 2);
        store_group_z2<NF, 0>(a, jj, sH + o, w.wx, wq, xi0, xi1, lin_mask, cub_mask);
        if constexpr (groups(NF) > 1)
            store_group_z2<NF, 1>(a, jj, sH + CfgZ::WMAX + o, w.wx, wq, xi0, xi1, lin_mask, cub_mask);
    } else {
        interp_global_z2(a, jj, ex, ey, xi0, xi1, lin_mask, cub_mask);
    }
    return r;
}

// Phases 3 and 4 of one quintic tile (window staged and waited for, flag plane M clear).
template <int NF>
__device__ __forceinline__ void tile_compute_z2(const TileArgs &a, int x0, int y0, const Win &w, bool staged,
                                                const TileSmemZ2<NF> &sm, LocalCounters &cnt)
{
    constexpr int TX = CfgZ::TX, NT = CfgZ::NT, ROWS = CfgZ::ROWS, TPT = CfgZ::TPT, WMAX = CfgZ::WMAX;
    constexpr int NG = groups(NF);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int n0 = a.n0, n1 = a.n1;
    const bool limit = a.thr >= 0.f;
    const int nwx = (w.wx + 31) >> 5, plane = w.wy * nwx;
    // ---- phase 3: jump flags (Sec. 2.3), then their OR over each element's 4x4 and 6x6 stencils
    if (limit) {
        flag_window<CfgZ, NF>(a, w, sm.H, sm.M, nwx, plane);
        __syncthreads();
        // rows 3 .. wy-5: the elements whose 6x6 stencil lies in the interior rows 1 .. wy-2
        const int brows = w.wy - 7;
        const float inv_b = 1.f / (float)max(brows, 1);
        for (int q = threadIdx.x; q < NF * brows; q += NT) {
            const int f = row_of(q, inv_b), y = q - f * brows + 3;
            const unsigned *m = sm.M + f * plane + (y - 2) * nwx;  // rows y-2 .. y+3
            unsigned *b1 = sm.B1 + f * plane + y * nwx;
            unsigned *b2 = sm.B2 + f * plane + y * nwx;
            unsigned p4 = 0u, p6 = 0u;
            unsigned c4 = m[nwx] | m[2 * nwx] | m[3 * nwx] | m[4 * nwx];
            unsigned c6 = c4 | m[0] | m[5 * nwx];
            for (int kw = 0; kw < nwx; ++kw) {
                const int k1 = kw + 1;
                unsigned q4 = 0u, q6 = 0u;
                if (k1 < nwx) {
                    q4 = m[nwx + k1] | m[2 * nwx + k1] | m[3 * nwx + k1] | m[4 * nwx + k1];
                    q6 = q4 | m[k1] | m[5 * nwx + k1];
                }
                b1[kw] = c4 | __funnelshift_l(p4, c4, 1) | __funnelshift_r(c4, q4, 1) | __funnelshift_r(c4, q4, 2);
                b2[kw] = c6 | __funnelshift_l(p6, c6, 1) | __funnelshift_l(p6, c6, 2) | __funnelshift_r(c6, q6, 1) |
                         __funnelshift_r(c6, q6, 2) | __funnelshift_r(c6, q6, 3);
                p4 = c4;
                c4 = q4;
                p6 = c6;
                c6 = q6;
            }
        }
        __syncthreads();
    }

    // ---- phase 4: per target: search, Newton, orders, tensor Z-spline sums ---------------------
    if (!staged && threadIdx.x == 0) cnt.fallback += 1;
    const unsigned full = (1u << NF) - 1u;
    unsigned slow = 0u;
#pragma unroll 1
    for (int k = 0; k < TPT; ++k) {
        const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
        if (jx >= n0 || jy >= n1) continue;
        const long long jj = (long long)jy * n0 + jx;
        int ex, ey;
        refined_start(w, sm.D, staged, jx, jy, sm.S[k * NT + threadIdx.x], ex, ey);
        int hops = 0, iters = 0;
        float xi0 = 0.f, xi1 = 0.f;
        bool ok = staged && walk_window(w, sm.D, a.walk_max, a.max_iter, jx, jy, ex, ey, xi0, xi1, hops, iters);
        const int rx = ex - w.lox, ry = ey - w.loy;
        ok = ok && z2_inside(w, rx, ry);
        if (ok) {
            cnt.targets += 1;
            cnt.hops += hops;
            cnt.hops_max = max(cnt.hops_max, (unsigned)hops);
            cnt.iters += iters;
            cnt.iters_max = max(cnt.iters_max, (unsigned)iters);
            // Sec. 2.3: a flag in the 6x6 stencil lowers a field to the cubic, one in the 4x4 to linear
            unsigned b1 = 0u, b2 = 0u;
            if (limit) {
                const int o = ry * nwx + (rx >> 5);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    b1 |= ((sm.B1[f * plane + o] >> (rx & 31)) & 1u) << f;
                    b2 |= ((sm.B2[f * plane + o] >> (rx & 31)) & 1u) << f;
                }
            }
            const unsigned lin_mask = b1 & full, cub_mask = b2 & ~b1 & full;
            const unsigned nlin = __popc(lin_mask), ncub = __popc(cub_mask);
            cnt.oh0 += nlin;
            cnt.oh1 += ncub;
            cnt.oh2 += NF - nlin - ncub;
            float wq[2][6];
            quintic_weights(xi0, wq[0]);
            quintic_weights(xi1, wq[1]);
            const int o = (ry - 2) * w.wx + (rx - 2);
            store_group_z2<NF, 0>(a, jj, sm.H + o, w.wx, wq, xi0, xi1, lin_mask, cub_mask);
            if constexpr (NG > 1) store_group_z2<NF, 1>(a, jj, sm.H + WMAX + o, w.wx, wq, xi0, xi1, lin_mask, cub_mask);
        } else {
            slow |= 1u << k;
        }
    }
#pragma unroll 1
    for (int k = 0; slow != 0u; ++k, slow >>= 1) {
        if (!(slow & 1u)) continue;
        const int jx = x0 + tx, jy = y0 + ty + k * ROWS;
        const long long jj = (long long)jy * n0 + jx;
        const float2 s0 = sm.S[k * NT + threadIdx.x];
        int ex, ey;
        refined_start(w, sm.D, staged, jx, jy, s0, ex, ey);
        const TargetOutZ2 r = slow_target_z2<NF>(a, w, sm.D, sm.H, sm.B1, sm.B2, limit, jj, jx, jy, ex, ey,
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
            cnt.oh1 += r.ncub;
            cnt.oh2 += NF - r.nlin - r.ncub;
        }
    }
}

// One quintic tile with origin (x0, y0), staged and computed in one pass (every thread of the CTA
// calls this; it synchronises the CTA).  FUSED: the next step's trajectories of the tile's nodes
// are integrated while the window copies are in flight.
template <int NF, bool FUSED>
__device__ __forceinline__ void process_tile_z2(const TileArgs &a, const VelArgs<float> &vn, int x0, int y0,
                                                const TileSmemZ2<NF> &sm, int *sBox, LocalCounters &cnt)
{
    constexpr int TX = CfgZ::TX, ROWS = CfgZ::ROWS, TPT = CfgZ::TPT, NT = CfgZ::NT;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    if (threadIdx.x < 4) sBox[threadIdx.x] = (threadIdx.x < 2) ? INT_MAX : INT_MIN;

    // ---- phase 1: start elements floor(j - D_j) and their bounding box ------------------------
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
    const Win w = window_of_z2<CfgZ::WMAX>(bx0, by0, bx1, by1, a.n0, a.n1, staged);

    // ---- phase 2: stage the window (copies in flight while the next step's trajectories run) --
    stage_window<CfgZ, NF>(a, w, sm.D, sm.H);
    if (a.thr >= 0.f) {
        const int nm = NF * w.wy * ((w.wx + 31) >> 5);
        for (int q = threadIdx.x; q < nm; q += NT) sm.M[q] = 0u;
    }
    if (FUSED && a.D_next != nullptr && !a.carried) integrate_next<CfgZ>(a, vn, x0, y0);
    cp_async_wait_all();
    __syncthreads();
    tile_compute_z2<NF>(a, x0, y0, w, staged, sm, cnt);
    if (FUSED && a.D_next != nullptr && a.carried) carried_next<CfgZ>(a, x0, y0);
}

}  // namespace
