// sl_nlsw.cu -- the shallow-water system on the moving nodes (Sec. 3.3, eq. nlsw, nu = 0):
//   Dh/Dt = -(1 + h) div u,   Du/Dt = -grad h - f (-u2, u1),   f = f0 x2,
// integrated over one step by the three stages of Williamson's low-storage RK3 (Sec. 2), the
// sources taken by differences on the node lattice (Sec. 2: differences on the reference grid; the
// derivative at a node of the Z-spline interpolant of order m_max: second order for m <= 1, fourth
// order for m = 2) and turned into physical derivatives through the Jacobian J = I + de/dX of the
// node positions; each node moves with its own current velocity.  The remap that follows is the
// library's ordinary one.
//
// One stage is two launches: the right-hand side (a stencil over the node values, so it cannot
// update them in place) folded into the RK registers q <- A q + dt S, then the pointwise update
// W <- W + B q of the node values and of the displacement.  The displacement is kept in cell units,
// interleaved per node: after the third stage it is the remap's D.
#include <math.h>
#include <string.h>

#include <type_traits>

#include "sl_internal.h"

namespace {

template <typename T>
struct NlswArgs {
    int n0, n1;
    long long N;
    const T *w[3];   // node values h, u1, u2 (the step's input fields at the first stage)
    T *q[3];         // RK registers of h, u1, u2
    T *D, *Dq;       // displacement and its RK register, cells, 2 per node
    T A, dt, f0, lo1, dx1;
    T inv_dx0, inv_dx1;  // 1 / dx_a (physical derivative = lattice difference / dx_a)
    T r01, r10;          // dx0 / dx1 and dx1 / dx0 (the Jacobian in cell units)
};

template <typename T2, typename T>
__device__ __forceinline__ T2 make_t2(T x, T y)
{
    T2 r;
    r.x = x;
    r.y = y;
    return r;
}

// lattice difference along one axis from the values at offsets -2 .. +2 (cell units)
template <typename T, bool FD4>
__device__ __forceinline__ T lat(T m2, T m1, T p1, T p2)
{
    if (FD4) return T(2.0 / 3.0) * (p1 - m1) - T(1.0 / 12.0) * (p2 - m2);
    return T(0.5) * (p1 - m1);
}

// Right-hand side of stage k at node i folded into the RK registers.  FIRST: the nodes sit on the
// reference grid (D = 0, J = I) and the registers start from zero.
template <typename T, bool FD4, bool FIRST>
__global__ void __launch_bounds__(256) nlsw_rhs_kernel(const NlswArgs<T> a)
{
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.N; i += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(i / a.n0), ix = (int)(i - (long long)iy * a.n0);
        const long long r = (long long)iy * a.n0;
        const int xm1 = wrap_near(ix - 1, a.n0), xp1 = wrap_near(ix + 1, a.n0);
        const int xm2 = FD4 ? wrap_near(ix - 2, a.n0) : 0, xp2 = FD4 ? wrap_near(ix + 2, a.n0) : 0;
        const long long ym1 = (long long)wrap_near(iy - 1, a.n1) * a.n0, yp1 = (long long)wrap_near(iy + 1, a.n1) * a.n0;
        const long long ym2 = FD4 ? (long long)wrap_near(iy - 2, a.n1) * a.n0 : 0;
        const long long yp2 = FD4 ? (long long)wrap_near(iy + 2, a.n1) * a.n0 : 0;
        // lattice differences along x (X) and y (Y) of plane p
        auto LX = [&](const T *p) {
            return lat<T, FD4>(FD4 ? __ldg(p + r + xm2) : T(0), __ldg(p + r + xm1), __ldg(p + r + xp1),
                               FD4 ? __ldg(p + r + xp2) : T(0));
        };
        auto LY = [&](const T *p) {
            return lat<T, FD4>(FD4 ? __ldg(p + ym2 + ix) : T(0), __ldg(p + ym1 + ix), __ldg(p + yp1 + ix),
                               FD4 ? __ldg(p + yp2 + ix) : T(0));
        };
        const T hX = LX(a.w[0]), hY = LY(a.w[0]);
        const T uX = LX(a.w[1]), uY = LY(a.w[1]);
        const T vX = LX(a.w[2]), vY = LY(a.w[2]);
        T hx, hy, div, ey = T(0);
        if (FIRST) {
            hx = hX * a.inv_dx0;
            hy = hY * a.inv_dx1;
            div = uX * a.inv_dx0 + vY * a.inv_dx1;
        } else {
            const T2 *D2 = reinterpret_cast<const T2 *>(a.D);
            auto eX = [&](long long o0, long long o1, long long o2, long long o3) {  // (ex, ey) differences
                const T2 m2 = FD4 ? D2[o0] : T2(), m1 = D2[o1], p1 = D2[o2], p2 = FD4 ? D2[o3] : T2();
                return make_t2<T2>(lat<T, FD4>(m2.x, m1.x, p1.x, p2.x), lat<T, FD4>(m2.y, m1.y, p1.y, p2.y));
            };
            const auto dX = eX(r + xm2, r + xm1, r + xp1, r + xp2);      // d(ex, ey)/dX, cells per cell
            const auto dY = eX(ym2 + ix, ym1 + ix, yp1 + ix, yp2 + ix);  // d(ex, ey)/dY
            // J_ab = delta_ab + (dx_a / dx_b) d e_a / d X_b with e in cells
            const T J00 = T(1) + dX.x, J01 = dY.x * a.r01, J10 = dX.y * a.r10, J11 = T(1) + dY.y;
            const T rdet = T(1) / (J00 * J11 - J01 * J10);
            const T I00 = J11 * rdet, I01 = -J01 * rdet, I10 = -J10 * rdet, I11 = J00 * rdet;
            const T hXp = hX * a.inv_dx0, hYp = hY * a.inv_dx1;
            hx = I00 * hXp + I10 * hYp;
            hy = I01 * hXp + I11 * hYp;
            div = uX * a.inv_dx0 * I00 + uY * a.inv_dx1 * I10 + vX * a.inv_dx0 * I01 + vY * a.inv_dx1 * I11;
            ey = D2[i].y;
        }
        const T h = __ldg(a.w[0] + i), u = __ldg(a.w[1] + i), v = __ldg(a.w[2] + i);
        const T f = a.f0 * (a.lo1 + (T(iy) + ey) * a.dx1);
        const T S0 = -(T(1) + h) * div, S1 = -hx + f * v, S2 = -hy - f * u;
        if (FIRST) {
            a.q[0][i] = a.dt * S0;
            a.q[1][i] = a.dt * S1;
            a.q[2][i] = a.dt * S2;
            reinterpret_cast<T2 *>(a.Dq)[i] = make_t2<T2>(a.dt * u * a.inv_dx0, a.dt * v * a.inv_dx1);
        } else {
            a.q[0][i] = a.A * a.q[0][i] + a.dt * S0;
            a.q[1][i] = a.A * a.q[1][i] + a.dt * S1;
            a.q[2][i] = a.A * a.q[2][i] + a.dt * S2;
            const T2 dq = reinterpret_cast<const T2 *>(a.Dq)[i];
            reinterpret_cast<T2 *>(a.Dq)[i] =
                make_t2<T2>(a.A * dq.x + a.dt * u * a.inv_dx0, a.A * dq.y + a.dt * v * a.inv_dx1);
        }
    }
}

template <typename T>
struct NlswUpdate {
    long long N;
    int nfields;
    const T *src[SL_MAX_FIELDS];  // the step's input fields (first stage) or the node values
    T *dst[SL_MAX_FIELDS];        // the node values
    const T *q[3];
    T *D;
    const T *Dq;
    T B;
};

// W <- W + B q for h, u1, u2 and D <- D + B Dq; FIRST: W and D start from the input fields and 0
// (passive fields are copied).
template <typename T, bool FIRST>
__global__ void __launch_bounds__(256) nlsw_update_kernel(const NlswUpdate<T> a)
{
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.dst[c][i] = a.src[c][i] + a.B * a.q[c][i];
        if (FIRST)
            for (int c = 3; c < a.nfields; ++c) a.dst[c][i] = a.src[c][i];
        const T2 dq = reinterpret_cast<const T2 *>(a.Dq)[i];
        T2 d = FIRST ? make_t2<T2>(T(0), T(0)) : reinterpret_cast<const T2 *>(a.D)[i];
        d.x += a.B * dq.x;
        d.y += a.B * dq.y;
        reinterpret_cast<T2 *>(a.D)[i] = d;
    }
}

}  // namespace

template <typename T>
cudaError_t Launch<T>::nlsw_stages(const sl_grid *g, const void *const *fields, void *const *nodes, void *D, void *Dq,
                                   double dt, cudaStream_t s)
{
    const double A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0}, B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    const long long N = g->N;
    T *rk = (T *)g->rk;
    NlswArgs<T> ra;
    memset(&ra, 0, sizeof(ra));
    ra.n0 = (int)g->n[0];
    ra.n1 = (int)g->n[1];
    ra.N = N;
    for (int c = 0; c < 3; ++c) ra.q[c] = rk + (long long)c * N;
    ra.D = (T *)D;
    ra.Dq = (T *)Dq;
    ra.dt = (T)dt;
    ra.f0 = (T)g->vel_params[0];
    ra.lo1 = (T)g->desc.lo[1];
    ra.dx1 = (T)g->dx[1];
    ra.inv_dx0 = (T)(1.0 / g->dx[0]);
    ra.inv_dx1 = (T)(1.0 / g->dx[1]);
    ra.r01 = (T)(g->dx[0] / g->dx[1]);
    ra.r10 = (T)(g->dx[1] / g->dx[0]);
    NlswUpdate<T> ua;
    memset(&ua, 0, sizeof(ua));
    ua.N = N;
    ua.nfields = g->nfields;
    for (int c = 0; c < g->nfields; ++c) ua.dst[c] = (T *)nodes[c];
    for (int c = 0; c < 3; ++c) ua.q[c] = rk + (long long)c * N;
    ua.D = (T *)D;
    ua.Dq = (const T *)Dq;
    const bool fd4 = g->desc.max_order >= 2;
    const int blocks = grid_stride_blocks(g, N, 256);
    for (int k = 0; k < 3; ++k) {
        const bool first = k == 0;
        for (int c = 0; c < 3; ++c) ra.w[c] = (const T *)(first ? fields[c] : nodes[c]);
        ra.A = (T)A[k];
        if (first) {
            if (fd4) nlsw_rhs_kernel<T, true, true><<<blocks, 256, 0, s>>>(ra);
            else nlsw_rhs_kernel<T, false, true><<<blocks, 256, 0, s>>>(ra);
        } else {
            if (fd4) nlsw_rhs_kernel<T, true, false><<<blocks, 256, 0, s>>>(ra);
            else nlsw_rhs_kernel<T, false, false><<<blocks, 256, 0, s>>>(ra);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        for (int c = 0; c < g->nfields; ++c) ua.src[c] = (const T *)(first ? fields[c] : nodes[c]);
        ua.B = (T)B[k];
        if (first) nlsw_update_kernel<T, true><<<blocks, 256, 0, s>>>(ua);
        else nlsw_update_kernel<T, false><<<blocks, 256, 0, s>>>(ua);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t Launch<float>::nlsw_stages(const sl_grid *, const void *const *, void *const *, void *, void *,
                                                double, cudaStream_t);
template cudaError_t Launch<double>::nlsw_stages(const sl_grid *, const void *const *, void *const *, void *, void *,
                                                 double, cudaStream_t);
