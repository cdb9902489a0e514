// sl_nlsw.cu -- the shallow-water system on the moving nodes (Sec. 3.3, eq. nlsw):
//   Dh/Dt = -(1 + h) div u,
//   Du/Dt = -grad h - f (-u2, u1) + nu div[(1 + h)(grad u + grad u^T)],   f = f0 x2,
// integrated over one step by the three stages of Williamson's low-storage RK3 (Sec. 2), the
// sources taken by differences on the node lattice (Sec. 2: differences on the reference grid; the
// derivative at a node of the Z-spline interpolant of order m_max: second order for m <= 1, fourth
// order for m = 2) and turned into physical derivatives through the Jacobian J = I + de/dX of the
// node positions; each node moves with its own current velocity.  The remap that follows is the
// library's ordinary one.
//
// A step is four launches.  The first computes the sources of the input fields into the RK
// registers, q <- dt S(W_0); each of the next two forms the node values of its stage on the fly,
// W_k = W_{k-1} + B_{k-1} q at every point of its stencil, writes them out and folds its own sources
// in, q <- A_k q + dt S(W_k) (the registers and node values alternate between two buffers, since a
// stencil kernel cannot update what its neighbours still read); the last applies W_3 = W_2 + B_2 q.
// The displacement (cell units, interleaved per node) and its register follow the same pattern;
// after the last launch it is the remap's D.  With viscosity each stage is preceded by a launch that
// writes the stress tau = (1 + h)(grad u + grad u^T) of the stage's node values at every node; the
// stage takes its divergence by the same differences.
#include <math.h>
#include <string.h>

#include <type_traits>

#include "sl_internal.h"

namespace {

template <typename T2, typename T>
__device__ __forceinline__ T2 make_t2(T x, T y)
{
    T2 r;
    r.x = x;
    r.y = y;
    return r;
}

// rounded products that the compiler may not fuse into a following subtraction: the displacement
// of stage 1 is a pure product B dq, and a difference of two such products contracted to
// fma(B, dq1, -B dq2) would leave the rounding residual of the second (a spurious ~1e-20 slope
// of a displacement that is constant along the axis)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// lattice difference along one axis from the values at offsets -2 .. +2 (cell units)
template <typename T, bool FD4>
__device__ __forceinline__ T lat(T m2, T m1, T p1, T p2)
{
    if (FD4) return T(2.0 / 3.0) * (p1 - m1) - T(1.0 / 12.0) * (p2 - m2);
    return T(0.5) * (p1 - m1);
}

template <typename T>
struct NlswStage {
    int n0, n1, nfields;
    long long N;
    const T *wp[SL_MAX_FIELDS];  // node values of the previous stage (the input fields at stage 0)
    const T *qp[3];              // RK registers of the previous stage (unused at stage 0)
    const T *ep, *dqp;           // displacement and its register, previous stage (cells, 2 per node)
    T *qn[3];                    // RK registers of this stage
    T *dqn;                      // displacement register of this stage
    T *wn[SL_MAX_FIELDS];        // node values of this stage (stages 1, 2)
    T *en;                       // displacement of this stage (stages 1, 2)
    T *tau[3];                   // stress of this stage's node values: tau11, tau12, tau22
    T A, Bp, dt, f0, nu, lo1, dx1;
    T inv_dx0, inv_dx1;  // 1 / dx_a (physical derivative = lattice difference / dx_a)
    T r01, r10;          // dx0 / dx1 and dx1 / dx0 (the Jacobian in cell units)
};

// The stencil of node i in stage K: node values W_K and displacements e_K formed on the fly, their
// lattice differences, and the inverse Jacobian of the node positions.
template <typename T, bool FD4, int K>
struct StageStencil {
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const NlswStage<T> &a;
    long long i, r, ym1, yp1, ym2, yp2;
    int ix, iy, xm1, xp1, xm2, xp2;
    __device__ __forceinline__ StageStencil(const NlswStage<T> &a_, long long i_) : a(a_), i(i_)
    {
        iy = (int)(i / a.n0);
        ix = (int)(i - (long long)iy * a.n0);
        r = (long long)iy * a.n0;
        xm1 = wrap_near(ix - 1, a.n0);
        xp1 = wrap_near(ix + 1, a.n0);
        xm2 = FD4 ? wrap_near(ix - 2, a.n0) : 0;
        xp2 = FD4 ? wrap_near(ix + 2, a.n0) : 0;
        ym1 = (long long)wrap_near(iy - 1, a.n1) * a.n0;
        yp1 = (long long)wrap_near(iy + 1, a.n1) * a.n0;
        ym2 = FD4 ? (long long)wrap_near(iy - 2, a.n1) * a.n0 : 0;
        yp2 = FD4 ? (long long)wrap_near(iy + 2, a.n1) * a.n0 : 0;
    }
    // node value of field c at node o in this stage
    __device__ __forceinline__ T W(int c, long long o) const
    {
        const T w = __ldg(a.wp[c] + o);
        return K == 0 ? w : w + a.Bp * __ldg(a.qp[c] + o);
    }
    // displacement at node o in this stage (cells)
    __device__ __forceinline__ T2 E(long long o) const
    {
        const T2 dq = reinterpret_cast<const T2 *>(a.dqp)[o];
        if (K == 1) return make_t2<T2>(mul_rn(a.Bp, dq.x), mul_rn(a.Bp, dq.y));
        const T2 e = reinterpret_cast<const T2 *>(a.ep)[o];
        return make_t2<T2>(e.x + a.Bp * dq.x, e.y + a.Bp * dq.y);
    }
    __device__ __forceinline__ T LX(int c) const
    {
        return lat<T, FD4>(FD4 ? W(c, r + xm2) : T(0), W(c, r + xm1), W(c, r + xp1), FD4 ? W(c, r + xp2) : T(0));
    }
    __device__ __forceinline__ T LY(int c) const
    {
        return lat<T, FD4>(FD4 ? W(c, ym2 + ix) : T(0), W(c, ym1 + ix), W(c, yp1 + ix), FD4 ? W(c, yp2 + ix) : T(0));
    }
    // lattice differences of a plain plane p (the stress)
    __device__ __forceinline__ T PX(const T *p) const
    {
        return lat<T, FD4>(FD4 ? __ldg(p + r + xm2) : T(0), __ldg(p + r + xm1), __ldg(p + r + xp1),
                           FD4 ? __ldg(p + r + xp2) : T(0));
    }
    __device__ __forceinline__ T PY(const T *p) const
    {
        return lat<T, FD4>(FD4 ? __ldg(p + ym2 + ix) : T(0), __ldg(p + ym1 + ix), __ldg(p + yp1 + ix),
                           FD4 ? __ldg(p + yp2 + ix) : T(0));
    }
    __device__ __forceinline__ T2 ED(long long o0, long long o1, long long o2, long long o3) const
    {
        const T2 m2 = FD4 ? E(o0) : T2(), m1 = E(o1), p1 = E(o2), p2 = FD4 ? E(o3) : T2();
        return make_t2<T2>(lat<T, FD4>(m2.x, m1.x, p1.x, p2.x), lat<T, FD4>(m2.y, m1.y, p1.y, p2.y));
    }
    // inverse of J = I + de/dX (identity at stage 0): I[0..3] = (J^-1)_00, _01, _10, _11
    __device__ __forceinline__ void jacobian_inverse(T I[4]) const
    {
        if (K == 0) {
            I[0] = T(1);
            I[1] = T(0);
            I[2] = T(0);
            I[3] = T(1);
            return;
        }
        const T2 dX = ED(r + xm2, r + xm1, r + xp1, r + xp2);      // d(ex, ey)/dX, cells per cell
        const T2 dY = ED(ym2 + ix, ym1 + ix, yp1 + ix, yp2 + ix);  // d(ex, ey)/dY
        // J_ab = delta_ab + (dx_a / dx_b) d e_a / d X_b with e in cells
        const T J00 = T(1) + dX.x, J01 = dY.x * a.r01, J10 = dX.y * a.r10, J11 = T(1) + dY.y;
        const T rdet = T(1) / (J00 * J11 - J01 * J10);
        I[0] = J11 * rdet;
        I[1] = -J01 * rdet;
        I[2] = -J10 * rdet;
        I[3] = J00 * rdet;
    }
};

// The stress tau = (1 + h)(grad u + grad u^T) of stage K's node values at every node (viscosity).
template <typename T, bool FD4, int K>
__global__ void __launch_bounds__(256) nlsw_stress_kernel(const NlswStage<T> a)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.N; i += (long long)gridDim.x * blockDim.x) {
        const StageStencil<T, FD4, K> st(a, i);
        T I[4];
        st.jacobian_inverse(I);
        const T uX = st.LX(1) * a.inv_dx0, uY = st.LY(1) * a.inv_dx1;
        const T vX = st.LX(2) * a.inv_dx0, vY = st.LY(2) * a.inv_dx1;
        const T ux = I[0] * uX + I[2] * uY, uy = I[1] * uX + I[3] * uY;
        const T vx = I[0] * vX + I[2] * vY, vy = I[1] * vX + I[3] * vY;
        const T d = T(1) + st.W(0, i);
        a.tau[0][i] = d * T(2) * ux;
        a.tau[1][i] = d * (uy + vx);
        a.tau[2][i] = d * T(2) * vy;
    }
}

// Stage K of the RK3 at every node.  K = 0: the node values are the input fields and the nodes
// sit on the reference grid (D = 0, J = I).  K = 1, 2: the node values W_K = W_{K-1} + B q and
// the displacement e_K = e_{K-1} + B Dq are formed at each stencil point (e_0 = 0), written out
// at the node, and the sources of W_K are folded into the new registers.  Stage 1 also carries the
// passive fields over.
template <typename T, bool FD4, int K>
__global__ void __launch_bounds__(256) nlsw_stage_kernel(const NlswStage<T> a)
{
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.N; i += (long long)gridDim.x * blockDim.x) {
        const StageStencil<T, FD4, K> st(a, i);
        T I[4];
        st.jacobian_inverse(I);
        const T hX = st.LX(0) * a.inv_dx0, hY = st.LY(0) * a.inv_dx1;
        const T uX = st.LX(1) * a.inv_dx0, uY = st.LY(1) * a.inv_dx1;
        const T vX = st.LX(2) * a.inv_dx0, vY = st.LY(2) * a.inv_dx1;
        const T h = st.W(0, i), u = st.W(1, i), v = st.W(2, i);
        // physical derivatives: grad h = J^-T (hX, hY); div u = du/dX_b (J^-1)_b0 + dv/dX_b (J^-1)_b1
        const T hx = I[0] * hX + I[2] * hY, hy = I[1] * hX + I[3] * hY;
        const T div = uX * I[0] + uY * I[2] + vX * I[1] + vY * I[3];
        T ey = T(0);
        if (K > 0) {
            const T2 ei = st.E(i);
            ey = ei.y;
            a.wn[0][i] = h;
            a.wn[1][i] = u;
            a.wn[2][i] = v;
            reinterpret_cast<T2 *>(a.en)[i] = ei;
            if (K == 1)
                for (int c = 3; c < a.nfields; ++c) a.wn[c][i] = __ldg(a.wp[c] + i);
        }
        const T f = a.f0 * (a.lo1 + (T(st.iy) + ey) * a.dx1);
        T S0 = -(T(1) + h) * div, S1 = -hx + f * v, S2 = -hy - f * u;
        if (a.nu != T(0)) {
            // nu div tau, (div tau)_a = d tau_a0 / dx + d tau_a1 / dy
            const T aX = st.PX(a.tau[0]) * a.inv_dx0, aY = st.PY(a.tau[0]) * a.inv_dx1;
            const T bX = st.PX(a.tau[1]) * a.inv_dx0, bY = st.PY(a.tau[1]) * a.inv_dx1;
            const T cX = st.PX(a.tau[2]) * a.inv_dx0, cY = st.PY(a.tau[2]) * a.inv_dx1;
            const T t11x = I[0] * aX + I[2] * aY, t12y = I[1] * bX + I[3] * bY;
            const T t12x = I[0] * bX + I[2] * bY, t22y = I[1] * cX + I[3] * cY;
            S1 += a.nu * (t11x + t12y);
            S2 += a.nu * (t12x + t22y);
        }
        const T du = a.dt * u * a.inv_dx0, dv = a.dt * v * a.inv_dx1;
        if (K == 0) {
            a.qn[0][i] = a.dt * S0;
            a.qn[1][i] = a.dt * S1;
            a.qn[2][i] = a.dt * S2;
            reinterpret_cast<T2 *>(a.dqn)[i] = make_t2<T2>(du, dv);
        } else {
            a.qn[0][i] = a.A * __ldg(a.qp[0] + i) + a.dt * S0;
            a.qn[1][i] = a.A * __ldg(a.qp[1] + i) + a.dt * S1;
            a.qn[2][i] = a.A * __ldg(a.qp[2] + i) + a.dt * S2;
            const T2 dq = reinterpret_cast<const T2 *>(a.dqp)[i];
            reinterpret_cast<T2 *>(a.dqn)[i] = make_t2<T2>(a.A * dq.x + du, a.A * dq.y + dv);
        }
    }
}

template <typename T>
struct NlswFinal {
    long long N;
    const T *w[3], *q[3], *dq;
    T *out[3];
    T *D;  // e_2 in, the step's displacement out (cells, 2 per node)
    T B;
};

// W_3 = W_2 + B_2 q and D = e_2 + B_2 Dq (pointwise; D in place)
template <typename T>
__global__ void __launch_bounds__(256) nlsw_final_kernel(const NlswFinal<T> a)
{
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.out[c][i] = a.w[c][i] + a.B * a.q[c][i];
        const T2 dq = reinterpret_cast<const T2 *>(a.dq)[i];
        T2 d = reinterpret_cast<T2 *>(a.D)[i];
        d.x += a.B * dq.x;
        d.y += a.B * dq.y;
        reinterpret_cast<T2 *>(a.D)[i] = d;
    }
}

template <typename T, int K>
cudaError_t launch_stage(bool fd4, int blocks, const NlswStage<T> &a, cudaStream_t s)
{
    if (a.nu != T(0)) {
        if (fd4)
            nlsw_stress_kernel<T, true, K><<<blocks, 256, 0, s>>>(a);
        else
            nlsw_stress_kernel<T, false, K><<<blocks, 256, 0, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (fd4)
        nlsw_stage_kernel<T, true, K><<<blocks, 256, 0, s>>>(a);
    else
        nlsw_stage_kernel<T, false, K><<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

double nlsw_viscosity(const sl_grid *g) { return g->desc.n_velocity_params > 1 ? g->vel_params[1] : 0.0; }

int nlsw_kernels_per_step(const sl_grid *g) { return nlsw_viscosity(g) != 0.0 ? 7 : 4; }

// Buffers: F = the caller's fields (input; W_2 after stage 2), S = the scratch planes (W_1, then
// W_3 and the passive fields: the remap's input), registers qA/qB (3 planes each), DqA/DqB (2
// per node) and the stress (3 planes) in the grid's workspace, e_1 in Dalt, e_2 and the final
// displacement in D.
template <typename T>
cudaError_t Launch<T>::nlsw_stages(const sl_grid *g, const void *const *fields, void *const *nodes, void *D, void *Dalt,
                                   double dt, cudaStream_t s)
{
    const double A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0}, B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    const long long N = g->N;
    T *rk = (T *)g->rk;
    T *qA[3] = {rk, rk + N, rk + 2 * N}, *qB[3] = {rk + 3 * N, rk + 4 * N, rk + 5 * N};
    T *DqA = rk + 6 * N, *DqB = rk + 8 * N;
    T *tau = rk + 10 * N;
    NlswStage<T> a;
    memset(&a, 0, sizeof(a));
    a.n0 = (int)g->n[0];
    a.n1 = (int)g->n[1];
    a.nfields = g->nfields;
    a.N = N;
    a.dt = (T)dt;
    a.f0 = (T)g->vel_params[0];
    a.nu = (T)nlsw_viscosity(g);
    for (int c = 0; c < 3; ++c) a.tau[c] = tau + (long long)c * N;
    a.lo1 = (T)g->desc.lo[1];
    a.dx1 = (T)g->dx[1];
    a.inv_dx0 = (T)(1.0 / g->dx[0]);
    a.inv_dx1 = (T)(1.0 / g->dx[1]);
    a.r01 = (T)(g->dx[0] / g->dx[1]);
    a.r10 = (T)(g->dx[1] / g->dx[0]);
    const bool fd4 = g->desc.max_order >= 2;
    const int blocks = grid_stride_blocks(g, N, 256);
    // stage 0: sources of the input fields
    for (int c = 0; c < g->nfields; ++c) a.wp[c] = (const T *)fields[c];
    for (int c = 0; c < 3; ++c) a.qn[c] = qA[c];
    a.dqn = DqA;
    cudaError_t e = launch_stage<T, 0>(fd4, blocks, a, s);
    if (e != cudaSuccess) return e;
    // stage 1: W_1 = F + B_0 qA into S (passive fields copied), e_1 into Dalt; registers into qB
    for (int c = 0; c < 3; ++c) {
        a.qp[c] = qA[c];
        a.qn[c] = qB[c];
    }
    for (int c = 0; c < g->nfields; ++c) a.wn[c] = (T *)nodes[c];
    a.dqp = DqA;
    a.dqn = DqB;
    a.en = (T *)Dalt;
    a.A = (T)A[1];
    a.Bp = (T)B[0];
    e = launch_stage<T, 1>(fd4, blocks, a, s);
    if (e != cudaSuccess) return e;
    // stage 2: W_2 = W_1 + B_1 qB into F, e_2 into D; registers into qA
    for (int c = 0; c < 3; ++c) {
        a.wp[c] = (const T *)nodes[c];
        a.qp[c] = qB[c];
        a.qn[c] = qA[c];
        a.wn[c] = (T *)fields[c];
    }
    a.ep = (const T *)Dalt;
    a.dqp = DqB;
    a.dqn = DqA;
    a.en = (T *)D;
    a.A = (T)A[2];
    a.Bp = (T)B[1];
    e = launch_stage<T, 2>(fd4, blocks, a, s);
    if (e != cudaSuccess) return e;
    // W_3 = W_2 + B_2 qA into S, D = e_2 + B_2 DqA
    NlswFinal<T> fa;
    memset(&fa, 0, sizeof(fa));
    fa.N = N;
    for (int c = 0; c < 3; ++c) {
        fa.w[c] = (const T *)fields[c];
        fa.q[c] = qA[c];
        fa.out[c] = (T *)nodes[c];
    }
    fa.dq = DqA;
    fa.D = (T *)D;
    fa.B = (T)B[2];
    nlsw_final_kernel<T><<<blocks, 256, 0, s>>>(fa);
    return cudaGetLastError();
}

template cudaError_t Launch<float>::nlsw_stages(const sl_grid *, const void *const *, void *const *, void *, void *,
                                                double, cudaStream_t);
template cudaError_t Launch<double>::nlsw_stages(const sl_grid *, const void *const *, void *const *, void *, void *,
                                                 double, cudaStream_t);
