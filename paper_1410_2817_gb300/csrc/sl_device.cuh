// sl_device.cuh -- device-side building blocks of the FSL step (arXiv:1410.2817), shared by the
// kernels of libsl.so.  Everything is templated on the arithmetic type T (double or float) and on
// the dimension DIM (2 or 3).
//
//   velocity / rk4_cells /   eq. (vel): analytic velocities, one classical RK4 step, and
//   trajectory_cells         sub-stepped RK4 or Williamson's low-storage RK3
//   newton_solve             Sec. 2.2, eq. (mapping1): inversion of the Z~0 (multilinear) map
//   zspline / zs_weights     Appendix: cardinal Z-spline basis Z~0 (hat), Z~1, Z~2
//   jump test                Sec. 2.3: |h+ - 2h + h-| > thr * max(|h+ - h|, |h - h-|)
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sl.h"

#define SL_MAX_FIELDS 8
#define SL_MAX_VEL_PARAMS 80

// ------------------------------------------------------------------------------------------------
// time factor cos(pi t / period) of the swirl and deformation flows (eq. vel), computed by the same
// operations on the host (single grids) and on the device (batches, from per-grid device times), so
// that a grid in a batch sees the very factors it sees alone
// ------------------------------------------------------------------------------------------------
// cos(pi x): a = |x - 2 rint(x / 2)| in [0, 1]; cos(pi a) = sin(pi (1/2 - a)) = -cos(pi (1 - a))
// folds it to an argument b in [0, 1/4] (both differences are exact); then the Taylor series of
// cos(pi b) through (pi b)^18 or of sin(pi b) through (pi b)^17 (first neglected terms below 1e-19)
// by Horner's rule with explicit fused multiply-adds.
__host__ __device__ inline double cospi_time(double x)
{
    const double a = fabs(x - 2.0 * rint(0.5 * x));
    const bool mid = a > 0.25 && a <= 0.75;
    const double b = a <= 0.25 ? a : (mid ? 0.5 - a : 1.0 - a);
    const double r = 3.141592653589793 * b, u = r * r;
    double p;
    if (mid) {  // sin(r) / r = sum (-1)^k u^k / (2k+1)!
        p = 1.0 / 355687428096000.0;
        p = fma(u, p, -1.0 / 1307674368000.0);
        p = fma(u, p, 1.0 / 6227020800.0);
        p = fma(u, p, -1.0 / 39916800.0);
        p = fma(u, p, 1.0 / 362880.0);
        p = fma(u, p, -1.0 / 5040.0);
        p = fma(u, p, 1.0 / 120.0);
        p = fma(u, p, -1.0 / 6.0);
        p = fma(u, p, 1.0);
        return r * p;
    }
    p = 1.0 / 6402373705728000.0;  // cos(r) = sum (-1)^k u^k / (2k)!
    p = fma(u, p, -1.0 / 20922789888000.0);
    p = fma(u, p, 1.0 / 87178291200.0);
    p = fma(u, p, -1.0 / 479001600.0);
    p = fma(u, p, 1.0 / 3628800.0);
    p = fma(u, p, -1.0 / 40320.0);
    p = fma(u, p, 1.0 / 720.0);
    p = fma(u, p, -1.0 / 24.0);
    p = fma(u, p, 0.5);
    // the last step by hand: cos = 1 - u p with the sign of the fold
    p = fma(-u, p, 1.0);
    return a <= 0.25 ? p : -p;
}

// The time factors of one step of length dt from t: sub-step s starts at t_s = t + s h, h = dt /
// substeps, its stages sit at t_s + c h with c = (0, 1/2, 1) for RK4 and (0, 1/3, 3/4) for
// Williamson's RK3; ct[3 s + k] = cos(pi (t_s + c_k h) / period).
template <typename T>
__host__ __device__ inline void stage_time_factors(double t, double dt, int substeps, int integrator, double period,
                                                   T *ct)
{
    const double h = dt / substeps;
    const bool w3 = integrator == SL_WRK3;
    const double c1 = w3 ? 1.0 / 3.0 : 0.5, c2 = w3 ? 0.75 : 1.0;
    for (int st = 0; st < substeps; ++st) {
        const double ts = fma((double)st, h, t);
        ct[3 * st + 0] = (T)cospi_time(ts / period);
        ct[3 * st + 1] = (T)cospi_time(fma(c1, h, ts) / period);
        ct[3 * st + 2] = (T)cospi_time(fma(c2, h, ts) / period);
    }
}

// ------------------------------------------------------------------------------------------------
// argument blocks (passed by value)
// ------------------------------------------------------------------------------------------------
struct DevCounters {
    unsigned long long targets, fail_locate, fail_newton, fail_fold;
    unsigned long long hops_sum, hops_max, iters_sum, iters_max;
    unsigned long long newton_f64, order_hist[3], tiles_fallback;
    unsigned long long timeouts;  // bounded waits on shared-memory copies that ran out
};

template <typename T>
struct VelArgs {
    int kind;
    int nmodes;
    int integrator;   // SL_RK4 or SL_WRK3
    int substeps;     // integrator steps of dt / substeps per step (1 .. SL_MAX_SUBSTEPS)
    T p[SL_MAX_VEL_PARAMS];
    // cos(pi t/T) at the stage times of sub-step s in ct[3 s + 0..2] (time-dependent flows):
    // RK4 t_s, t_s + h/2, t_s + h; WRK3 t_s, t_s + h/3, t_s + 3h/4 (h = dt / substeps)
    T ct[3 * SL_MAX_SUBSTEPS];
    T lo[3], dx[3], inv_dx[3];
    T dt;
    // sin(pi x), cos(pi x) at the grid's node coordinates x = lo + k dx of each axis (pairs, node k
    // at 2k), tabulated once per grid for the swirl and the deformation flow; null otherwise
    const T *sc[3];
};

template <typename T>
struct GridArgs {
    int n[3];
    long long N;
    int nfields;
    int max_order;
    T threshold;
    int newton_max_iter;
    int walk_max;
    int walk_start;
    T tol;    // Newton stop rule on max |dxi|
    T slack;  // face tolerance of the element test
};

enum { ST_OK = 0, ST_LOCATE = 1, ST_NEWTON = 2, ST_FOLD = 3 };

// ------------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------------
// periodic index: a compare and select for the common case, a modulo only for k outside [0, n)
__device__ __forceinline__ int wrap_idx(int k, int n)
{
    if ((unsigned)k < (unsigned)n) return k;
    int r = k % n;
    return r < 0 ? r + n : r;
}

// periodic index for k in [-n, 2n) only (callers guarantee the range): compares and one add
__device__ __forceinline__ int wrap_near(int k, int n)
{
    return k < 0 ? k + n : (k >= n ? k - n : k);
}

// Type-exact math: a float argument must never reach a double overload (GB300 runs FP64 at a
// small fraction of its FP32 rate, so one stray conversion per tap or iteration dominates).
__device__ __forceinline__ float abs_t(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_t(double x) { return fabs(x); }
__device__ __forceinline__ float max_t(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double max_t(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float min_t(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double min_t(double a, double b) { return fmin(a, b); }
// finite: false for NaN and +-Inf, without the generic isfinite()
__device__ __forceinline__ bool finite_t(float x) { return fabsf(x) <= 3.40282346638528859812e+38f; }
__device__ __forceinline__ bool finite_t(double x) { return fabs(x) <= 1.79769313486231570815e+308; }

// 1/x: the FP32 paths take the approximate hardware reciprocal (Newton converges to the root of
// x(xi) = 0 whatever the last bits of J^-1 are), FP64 keeps the IEEE division
// FP32: the hardware's approximate reciprocal (within a few ulp; denormals flush to zero).  The
// Newton step tolerance is far above its error, and a determinant that small is degenerate anyway.
__device__ __forceinline__ float recip_t(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double recip_t(double x) { return 1.0 / x; }

__device__ __forceinline__ void sincospi_t(double x, double *s, double *c) { sincospi(x, s, c); }
// FP32 sin(pi x), cos(pi x): x = q/2 + r with q = rint(2x) and |r| <= 1/4 (both exact), the Taylor
// series of sin(pi r) through r^9 and of cos(pi r) through r^10 (truncation below 2e-9 for
// |pi r| <= pi/4) by Horner's rule in r^2, then the quadrant q mod 4.  Integers and half-integers
// give exact zeros (stagnation lines stay at rest).  Valid for |x| < 2^30.
// (-1)^k pi^(2k+1) / (2k+1)!, k = 4 .. 0, and (-1)^k pi^(2k) / (2k)!, k = 5 .. 1
struct SinPiF32 {
    static constexpr float s4 = 8.214588661e-2f, s3 = -5.992645293e-1f, s2 = 2.550164040e+0f, s1 = -5.167712780e+0f,
                           s0 = 3.141592654e+0f;
    static constexpr float c5 = -2.580689139e-2f, c4 = 2.353306304e-1f, c3 = -1.335262769e+0f, c2 = 4.058712126e+0f,
                           c1 = -4.934802201e+0f;
};

__device__ __forceinline__ void sincospi_t(float x, float *s, float *c)
{
    const float q = rintf(2.f * x);
    const float r = fmaf(-0.5f, q, x);
    const float u = r * r;
    typedef SinPiF32 K;
    float sn = r * fmaf(u, fmaf(u, fmaf(u, fmaf(u, K::s4, K::s3), K::s2), K::s1), K::s0);
    float cs = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, K::c5, K::c4), K::c3), K::c2), K::c1), 1.f);
    const int qi = (int)q;
    if (qi & 1) {
        const float t = sn;
        sn = cs;
        cs = -t;
    }
    if (qi & 2) {
        sn = -sn;
        cs = -cs;
    }
    *s = sn;
    *c = cs;
}

template <typename T>
__device__ __forceinline__ T floor_t(T x);
template <>
__device__ __forceinline__ double floor_t<double>(double x) { return floor(x); }
template <>
__device__ __forceinline__ float floor_t<float>(float x) { return floorf(x); }

// ------------------------------------------------------------------------------------------------
// eq. (vel): velocity fields of the workloads at an unwrapped physical position
// ------------------------------------------------------------------------------------------------
template <typename T, int DIM>
__device__ __forceinline__ void velocity(const VelArgs<T> &v, const T x[3], int stage, T u[3])
{
    const T two = T(2);
    u[0] = u[1] = u[2] = T(0);
    switch (v.kind) {
    case SL_VEL_UNIFORM:
        for (int a = 0; a < DIM; ++a) u[a] = v.p[a];
        break;
    case SL_VEL_SOLID_BODY:
        u[0] = v.p[0] * (v.p[2] - x[1]);
        u[1] = v.p[0] * (x[0] - v.p[1]);
        break;
    case SL_VEL_SWIRL2D: {
        T sx, cx, sy, cy;
        sincospi_t(x[0], &sx, &cx);
        sincospi_t(x[1], &sy, &cy);
        const T ct = v.ct[stage];
        u[0] = sx * sx * (two * sy * cy) * ct;   // sin(2 pi y) = 2 sin(pi y) cos(pi y)
        u[1] = -(sy * sy) * (two * sx * cx) * ct;
        break;
    }
    case SL_VEL_DEFORM3D: {
        T sx, cx, sy, cy, sz, cz;
        sincospi_t(x[0], &sx, &cx);
        sincospi_t(x[1], &sy, &cy);
        sincospi_t(x[2], &sz, &cz);
        const T ct = v.ct[stage];
        const T s2x = two * sx * cx, s2y = two * sy * cy, s2z = two * sz * cz;
        u[0] = two * sx * sx * s2y * s2z * ct;
        u[1] = -(sy * sy) * s2z * s2x * ct;
        u[2] = -(sz * sz) * s2x * s2y * ct;
        break;
    }
    case SL_VEL_FOURIER2D: {
        const T twopi = T(6.283185307179586476925286766559);
        for (int q = 0; q < v.nmodes; ++q) {
            const T *m = v.p + 1 + 4 * q;
            T s, c;
            sincospi_t(two * (m[0] * x[0] + m[1] * x[1]), &s, &c);
            const T dpsi = twopi * (m[3] * c - m[2] * s);
            u[0] += m[1] * dpsi;
            u[1] -= m[0] * dpsi;
        }
        break;
    }
    case SL_VEL_FOURIER3D: {
        const T twopi = T(6.283185307179586476925286766559);
        for (int q = 0; q < v.nmodes; ++q) {
            const T *m = v.p + 1 + 9 * q;
            T s, c;
            sincospi_t(two * (m[0] * x[0] + m[1] * x[1] + m[2] * x[2]), &s, &c);
            // k x b and k x a
            const T kb0 = m[1] * m[8] - m[2] * m[7], kb1 = m[2] * m[6] - m[0] * m[8], kb2 = m[0] * m[7] - m[1] * m[6];
            const T ka0 = m[1] * m[5] - m[2] * m[4], ka1 = m[2] * m[3] - m[0] * m[5], ka2 = m[0] * m[4] - m[1] * m[3];
            u[0] += twopi * (c * kb0 - s * ka0);
            u[1] += twopi * (c * kb1 - s * ka1);
            u[2] += twopi * (c * kb2 - s * ka2);
        }
        break;
    }
    default:
        break;
    }
}

// One classical RK4 step of eq. (vel) from the reference position X over [t, t + dt]; returns the
// displacement in cell units.
template <typename T, int DIM>
__device__ __forceinline__ void rk4_cells(const VelArgs<T> &v, const T X[3], T out[3]);

// eq. (vel) over [t, t + dt] from the reference position X with `substeps` steps of h = dt/substeps
// of classical RK4 or of Williamson's low-storage RK3 (two registers per component: q, e):
//   q <- A_k q + h u(X + e, t_s + c_k h),  e <- e + B_k q,  A = (0, -5/9, -153/128),
//   B = (1/3, 15/16, 8/15), c = (0, 1/3, 3/4);
// returns the displacement e in cell units.  The displacement, not the position, is accumulated:
// in FP32 a position near 1 would round every update to ~6e-8 of the box.  One RK4 step is
// rk4_cells itself.
template <typename T, int DIM>
__device__ __forceinline__ void trajectory_cells(const VelArgs<T> &v, const T X[3], T out[3])
{
    if (v.integrator == SL_RK4 && v.substeps == 1) {
        rk4_cells<T, DIM>(v, X, out);
        return;
    }
    const T h = v.dt / T(v.substeps);
    T e[3] = {T(0), T(0), T(0)}, y[3] = {X[0], X[1], X[2]}, k[3];
    for (int st = 0; st < v.substeps; ++st) {
        if (v.integrator == SL_WRK3) {
            T q[3];
#pragma unroll
            for (int a = 0; a < DIM; ++a) y[a] = X[a] + e[a];
            velocity<T, DIM>(v, y, 3 * st + 0, k);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                q[a] = h * k[a];
                e[a] += T(1.0 / 3.0) * q[a];
                y[a] = X[a] + e[a];
            }
            velocity<T, DIM>(v, y, 3 * st + 1, k);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                q[a] = T(-5.0 / 9.0) * q[a] + h * k[a];
                e[a] += T(15.0 / 16.0) * q[a];
                y[a] = X[a] + e[a];
            }
            velocity<T, DIM>(v, y, 3 * st + 2, k);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                q[a] = T(-153.0 / 128.0) * q[a] + h * k[a];
                e[a] += T(8.0 / 15.0) * q[a];
            }
        } else {
            T k1[3], k2[3], k3[3];
            const T hh = T(0.5) * h;
#pragma unroll
            for (int a = 0; a < DIM; ++a) y[a] = X[a] + e[a];
            velocity<T, DIM>(v, y, 3 * st + 0, k1);
#pragma unroll
            for (int a = 0; a < DIM; ++a) y[a] = X[a] + (e[a] + hh * k1[a]);
            velocity<T, DIM>(v, y, 3 * st + 1, k2);
#pragma unroll
            for (int a = 0; a < DIM; ++a) y[a] = X[a] + (e[a] + hh * k2[a]);
            velocity<T, DIM>(v, y, 3 * st + 1, k3);
#pragma unroll
            for (int a = 0; a < DIM; ++a) y[a] = X[a] + (e[a] + h * k3[a]);
            velocity<T, DIM>(v, y, 3 * st + 2, k);
#pragma unroll
            for (int a = 0; a < DIM; ++a) e[a] += h / T(6) * (k1[a] + T(2) * k2[a] + T(2) * k3[a] + k[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) out[a] = e[a] * v.inv_dx[a];
    if (DIM == 2) out[2] = T(0);
}

// a * b + c with one rounding, and a * b rounded alone (never contracted into a neighbouring add):
// the trajectories below are inlined into several kernels, and each must round them the same way
__device__ __forceinline__ float fma_rn_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn_t(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn_t(double a, double b) { return __dmul_rn(a, b); }

// physical position lo + k dx of node k along one axis (one rounding, the same in every kernel)
template <typename T>
__device__ __forceinline__ T node_position(T lo, int k, T dx) { return fma_rn_t(T(k), dx, lo); }

// sin(pi d), cos(pi d) of a small offset d from their Taylor series in r = pi d by Horner's rule
// in u = r^2, with fewer terms for the smallest offsets (the first neglected term relative to the
// result in brackets):
//   FP64, |d| <= 1/256 (|r| <= 0.0123): sin through r^7, cos through r^6 [1e-20];
//   FP64, |d| <= 1/16  (|r| <= 0.2):    sin through r^11, cos through r^12 [1e-19];
//   FP32, |d| <= 1/256: sin through r^3, cos through r^2 [1e-9];
//   FP32, |d| <= 1/8   (|r| <= 0.4):    sin through r^7, cos through r^8 [1e-9].
template <typename T>
__device__ __forceinline__ T small_offset_limit();
template <>
__device__ __forceinline__ double small_offset_limit<double>() { return 1.0 / 16.0; }
template <>
__device__ __forceinline__ float small_offset_limit<float>() { return 0.125f; }

__device__ __forceinline__ void sincospi_small(double d, double *s, double *c)
{
    const double r = mul_rn_t(3.141592653589793238462643, d), u = mul_rn_t(r, r);
    double ps, pc;
    if (fabs(d) <= 1.0 / 256.0) {
        ps = fma_rn_t(u, -1.0 / 5040.0, 1.0 / 120.0);
        pc = fma_rn_t(u, -1.0 / 720.0, 1.0 / 24.0);
    } else {
        ps = fma_rn_t(u, -1.0 / 39916800.0, 1.0 / 362880.0);
        pc = fma_rn_t(u, 1.0 / 479001600.0, -1.0 / 3628800.0);
        ps = fma_rn_t(u, ps, -1.0 / 5040.0);
        pc = fma_rn_t(u, pc, 1.0 / 40320.0);
        ps = fma_rn_t(u, ps, 1.0 / 120.0);
        pc = fma_rn_t(u, pc, -1.0 / 720.0);
        pc = fma_rn_t(u, pc, 1.0 / 24.0);
    }
    ps = fma_rn_t(u, ps, -1.0 / 6.0);
    pc = fma_rn_t(u, pc, -0.5);
    ps = fma_rn_t(u, ps, 1.0);
    *s = mul_rn_t(r, ps);
    *c = fma_rn_t(u, pc, 1.0);
}
__device__ __forceinline__ void sincospi_small(float d, float *s, float *c)
{
    const float r = mul_rn_t(3.14159265358979f, d), u = mul_rn_t(r, r);
    if (fabsf(d) <= 1.f / 256.f) {
        *s = mul_rn_t(r, fma_rn_t(u, -1.f / 6.f, 1.f));
        *c = fma_rn_t(u, -0.5f, 1.f);
        return;
    }
    float ps = fma_rn_t(u, -1.f / 5040.f, 1.f / 120.f), pc = fma_rn_t(u, 1.f / 40320.f, -1.f / 720.f);
    ps = fma_rn_t(u, ps, -1.f / 6.f);
    ps = fma_rn_t(u, ps, 1.f);
    pc = fma_rn_t(u, pc, 1.f / 24.f);
    pc = fma_rn_t(u, pc, -0.5f);
    *s = mul_rn_t(r, ps);
    *c = fma_rn_t(u, pc, 1.f);
}

// sin(pi (x + d)), cos(pi (x + d)) with d = h k from sx = sin(pi x), cx = cos(pi x): by the
// angle-addition formulas for a small offset d, else directly at x + h k (one rounding)
template <typename T>
__device__ __forceinline__ void sincospi_near(T sx, T cx, T x, T h, T k, T *s, T *c)
{
    const T d = mul_rn_t(h, k);
    if (abs_t(d) <= small_offset_limit<T>()) {
        T sd, cd;
        sincospi_small(d, &sd, &cd);
        *s = fma_rn_t(sx, cd, mul_rn_t(cx, sd));
        *c = fma_rn_t(cx, cd, -mul_rn_t(sx, sd));
    } else {
        sincospi_t(fma_rn_t(h, k, x), s, c);
    }
}

// The swirl and the 3-D deformation velocities of eq. (vel) (the formulas of `velocity`) from the
// sines and cosines of pi x_a, every product rounded in the order written.
template <typename T, int DIM>
__device__ __forceinline__ void trig_velocity(int kind, const T s[3], const T c[3], T ct, T u[3])
{
    const T s2x = T(2) * mul_rn_t(s[0], c[0]), s2y = T(2) * mul_rn_t(s[1], c[1]);  // sin(2 pi x_a), exact doubling
    if (kind == SL_VEL_SWIRL2D) {
        u[0] = mul_rn_t(mul_rn_t(mul_rn_t(s[0], s[0]), s2y), ct);
        u[1] = -mul_rn_t(mul_rn_t(mul_rn_t(s[1], s[1]), s2x), ct);
        u[2] = T(0);
    } else {
        const T s2z = T(2) * mul_rn_t(s[2], c[2]);
        u[0] = T(2) * mul_rn_t(mul_rn_t(mul_rn_t(mul_rn_t(s[0], s[0]), s2y), s2z), ct);
        u[1] = -mul_rn_t(mul_rn_t(mul_rn_t(mul_rn_t(s[1], s[1]), s2z), s2x), ct);
        u[2] = -mul_rn_t(mul_rn_t(mul_rn_t(mul_rn_t(s[2], s[2]), s2x), s2y), ct);
    }
}

// One classical RK4 step of eq. (vel) for the swirl or the 3-D deformation flow: the sines and
// cosines of pi X are evaluated once, those of each later stage's position X + delta from them
// (sincospi_near); the stages, times and weights are rk4_cells' own, k1 + 2 k2 + 2 k3 + k4 summed
// left to right.
template <typename T, int DIM>
__device__ __forceinline__ void rk4_trig_from(const VelArgs<T> &v, const T X[3], const T s0[3], const T c0[3],
                                             T out[3])
{
    T s[3], c[3];
    T k1[3], k2[3], k3[3], k4[3];
    const T h = v.dt, hh = T(0.5) * v.dt, h6 = v.dt / T(6);
    trig_velocity<T, DIM>(v.kind, s0, c0, v.ct[0], k1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        s[a] = s0[a];
        c[a] = c0[a];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) sincospi_near(s0[a], c0[a], X[a], hh, k1[a], &s[a], &c[a]);
    trig_velocity<T, DIM>(v.kind, s, c, v.ct[1], k2);
#pragma unroll
    for (int a = 0; a < DIM; ++a) sincospi_near(s0[a], c0[a], X[a], hh, k2[a], &s[a], &c[a]);
    trig_velocity<T, DIM>(v.kind, s, c, v.ct[1], k3);
#pragma unroll
    for (int a = 0; a < DIM; ++a) sincospi_near(s0[a], c0[a], X[a], h, k3[a], &s[a], &c[a]);
    trig_velocity<T, DIM>(v.kind, s, c, v.ct[2], k4);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const T sum = fma_rn_t(T(2), k3[a], fma_rn_t(T(2), k2[a], k1[a])) + k4[a];
        out[a] = mul_rn_t(mul_rn_t(h6, sum), v.inv_dx[a]);
    }
}

// rk4_trig_from with the sines and cosines of pi X evaluated here
template <typename T, int DIM>
__device__ __forceinline__ void rk4_trig_cells(const VelArgs<T> &v, const T X[3], T out[3])
{
    T s0[3] = {T(0), T(0), T(0)}, c0[3] = {T(1), T(1), T(1)};
#pragma unroll
    for (int a = 0; a < DIM; ++a) sincospi_t(X[a], &s0[a], &c0[a]);
    rk4_trig_from<T, DIM>(v, X, s0, c0, out);
}

// trajectory_cells for grid node j (X its position): the swirl's and the deformation flow's RK4
// step takes sin(pi X), cos(pi X) from the grid's table (the same bits sincospi_t gives; used by
// the trajectory launch, where it saves the FP64 path two sincospi per node; the fused launches
// evaluate them, which measured faster there)
template <typename T, int DIM>
__device__ __forceinline__ void trajectory_cells_node(const VelArgs<T> &v, const T X[3], const int j[3], T out[3])
{
    if (v.sc[0] != nullptr && v.integrator == SL_RK4 && v.substeps == 1 &&
        ((DIM == 2 && v.kind == SL_VEL_SWIRL2D) || (DIM == 3 && v.kind == SL_VEL_DEFORM3D))) {
        T s0[3] = {T(0), T(0), T(0)}, c0[3] = {T(1), T(1), T(1)};
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            s0[a] = __ldg(v.sc[a] + 2 * j[a]);
            c0[a] = __ldg(v.sc[a] + 2 * j[a] + 1);
        }
        rk4_trig_from<T, DIM>(v, X, s0, c0, out);
        return;
    }
    trajectory_cells<T, DIM>(v, X, out);
}

// ---- the swirl's RK4 step for two nodes at once -------------------------------------------------
// The operations of rk4_trig_cells<float, 2> lane by lane on packed FP32x2 instructions (each lane
// of __ffma2_rn / __fmul2_rn rounds as fmaf / __fmul_rn do, so that every node gets the bits the
// scalar code gives it); where the two nodes' stage offsets need different series, each lane takes
// the scalar path.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void quadrant_fix(int qi, float &sn, float &cs)
{
    if (qi & 1) {
        const float t = sn;
        sn = cs;
        cs = -t;
    }
    if (qi & 2) {
        sn = -sn;
        cs = -cs;
    }
}

__device__ __forceinline__ void sincospi_pair(float2 x, float2 *s, float2 *c)
{
    typedef SinPiF32 K;
    const float2 q = make_float2(rintf(2.f * x.x), rintf(2.f * x.y));
    const float2 r = __ffma2_rn(f2(-0.5f), q, x);
    const float2 u = __fmul2_rn(r, r);
    float2 ps = __ffma2_rn(u, f2(K::s4), f2(K::s3));
    ps = __ffma2_rn(u, ps, f2(K::s2));
    ps = __ffma2_rn(u, ps, f2(K::s1));
    ps = __ffma2_rn(u, ps, f2(K::s0));
    float2 pc = __ffma2_rn(u, f2(K::c5), f2(K::c4));
    pc = __ffma2_rn(u, pc, f2(K::c3));
    pc = __ffma2_rn(u, pc, f2(K::c2));
    pc = __ffma2_rn(u, pc, f2(K::c1));
    pc = __ffma2_rn(u, pc, f2(1.f));
    float2 sn = __fmul2_rn(r, ps), cs = pc;
    quadrant_fix((int)q.x, sn.x, cs.x);
    quadrant_fix((int)q.y, sn.y, cs.y);
    *s = sn;
    *c = cs;
}

// which series sincospi_near takes for the offset d: 0 the short one, 1 the long one, 2 none
__device__ __forceinline__ int offset_tier(float d)
{
    const float a = fabsf(d);
    return a <= 1.f / 256.f ? 0 : (a <= small_offset_limit<float>() ? 1 : 2);
}

// sincospi_near for two nodes: (sx, cx) of the base positions x, offsets d = h k
__device__ __forceinline__ void sincospi_near_pair(float2 sx, float2 cx, float2 x, float h, float2 k, float2 *s,
                                                   float2 *c)
{
    const float2 d = __fmul2_rn(f2(h), k);
    const int ta = offset_tier(d.x), tb = offset_tier(d.y);
    if (ta != tb || ta == 2) {
        sincospi_near(sx.x, cx.x, x.x, h, k.x, &s->x, &c->x);
        sincospi_near(sx.y, cx.y, x.y, h, k.y, &s->y, &c->y);
        return;
    }
    const float2 r = __fmul2_rn(f2(3.14159265358979f), d), u = __fmul2_rn(r, r);
    float2 sd, cd;
    if (ta == 0) {
        sd = __fmul2_rn(r, __ffma2_rn(u, f2(-1.f / 6.f), f2(1.f)));
        cd = __ffma2_rn(u, f2(-0.5f), f2(1.f));
    } else {
        float2 ps = __ffma2_rn(u, f2(-1.f / 5040.f), f2(1.f / 120.f));
        float2 pc = __ffma2_rn(u, f2(1.f / 40320.f), f2(-1.f / 720.f));
        ps = __ffma2_rn(u, ps, f2(-1.f / 6.f));
        ps = __ffma2_rn(u, ps, f2(1.f));
        pc = __ffma2_rn(u, pc, f2(1.f / 24.f));
        pc = __ffma2_rn(u, pc, f2(-0.5f));
        sd = __fmul2_rn(r, ps);
        cd = __ffma2_rn(u, pc, f2(1.f));
    }
    *s = __ffma2_rn(sx, cd, __fmul2_rn(cx, sd));
    *c = __ffma2_rn(cx, cd, neg2(__fmul2_rn(sx, sd)));
}

// trig_velocity<float, 2> of the swirl for two nodes
__device__ __forceinline__ void swirl_velocity_pair(float2 sX, float2 cX, float2 sY, float2 cY, float ct, float2 &u0,
                                                    float2 &u1)
{
    const float2 s2x = __fmul2_rn(f2(2.f), __fmul2_rn(sX, cX)), s2y = __fmul2_rn(f2(2.f), __fmul2_rn(sY, cY));
    u0 = __fmul2_rn(__fmul2_rn(__fmul2_rn(sX, sX), s2y), f2(ct));
    u1 = neg2(__fmul2_rn(__fmul2_rn(__fmul2_rn(sY, sY), s2x), f2(ct)));
}

// rk4_trig_cells<float, 2> for the swirl at the positions (X.x, Y.x) and (X.y, Y.y): the
// displacements in cell units, dx of the two nodes in Dx, dy in Dy
// (s0x, c0x, s0y, c0y: the sines and cosines of pi X and pi Y of the two nodes)
__device__ __forceinline__ void rk4_swirl_pair_from(const VelArgs<float> &v, float2 X, float2 Y, float2 s0x, float2 c0x,
                                                    float2 s0y, float2 c0y, float2 &Dx, float2 &Dy)
{
    const float h = v.dt, hh = 0.5f * v.dt, h6 = v.dt / 6.f;
    float2 sx, cx, sy, cy, k1x, k1y, k2x, k2y, k3x, k3y, k4x, k4y;
    swirl_velocity_pair(s0x, c0x, s0y, c0y, v.ct[0], k1x, k1y);
    sincospi_near_pair(s0x, c0x, X, hh, k1x, &sx, &cx);
    sincospi_near_pair(s0y, c0y, Y, hh, k1y, &sy, &cy);
    swirl_velocity_pair(sx, cx, sy, cy, v.ct[1], k2x, k2y);
    sincospi_near_pair(s0x, c0x, X, hh, k2x, &sx, &cx);
    sincospi_near_pair(s0y, c0y, Y, hh, k2y, &sy, &cy);
    swirl_velocity_pair(sx, cx, sy, cy, v.ct[1], k3x, k3y);
    sincospi_near_pair(s0x, c0x, X, h, k3x, &sx, &cx);
    sincospi_near_pair(s0y, c0y, Y, h, k3y, &sy, &cy);
    swirl_velocity_pair(sx, cx, sy, cy, v.ct[2], k4x, k4y);
    const float2 ax = __ffma2_rn(f2(2.f), k3x, __ffma2_rn(f2(2.f), k2x, k1x));
    const float2 ay = __ffma2_rn(f2(2.f), k3y, __ffma2_rn(f2(2.f), k2y, k1y));
    const float2 sumx = make_float2(ax.x + k4x.x, ax.y + k4x.y), sumy = make_float2(ay.x + k4y.x, ay.y + k4y.y);
    Dx = __fmul2_rn(__fmul2_rn(f2(h6), sumx), f2(v.inv_dx[0]));
    Dy = __fmul2_rn(__fmul2_rn(f2(h6), sumy), f2(v.inv_dx[1]));
}

__device__ __forceinline__ void rk4_swirl_pair(const VelArgs<float> &v, float2 X, float2 Y, float2 &Dx, float2 &Dy)
{
    float2 s0x, c0x, s0y, c0y;
    sincospi_pair(X, &s0x, &c0x);
    sincospi_pair(Y, &s0y, &c0y);
    rk4_swirl_pair_from(v, X, Y, s0x, c0x, s0y, c0y, Dx, Dy);
}

template <typename T, int DIM>
__device__ __forceinline__ void rk4_cells(const VelArgs<T> &v, const T X[3], T out[3])
{
    if ((DIM == 2 && v.kind == SL_VEL_SWIRL2D) || (DIM == 3 && v.kind == SL_VEL_DEFORM3D)) {
        rk4_trig_cells<T, DIM>(v, X, out);
        return;
    }
    T k1[3], k2[3], k3[3], k4[3], y[3] = {T(0), T(0), T(0)};
    const T h = v.dt, hh = T(0.5) * v.dt;
    velocity<T, DIM>(v, X, 0, k1);
#pragma unroll
    for (int a = 0; a < DIM; ++a) y[a] = X[a] + hh * k1[a];
    velocity<T, DIM>(v, y, 1, k2);
#pragma unroll
    for (int a = 0; a < DIM; ++a) y[a] = X[a] + hh * k2[a];
    velocity<T, DIM>(v, y, 1, k3);
#pragma unroll
    for (int a = 0; a < DIM; ++a) y[a] = X[a] + h * k3[a];
    velocity<T, DIM>(v, y, 2, k4);
#pragma unroll
    for (int a = 0; a < DIM; ++a) out[a] = (h / T(6) * (k1[a] + T(2) * k2[a] + T(2) * k3[a] + k4[a])) * v.inv_dx[a];
}

// FP32 production paths: Newton stops once |dxi| <= 3e-4; with quadratic convergence the error
// left is about K * tol^2 (K = curvature / Jacobian of the element, below 1 for a non-degenerate
// element), i.e. at FP32 rounding level.  An element is re-solved in FP64 only if the FP32
// inversion failed or the element is close to degenerate (relative det below SL_DEGENERATE).
#define SL_NEWTON_TOL_F32 3e-4f
#define SL_SLACK_F32 1e-5f
#define SL_DEGENERATE 1e-3f

// ------------------------------------------------------------------------------------------------
// Sec. 2.2, eq. (mapping1): Newton inversion of the multilinear element map.
// P[v][a]: vertex v (bit a = offset along axis a) relative to the target, cell units.  The map is
// expanded about the lower corner: x(xi) = P0 + sum_a xi_a A_a + sum_{a<b} xi_a xi_b E_ab
// (+ xi_0 xi_1 xi_2 G in 3-D); Newton starts from the solution of the linear part.
// Returns ST_OK, ST_NEWTON (iteration cap) or ST_FOLD (det J <= 0); xi holds the last iterate and
// *degenerate (if given) whether the converged Jacobian's det is below SL_DEGENERATE times the
// product of its columns' 1-norms (1 for a square element, 0 for a collapsed one).
// ------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int newton_solve2(const T P[8][3], int max_iter, T tol, T xi[3], int *iters,
                                             bool *degenerate = nullptr)
{
    const T ax = P[1][0] - P[0][0], ay = P[1][1] - P[0][1];
    const T bx = P[2][0] - P[0][0], by = P[2][1] - P[0][1];
    const T ex = P[3][0] - P[1][0] - P[2][0] + P[0][0], ey = P[3][1] - P[1][1] - P[2][1] + P[0][1];
    const T px = P[0][0], py = P[0][1];
    *iters = 0;
    T det = ax * by - bx * ay;
    if (degenerate) *degenerate = true;
    if (!(det > T(0))) {
        xi[0] = xi[1] = T(NAN);
        return ST_FOLD;
    }
    T inv = recip_t(det);
    T s = -(px * by - py * bx) * inv;
    T t = -(ax * py - ay * px) * inv;
    for (int it = 1; it <= max_iter; ++it) {
        *iters = it;
        const T j11 = ax + t * ex, j21 = ay + t * ey;
        const T j12 = bx + s * ex, j22 = by + s * ey;
        const T st = s * t;
        const T fx = px + s * ax + t * bx + st * ex;
        const T fy = py + s * ay + t * by + st * ey;
        det = j11 * j22 - j12 * j21;
        if (!(det > T(0))) {
            xi[0] = s;
            xi[1] = t;
            return ST_FOLD;
        }
        inv = recip_t(det);
        const T d0 = (fx * j22 - fy * j12) * inv;
        const T d1 = (j11 * fy - j21 * fx) * inv;
        s -= d0;
        t -= d1;
        if (max_t(abs_t(d0), abs_t(d1)) <= tol) {
            xi[0] = s;
            xi[1] = t;
            if (degenerate)
                *degenerate = det < T(SL_DEGENERATE) * ((abs_t(j11) + abs_t(j21)) * (abs_t(j12) + abs_t(j22)));
            return ST_OK;
        }
    }
    xi[0] = s;
    xi[1] = t;
    return ST_NEWTON;
}

// 3x3 determinant by the first row's cofactors.  Every product and sum is rounded explicitly (as
// in the trilinear map below), so that the compiler cannot contract them differently in the
// kernels that inline this: the staged and the blocked 3-D kernels, the latter fused or not, then
// invert every element to the same bits.
template <typename T>
__device__ __forceinline__ T det3(T a00, T a01, T a02, T a10, T a11, T a12, T a20, T a21, T a22)
{
    const T m0 = fma_rn_t(a11, a22, -mul_rn_t(a12, a21));
    const T m1 = fma_rn_t(a10, a22, -mul_rn_t(a12, a20));
    const T m2 = fma_rn_t(a10, a21, -mul_rn_t(a11, a20));
    return fma_rn_t(a02, m2, fma_rn_t(-a01, m1, mul_rn_t(a00, m0)));
}

// Newton inversion of the trilinear element map (eq. mapping1 in 3-D) from the solution of its
// linear part; vertices P[v] relative to the target, v = x + 2 y + 4 z.
template <typename T>
__device__ __forceinline__ int newton_solve3(const T P[8][3], int max_iter, T tol, T xi[3], int *iters,
                                             bool *degenerate = nullptr)
{
    T A[3][3], E01[3], E02[3], E12[3], G[3], P0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P0[a] = P[0][a];
        A[a][0] = P[1][a] - P[0][a];
        A[a][1] = P[2][a] - P[0][a];
        A[a][2] = P[4][a] - P[0][a];
        E01[a] = P[3][a] - P[1][a] - P[2][a] + P[0][a];
        E02[a] = P[5][a] - P[1][a] - P[4][a] + P[0][a];
        E12[a] = P[6][a] - P[2][a] - P[4][a] + P[0][a];
        G[a] = P[7][a] - P[6][a] - P[5][a] - P[3][a] + P[1][a] + P[2][a] + P[4][a] - P[0][a];
    }
    *iters = 0;
    if (degenerate) *degenerate = true;
    T det = det3(A[0][0], A[0][1], A[0][2], A[1][0], A[1][1], A[1][2], A[2][0], A[2][1], A[2][2]);
    if (!(det > T(0))) {
        xi[0] = xi[1] = xi[2] = T(NAN);
        return ST_FOLD;
    }
    T r0 = -P0[0], r1 = -P0[1], r2 = -P0[2];
    T inv = recip_t(det);
    T s0 = mul_rn_t(det3(r0, A[0][1], A[0][2], r1, A[1][1], A[1][2], r2, A[2][1], A[2][2]), inv);
    T s1 = mul_rn_t(det3(A[0][0], r0, A[0][2], A[1][0], r1, A[1][2], A[2][0], r2, A[2][2]), inv);
    T s2 = mul_rn_t(det3(A[0][0], A[0][1], r0, A[1][0], A[1][1], r1, A[2][0], A[2][1], r2), inv);
    for (int it = 1; it <= max_iter; ++it) {
        *iters = it;
        T F[3], J[3][3];
        const T s01 = mul_rn_t(s0, s1), s02 = mul_rn_t(s0, s2), s12 = mul_rn_t(s1, s2), s012 = mul_rn_t(s01, s2);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            T f = fma_rn_t(s0, A[a][0], P0[a]);
            f = fma_rn_t(s1, A[a][1], f);
            f = fma_rn_t(s2, A[a][2], f);
            f = fma_rn_t(s01, E01[a], f);
            f = fma_rn_t(s02, E02[a], f);
            f = fma_rn_t(s12, E12[a], f);
            F[a] = fma_rn_t(s012, G[a], f);
            J[a][0] = fma_rn_t(s12, G[a], fma_rn_t(s2, E02[a], fma_rn_t(s1, E01[a], A[a][0])));
            J[a][1] = fma_rn_t(s02, G[a], fma_rn_t(s2, E12[a], fma_rn_t(s0, E01[a], A[a][1])));
            J[a][2] = fma_rn_t(s01, G[a], fma_rn_t(s1, E12[a], fma_rn_t(s0, E02[a], A[a][2])));
        }
        det = det3(J[0][0], J[0][1], J[0][2], J[1][0], J[1][1], J[1][2], J[2][0], J[2][1], J[2][2]);
        if (!(det > T(0))) {
            xi[0] = s0;
            xi[1] = s1;
            xi[2] = s2;
            return ST_FOLD;
        }
        inv = recip_t(det);
        const T d0 = mul_rn_t(det3(F[0], J[0][1], J[0][2], F[1], J[1][1], J[1][2], F[2], J[2][1], J[2][2]), inv);
        const T d1 = mul_rn_t(det3(J[0][0], F[0], J[0][2], J[1][0], F[1], J[1][2], J[2][0], F[2], J[2][2]), inv);
        const T d2 = mul_rn_t(det3(J[0][0], J[0][1], F[0], J[1][0], J[1][1], F[1], J[2][0], J[2][1], F[2]), inv);
        s0 -= d0;
        s1 -= d1;
        s2 -= d2;
        if (max_t(max_t(abs_t(d0), abs_t(d1)), abs_t(d2)) <= tol) {
            xi[0] = s0;
            xi[1] = s1;
            xi[2] = s2;
            if (degenerate) {
                T cn[3];
#pragma unroll
                for (int b = 0; b < 3; ++b) cn[b] = abs_t(J[0][b]) + abs_t(J[1][b]) + abs_t(J[2][b]);
                *degenerate = det < mul_rn_t(T(SL_DEGENERATE), mul_rn_t(mul_rn_t(cn[0], cn[1]), cn[2]));
            }
            return ST_OK;
        }
    }
    xi[0] = s0;
    xi[1] = s1;
    xi[2] = s2;
    return ST_NEWTON;
}

template <typename T, int DIM>
__device__ __forceinline__ int newton_solve(const T P[8][3], int max_iter, T tol, T xi[3], int *iters,
                                            bool *degenerate = nullptr)
{
    if (DIM == 2) return newton_solve2<T>(P, max_iter, tol, xi, iters, degenerate);
    return newton_solve3<T>(P, max_iter, tol, xi, iters, degenerate);
}

// ------------------------------------------------------------------------------------------------
// Appendix: cardinal Z-spline basis functions (piecewise form, any argument).  The quintic's three
// pieces are evaluated in the local variable of their own interval, where the Horner coefficients
// stay below 6: P1(a) on [0, 1], P2(1 + s) and P3(3 - u) with s, u in [0, 1].  (Expanded in |x|,
// the outer piece sums terms of ~350 to values of ~1e-2, which in FP32 leaves errors of ~2e-5.)
// ------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T z2_inner(T a)  // |x| = a in [0, 1]
{
    return T(1) + a * a * (T(-1.25) + a * (T(-35.0 / 12.0) + a * (T(5.25) + a * T(-25.0 / 12.0))));
}
template <typename T>
__device__ __forceinline__ T z2_middle(T s)  // |x| = 1 + s, s in [0, 1]
{
    return s * (T(-2.0 / 3.0) + s * (T(2.0 / 3.0) + s * (T(1.625) + s * (T(-8.0 / 3.0) + s * T(25.0 / 24.0)))));
}
template <typename T>
__device__ __forceinline__ T z2_outer(T u)  // |x| = 3 - u, u in [0, 1]
{
    return u * u * u * (T(7.0 / 24.0) + u * (T(-0.5) + u * T(5.0 / 24.0)));
}

template <typename T>
__device__ __forceinline__ T zspline(int m, T x)
{
    const T ax = abs_t(x);
    if (m == 0) return ax < T(1) ? T(1) - ax : T(0);
    if (m == 1) {
        const T x2 = ax * ax, x3 = x2 * ax;
        if (ax <= T(1)) return T(1) - T(2.5) * x2 + T(1.5) * x3;
        if (ax <= T(2)) return T(0.5) * (T(2) - ax) * (T(2) - ax) * (T(1) - ax);
        return T(0);
    }
    if (ax <= T(1)) return z2_inner(ax);
    if (ax <= T(2)) return z2_middle(ax - T(1));
    if (ax <= T(3)) return z2_outer(T(3) - ax);
    return T(0);
}

// Weights of the 2m+2 taps c-m .. c+m+1 at local coordinate xi (argument of tap k: m - k + xi).
// For the quintic each tap's piece is known from k, and its local variable is xi or 1 - xi.
template <typename T>
__device__ __forceinline__ void zs_weights(int m, T xi, T w[6])
{
    if (m == 2) {
        const T y = T(1) - xi;
        w[0] = z2_outer(y);
        w[1] = z2_middle(xi);
        w[2] = z2_inner(xi);
        w[3] = z2_inner(y);
        w[4] = z2_middle(y);
        w[5] = z2_outer(xi);
        return;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = (k < 2 * m + 2) ? zspline<T>(m, T(m - k) + xi) : T(0);
}

// Sec. 2.2 element search: the next element depends on the current element alone, so a walk that
// returns to an element it has already tried cycles until its hop limit and fails.  Brent's cycle
// test stops it at the first repeat: `seen` holds the element reached after 1, 2, 4, 8, ... hops
// and every later element is compared with it.  step() is called after each move and returns true
// when the walk has come back to `seen` (the caller then gives up with ST_LOCATE, the status the
// exhausted walk would return).
struct CycleCheck {
    int s0, s1, s2, power, lam;
    __device__ __forceinline__ void start(int c0, int c1, int c2)
    {
        s0 = c0;
        s1 = c1;
        s2 = c2;
        power = 1;
        lam = 0;
    }
    __device__ __forceinline__ bool step(int c0, int c1, int c2)
    {
        if (c0 == s0 && c1 == s1 && c2 == s2) return true;
        if (++lam == power) {
            s0 = c0;
            s1 = c1;
            s2 = c2;
            power <<= 1;
            lam = 0;
        }
        return false;
    }
};

// Sec. 2.3 jump test of one node along one axis.
template <typename T>
__device__ __forceinline__ bool jump_test(T hm, T h0, T hp, T thr)
{
    const T dp = hp - h0, dm = h0 - hm;
    return abs_t(dp - dm) > thr * max_t(abs_t(dp), abs_t(dm));
}

// ------------------------------------------------------------------------------------------------
// counters: warp + block aggregation, one global atomic per counter and block
// ------------------------------------------------------------------------------------------------
struct LocalCounters {
    unsigned int targets, fl, fn, ff, hops, hops_max, iters, iters_max, f64, oh0, oh1, oh2, fallback;
    __device__ __forceinline__ void clear()
    {
        targets = fl = fn = ff = hops = hops_max = iters = iters_max = f64 = oh0 = oh1 = oh2 = fallback = 0u;
    }
};

__device__ __forceinline__ unsigned int warp_sum(unsigned int v) { return __reduce_add_sync(0xffffffffu, v); }
__device__ __forceinline__ unsigned int warp_max(unsigned int v) { return __reduce_max_sync(0xffffffffu, v); }

// Must be called by every thread of the block (after its work loop).
__device__ __forceinline__ void flush_counters(const LocalCounters &c, DevCounters *g)
{
    if (g == nullptr) return;
    __shared__ unsigned long long s[13];
    if (threadIdx.x < 13) s[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned int v[13] = {warp_sum(c.targets), warp_sum(c.fl),   warp_sum(c.fn),    warp_sum(c.ff),
                          warp_sum(c.hops),    warp_max(c.hops_max), warp_sum(c.iters), warp_max(c.iters_max),
                          warp_sum(c.f64),     warp_sum(c.oh0),  warp_sum(c.oh1),   warp_sum(c.oh2),
                          warp_sum(c.fallback)};
    if ((threadIdx.x & 31) == 0) {
        for (int q = 0; q < 13; ++q) {
            if (q == 5 || q == 7)
                atomicMax(&s[q], (unsigned long long)v[q]);
            else if (v[q])
                atomicAdd(&s[q], (unsigned long long)v[q]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long *dst[13] = {&g->targets,   &g->fail_locate,   &g->fail_newton,   &g->fail_fold,
                                       &g->hops_sum,  &g->hops_max,      &g->iters_sum,     &g->iters_max,
                                       &g->newton_f64, &g->order_hist[0], &g->order_hist[1], &g->order_hist[2],
                                       &g->tiles_fallback};
        for (int q = 0; q < 13; ++q) {
            if (q == 5 || q == 7) {
                if (s[q]) atomicMax(dst[q], s[q]);
            } else if (s[q]) {
                atomicAdd(dst[q], s[q]);
            }
        }
    }
}

// Per-warp flush with no block barrier (a barrier at the end of a block costs its early warps the
// wait for its slowest target): the warp's sums and maxima go straight to global memory from lane
// 0, the rare counters only where the warp met one.  For kernels whose counters see few concurrent
// adders (the 3-D kernels add into per-SM copies).
__device__ __forceinline__ void flush_counters_warp(const LocalCounters &c, DevCounters *g)
{
    if (g == nullptr) return;
    const unsigned v[7] = {warp_sum(c.targets), warp_sum(c.hops), warp_max(c.hops_max), warp_sum(c.iters),
                           warp_max(c.iters_max), warp_sum(c.oh0), warp_sum(c.oh1)};
    const unsigned rare = c.fl | c.fn | c.ff | c.f64 | c.oh2 | c.fallback;
    const bool any_rare = __any_sync(0xffffffffu, rare != 0u);
    unsigned r[6] = {0u, 0u, 0u, 0u, 0u, 0u};
    if (any_rare) {
        r[0] = warp_sum(c.fl);
        r[1] = warp_sum(c.fn);
        r[2] = warp_sum(c.ff);
        r[3] = warp_sum(c.f64);
        r[4] = warp_sum(c.oh2);
        r[5] = warp_sum(c.fallback);
    }
    if ((threadIdx.x & 31) == 0) {
        if (v[0]) atomicAdd(&g->targets, (unsigned long long)v[0]);
        if (v[1]) atomicAdd(&g->hops_sum, (unsigned long long)v[1]);
        if (v[2]) atomicMax(&g->hops_max, (unsigned long long)v[2]);
        if (v[3]) atomicAdd(&g->iters_sum, (unsigned long long)v[3]);
        if (v[4]) atomicMax(&g->iters_max, (unsigned long long)v[4]);
        if (v[5]) atomicAdd(&g->order_hist[0], (unsigned long long)v[5]);
        if (v[6]) atomicAdd(&g->order_hist[1], (unsigned long long)v[6]);
        if (any_rare) {
            unsigned long long *dst[6] = {&g->fail_locate, &g->fail_newton, &g->fail_fold, &g->newton_f64,
                                          &g->order_hist[2], &g->tiles_fallback};
#pragma unroll
            for (int q = 0; q < 6; ++q)
                if (r[q]) atomicAdd(dst[q], (unsigned long long)r[q]);
        }
    }
}

