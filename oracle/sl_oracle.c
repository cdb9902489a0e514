/*
 * sl_oracle.c -- plain, slow, FP64 CPU statement of the forward semi-Lagrangian (FSL) step of
 * Becerra-Sagredo, Malaga & Mandujano, "Moments Preserving and high-resolution Semi-Lagrangian
 * Advection Scheme" (arXiv:1410.2817).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is checked against.
 * Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA path, and the CUDA path never calls it.
 *
 * Every function restates one passage of the paper in plain loops, in the paper's order:
 *   Sec. 2, eqs. (momento)/(vel)        transport along trajectories (classical RK4 or Williamson's
 *                                       low-storage RK3, S = 0; the velocity either given or carried
 *                                       by the nodes as transported fields, Sec. 3.2)
 *   Sec. 2.1, eq. (multiZ) + Appendix   cardinal Z-spline basis and its tensor-product sum
 *   Sec. 2.2, eq. (mapping1)            multilinear (Z0) element map, Newton inversion, element search
 *   Sec. 2.3                            jump criterion (limiter flags) and adaptive order reduction
 *   Sec. 3.1, moments definition        discrete moments m_p (Table 1)
 *   Sec. 3.3, eq. (nlsw)                shallow-water sources (pressure gradient, divergence,
 *                                       Coriolis) by finite differences on the node lattice,
 *                                       integrated with the low-storage RK3, then the remap
 *
 * Readings where the paper is silent or garbled (each is also listed with the design notes):
 *   - Z0 is not printed; it is the hat max(0, 1-|x|).
 *   - Limiter numerator |h+ - 2h + h-| is evaluated as |(h+ - h) - (h - h-)| and the ratio test
 *     "num/den > thr" as "num > thr*den" (0/0 is therefore never flagged); multi-D = OR over axes;
 *     one flag bit per field.
 *   - The element map is expanded about the cell's lower corner; the Newton start is the solution
 *     of the linear part; the stop rule is max|dxi| <= tol (default 1e-14) or max_iter (8).
 *   - Search start against the node's velocity: the element that has Lagrangian node j as a vertex
 *     on the side opposite its own step displacement (c_a = j_a - [D_j,a > 0]).  A target within
 *     `slack` of a face is accepted in the first element the walk reaches.
 *   - Order reduction is isotropic and per field: m drops while any flag lies in [c-m, c+m+1]^d.
 *   - Velocity is evaluated at unwrapped positions; sin(pi x)/cos(pi x) use an exact argument
 *     reduction so that stagnation lines give exact zeros.
 *   - Shallow water: each step starts with the nodes on the reference grid and ends with one remap;
 *     a stage's differences are taken on the node lattice (the Z-spline derivative at the nodes:
 *     second order for m_max <= 1, fourth order for m_max = 2) and made physical through the
 *     inverse Jacobian of the node positions; f = f0 x2 at the node's current position; with
 *     viscosity the stress (1 + h)(grad u + grad u^T) is formed at every node first and its
 *     divergence taken by the same differences.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see oracle.py).  Threads only split the
 * loop over independent target nodes; results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* status codes of one target (kept numerically equal to nothing outside this file) */
enum { OR_OK = 0, OR_LOCATE = 1, OR_NEWTON = 2, OR_FOLD = 3 };
/* velocity kinds */
enum { OR_VEL_UNIFORM = 0, OR_VEL_SOLID_BODY = 1, OR_VEL_SWIRL2D = 2, OR_VEL_DEFORM3D = 3,
       OR_VEL_FOURIER2D = 4, OR_VEL_FOURIER3D = 5, OR_VEL_CARRIED = 6, OR_VEL_NLSW = 7 };
/* element-search start */
enum { OR_START_PAPER = 0, OR_START_BACKWARD = 1 };
enum { OR_RK4 = 0, OR_WRK3 = 1 };

/* Grid and method parameters.  The Python wrapper mirrors this layout with ctypes. */
typedef struct {
    int dim;                  /* 2 or 3 */
    int nfields;              /* 1..8 */
    int64_t n[3];             /* nodes per axis (n[2] = 1 in 2-D) */
    double lo[3], hi[3];      /* periodic box; node i sits at lo + i*(hi-lo)/n */
    int max_order;            /* m_max: 0, 1 or 2 */
    double threshold;         /* limiter threshold (0.25 in the paper); < 0 disables */
    int vel_kind;
    int n_vel_params;
    const double *vel_params;
    int newton_max_iter;      /* 8 */
    double newton_tol;        /* 1e-14 */
    int walk_max;             /* 64 */
    double slack;             /* 1e-12: face tolerance of the element test */
    int start_mode;           /* OR_START_PAPER (default) */
    int fail_keep;            /* 1: a failed target keeps its old value (also done when 0; flag only) */
    int nthreads;             /* <= 0: library default */
    int integrator;           /* OR_RK4 (classical) or OR_WRK3 (Williamson's low-storage RK3) */
    int substeps;             /* integrator steps of dt / substeps per remap (<= 1: one)      */
} or_grid;

/* ------------------------------------------------------------------------------------------ */
/* helpers                                                                                      */
/* ------------------------------------------------------------------------------------------ */

static int64_t wrap_index(int64_t k, int64_t n)
{
    int64_t r = k % n;
    return r < 0 ? r + n : r;
}

static int64_t total_nodes(const or_grid *g)
{
    int64_t N = 1;
    for (int a = 0; a < g->dim; ++a) N *= g->n[a];
    return N;
}

/* linear node index of the (possibly unwrapped) integer vector k; x fastest */
static int64_t node_index(const or_grid *g, const int64_t k[3])
{
    int64_t idx = 0, stride = 1;
    for (int a = 0; a < g->dim; ++a) {
        idx += wrap_index(k[a], g->n[a]) * stride;
        stride *= g->n[a];
    }
    return idx;
}

static void node_coords(const or_grid *g, int64_t i, int64_t k[3])
{
    k[0] = k[1] = k[2] = 0;
    for (int a = 0; a < g->dim; ++a) {
        k[a] = i % g->n[a];
        i /= g->n[a];
    }
}

static void set_threads(const or_grid *g)
{
#ifdef _OPENMP
    if (g->nthreads > 0) omp_set_num_threads(g->nthreads);
#else
    (void)g;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Appendix: cardinal Z-spline basis functions.  Z0 (not printed) is the hat function.           */
/* ------------------------------------------------------------------------------------------ */
double or_zspline(int m, double x)
{
    double ax = fabs(x);
    double x2 = ax * ax, x3 = x2 * ax, x4 = x3 * ax, x5 = x4 * ax;
    if (m == 0) {
        return ax < 1.0 ? 1.0 - ax : 0.0;
    }
    if (m == 1) { /* C1 cubic, Appendix eq. (z1) */
        if (ax <= 1.0) return 1.0 - 2.5 * x2 + 1.5 * x3;
        if (ax <= 2.0) return 0.5 * (2.0 - ax) * (2.0 - ax) * (1.0 - ax);
        return 0.0;
    }
    if (m == 2) { /* C2 quintic, Appendix */
        if (ax <= 1.0)
            return 1.0 - (15.0 / 12.0) * x2 - (35.0 / 12.0) * x3 + (63.0 / 12.0) * x4 - (25.0 / 12.0) * x5;
        if (ax <= 2.0)
            return -4.0 + (75.0 / 4.0) * ax - (245.0 / 8.0) * x2 + (545.0 / 24.0) * x3 - (63.0 / 8.0) * x4
                   + (25.0 / 24.0) * x5;
        if (ax <= 3.0)
            return 18.0 - (153.0 / 4.0) * ax + (255.0 / 8.0) * x2 - (313.0 / 24.0) * x3 + (21.0 / 8.0) * x4
                   - (5.0 / 24.0) * x5;
        return 0.0;
    }
    return NAN;
}

void or_zspline_array(int m, int64_t count, const double *x, double *out)
{
    for (int64_t i = 0; i < count; ++i) out[i] = or_zspline(m, x[i]);
}

/* ------------------------------------------------------------------------------------------ */
/* Sec. 2.3: jump criterion.  Flag bit f of node i is set when, along any axis,                 */
/* |h+ - 2h + h-| > thr * max(|h+ - h|, |h - h-|)  (periodic neighbours).                       */
/* ------------------------------------------------------------------------------------------ */
void or_flags(const or_grid *g, const double *h, uint8_t *flags)
{
    int64_t N = total_nodes(g);
    memset(flags, 0, (size_t)N);
    if (g->threshold < 0.0) return;
    set_threads(g);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int64_t k[3];
        node_coords(g, i, k);
        uint8_t bits = 0;
        for (int f = 0; f < g->nfields; ++f) {
            const double *hf = h + (int64_t)f * N;
            for (int a = 0; a < g->dim; ++a) {
                int64_t kp[3] = {k[0], k[1], k[2]}, km[3] = {k[0], k[1], k[2]};
                kp[a] += 1;
                km[a] -= 1;
                double hp = hf[node_index(g, kp)], h0 = hf[i], hm = hf[node_index(g, km)];
                double dp = hp - h0, dm = h0 - hm;
                double num = fabs(dp - dm);
                double den = fmax(fabs(dp), fabs(dm));
                if (num > g->threshold * den) bits |= (uint8_t)(1u << f);
            }
        }
        flags[i] = bits;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Velocity fields of the workloads, evaluated at unwrapped physical positions.                 */
/* sin(pi x) and cos(pi x) after an exact reduction of x to [-1, 1].                            */
/* ------------------------------------------------------------------------------------------ */
static double reduce_pi_arg(double x) /* x - 2*round(x/2), exact for |x| < 2^52 */
{
    return x - 2.0 * nearbyint(0.5 * x);
}

double or_sinpi(double x)
{
    double r = reduce_pi_arg(x);
    double s = r < 0.0 ? -1.0 : 1.0;
    double a = fabs(r);          /* a in [0, 1] */
    if (a > 0.5) a = 1.0 - a;    /* sin(pi a) = sin(pi (1 - a)); exact subtraction */
    return s * sin(M_PI * a);
}

double or_cospi(double x)
{
    double a = fabs(reduce_pi_arg(x)); /* cos is even */
    if (a <= 0.25) return cos(M_PI * a);
    if (a <= 0.75) return sin(M_PI * (0.5 - a));
    return -cos(M_PI * (1.0 - a));
}

void or_velocity(const or_grid *g, const double x[3], double t, double u[3])
{
    const double *p = g->vel_params;
    u[0] = u[1] = u[2] = 0.0;
    switch (g->vel_kind) {
    case OR_VEL_UNIFORM: /* p = (u, v[, w]) */
        for (int a = 0; a < g->dim; ++a) u[a] = p[a];
        break;
    case OR_VEL_SOLID_BODY: /* p = (Omega, cx, cy):  u = Omega * (cy - y, x - cx) */
        u[0] = p[0] * (p[2] - x[1]);
        u[1] = p[0] * (x[0] - p[1]);
        break;
    case OR_VEL_SWIRL2D: { /* p = (T): u = sin^2(pi x) sin(2 pi y) cos(pi t/T), v = -sin^2(pi y) sin(2 pi x) cos(pi t/T) */
        double ct = or_cospi(t / p[0]);
        double sx = or_sinpi(x[0]), sy = or_sinpi(x[1]);
        u[0] = sx * sx * or_sinpi(2.0 * x[1]) * ct;
        u[1] = -(sy * sy) * or_sinpi(2.0 * x[0]) * ct;
        break;
    }
    case OR_VEL_DEFORM3D: { /* p = (T): u = 2 sin^2(pi x) sin(2pi y) sin(2pi z) cos(pi t/T), v, w cyclic with -1 */
        double ct = or_cospi(t / p[0]);
        double sx = or_sinpi(x[0]), sy = or_sinpi(x[1]), sz = or_sinpi(x[2]);
        double s2x = or_sinpi(2.0 * x[0]), s2y = or_sinpi(2.0 * x[1]), s2z = or_sinpi(2.0 * x[2]);
        u[0] = 2.0 * sx * sx * s2y * s2z * ct;
        u[1] = -(sy * sy) * s2z * s2x * ct;
        u[2] = -(sz * sz) * s2x * s2y * ct;
        break;
    }
    case OR_VEL_FOURIER2D: {
        /* streamfunction psi = sum_q a_q cos(2 pi k_q.x) + b_q sin(2 pi k_q.x);
         * p = (nmodes, then per mode kx, ky, a, b);  u = d psi/dy,  v = -d psi/dx */
        int nm = (int)p[0];
        for (int q = 0; q < nm; ++q) {
            const double *m = p + 1 + 4 * q;
            double arg = 2.0 * (m[0] * x[0] + m[1] * x[1]); /* theta / pi */
            double dpsi = 2.0 * M_PI * (-m[2] * or_sinpi(arg) + m[3] * or_cospi(arg)); /* d psi / d theta-direction */
            u[0] += m[1] * dpsi;
            u[1] -= m[0] * dpsi;
        }
        break;
    }
    case OR_VEL_FOURIER3D: {
        /* vector potential A = sum_q a_q cos(theta_q) + b_q sin(theta_q), theta_q = 2 pi k_q.x;
         * u = curl A = 2 pi sum_q [cos(theta) (k x b) - sin(theta) (k x a)];
         * p = (nmodes, then per mode kx, ky, kz, ax, ay, az, bx, by, bz) */
        int nm = (int)p[0];
        for (int q = 0; q < nm; ++q) {
            const double *m = p + 1 + 9 * q;
            const double *k = m, *av = m + 3, *bv = m + 6;
            double arg = 2.0 * (k[0] * x[0] + k[1] * x[1] + k[2] * x[2]);
            double c = or_cospi(arg), s = or_sinpi(arg);
            double kxa[3] = {k[1] * av[2] - k[2] * av[1], k[2] * av[0] - k[0] * av[2], k[0] * av[1] - k[1] * av[0]};
            double kxb[3] = {k[1] * bv[2] - k[2] * bv[1], k[2] * bv[0] - k[0] * bv[2], k[0] * bv[1] - k[1] * bv[0]};
            for (int a = 0; a < 3; ++a) u[a] += 2.0 * M_PI * (c * kxb[a] - s * kxa[a]);
        }
        break;
    }
    default:
        u[0] = u[1] = u[2] = NAN;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* eq. (vel): trajectory of every Lagrangian node over one step, classical RK4 from the         */
/* reference position X_i at time t.  Output: displacement in cell units, D[i*dim + a].          */
/* With substeps > 1 or the low-storage RK3, the position is carried through substeps steps of   */
/* h = dt / substeps (Sec. 2: the Lagrangian grid may move for several time steps before the     */
/* fields are interpolated back); the low-storage RK3 is Williamson's (J. Comp. Phys. 35, 1980)  */
/* three-stage scheme q <- A_k q + h u(x, t_s + c_k h), x <- x + B_k q with                        */
/* A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15) and stage times c = (0, 1/3, 3/4).            */
/* A carried velocity (ucar != NULL: the node's own velocity, a transported field with no source, */
/* so constant along the trajectory) replaces the analytic one at every stage.                    */
/* ------------------------------------------------------------------------------------------ */
static void stage_velocity(const or_grid *g, const double *ucar, const double x[3], double t, double u[3])
{
    if (ucar) {
        for (int a = 0; a < 3; ++a) u[a] = ucar[a];
    } else {
        or_velocity(g, x, t, u);
    }
}

static void trajectory_substeps(const or_grid *g, const double *ucar, const double X[3], double t, double dt,
                                double x[3])
{
    const int d = g->dim, S = g->substeps > 1 ? g->substeps : 1;
    const double h = dt / (double)S;
    for (int a = 0; a < 3; ++a) x[a] = X[a];
    for (int st = 0; st < S; ++st) {
        const double ts = t + (double)st * h;
        if (g->integrator == OR_WRK3) {
            double q[3] = {0, 0, 0}, u[3];
            stage_velocity(g, ucar, x, ts, u);
            for (int a = 0; a < d; ++a) {
                q[a] = h * u[a];
                x[a] += (1.0 / 3.0) * q[a];
            }
            stage_velocity(g, ucar, x, ts + h / 3.0, u);
            for (int a = 0; a < d; ++a) {
                q[a] = (-5.0 / 9.0) * q[a] + h * u[a];
                x[a] += (15.0 / 16.0) * q[a];
            }
            stage_velocity(g, ucar, x, ts + 0.75 * h, u);
            for (int a = 0; a < d; ++a) {
                q[a] = (-153.0 / 128.0) * q[a] + h * u[a];
                x[a] += (8.0 / 15.0) * q[a];
            }
        } else {
            double k1[3], k2[3], k3[3], k4[3], y[3] = {0, 0, 0};
            stage_velocity(g, ucar, x, ts, k1);
            for (int a = 0; a < d; ++a) y[a] = x[a] + 0.5 * h * k1[a];
            stage_velocity(g, ucar, y, ts + 0.5 * h, k2);
            for (int a = 0; a < d; ++a) y[a] = x[a] + 0.5 * h * k2[a];
            stage_velocity(g, ucar, y, ts + 0.5 * h, k3);
            for (int a = 0; a < d; ++a) y[a] = x[a] + h * k3[a];
            stage_velocity(g, ucar, y, ts + h, k4);
            for (int a = 0; a < d; ++a) x[a] += h / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        }
    }
}

/* Field plane holding velocity component a of a carried velocity: parameter a when given, else a. */
static int carried_field(const or_grid *g, int a)
{
    return g->n_vel_params > a ? (int)g->vel_params[a] : a;
}

/* Sec. 3.2 (Burgers): the velocity is one of the transported fields, Du/Dt = 0, so every node moves
 * with the value it carries: D_i = trajectory of X_i at the constant velocity u_i (the fields h are
 * those at the start of the step, nfields planes of N values). */
void or_advect_carried(const or_grid *g, const double *h, double dt, double *D)
{
    int64_t N = total_nodes(g);
    int d = g->dim;
    double dx[3];
    for (int a = 0; a < d; ++a) dx[a] = (g->hi[a] - g->lo[a]) / (double)g->n[a];
    set_threads(g);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int64_t k[3];
        node_coords(g, i, k);
        double X[3] = {0, 0, 0}, u[3] = {0, 0, 0}, x[3];
        for (int a = 0; a < d; ++a) {
            X[a] = g->lo[a] + (double)k[a] * dx[a];
            u[a] = h[(int64_t)carried_field(g, a) * N + i];
        }
        trajectory_substeps(g, u, X, 0.0, dt, x);
        for (int a = 0; a < d; ++a) D[i * d + a] = (x[a] - X[a]) / dx[a];
    }
}

void or_advect(const or_grid *g, double t, double dt, double *D)
{
    int64_t N = total_nodes(g);
    int d = g->dim;
    double dx[3];
    for (int a = 0; a < d; ++a) dx[a] = (g->hi[a] - g->lo[a]) / (double)g->n[a];
    const int general = g->integrator == OR_WRK3 || g->substeps > 1;
    set_threads(g);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int64_t k[3];
        node_coords(g, i, k);
        double X[3] = {0, 0, 0}, y[3] = {0, 0, 0};
        double k1[3], k2[3], k3[3], k4[3];
        for (int a = 0; a < d; ++a) X[a] = g->lo[a] + (double)k[a] * dx[a];
        if (general) {
            double x[3];
            trajectory_substeps(g, NULL, X, t, dt, x);
            for (int a = 0; a < d; ++a) D[i * d + a] = (x[a] - X[a]) / dx[a];
            continue;
        }
        or_velocity(g, X, t, k1);
        for (int a = 0; a < d; ++a) y[a] = X[a] + 0.5 * dt * k1[a];
        or_velocity(g, y, t + 0.5 * dt, k2);
        for (int a = 0; a < d; ++a) y[a] = X[a] + 0.5 * dt * k2[a];
        or_velocity(g, y, t + 0.5 * dt, k3);
        for (int a = 0; a < d; ++a) y[a] = X[a] + dt * k3[a];
        or_velocity(g, y, t + dt, k4);
        for (int a = 0; a < d; ++a) {
            double disp = dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
            D[i * d + a] = disp / dx[a];
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Sec. 2.2, eq. (mapping1): the Z0 (multilinear) map of one element.                            */
/* P[v*d + a]: vertex v (bit a of v = offset along axis a) relative to the target, cell units.  */
/* x(xi) = sum_v P_v prod_a (v_a ? xi_a : 1 - xi_a), and its Jacobian J[a][b] = dx_a/dxi_b.      */
/* ------------------------------------------------------------------------------------------ */
static void map_eval(int d, const double *P, const double xi[3], double F[3], double J[3][3])
{
    int nv = 1 << d;
    for (int a = 0; a < 3; ++a) {
        F[a] = 0.0;
        for (int b = 0; b < 3; ++b) J[a][b] = 0.0;
    }
    for (int v = 0; v < nv; ++v) {
        double fac[3], w = 1.0;
        for (int a = 0; a < d; ++a) {
            fac[a] = ((v >> a) & 1) ? xi[a] : 1.0 - xi[a];
            w *= fac[a];
        }
        for (int b = 0; b < d; ++b) {
            double dw = ((v >> b) & 1) ? 1.0 : -1.0; /* derivative of fac[b] */
            for (int a = 0; a < d; ++a)
                if (a != b) dw *= fac[a];
            for (int a = 0; a < d; ++a) J[a][b] += dw * P[v * d + a];
        }
        for (int a = 0; a < d; ++a) F[a] += w * P[v * d + a];
    }
}

static double det_of(int d, double J[3][3])
{
    if (d == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
           + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* Cramer's rule: solve J s = r */
static void cramer(int d, double J[3][3], const double r[3], double det, double s[3])
{
    for (int c = 0; c < d; ++c) {
        double M[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[a][b] = (b == c) ? r[a] : J[a][b];
        s[c] = det_of(d, M) / det;
    }
}

/* Newton inversion: solve x(xi) = 0 starting from the solution of the linear part.
 * Returns OR_OK (converged), OR_NEWTON (iteration cap), OR_FOLD (det J <= 0 at an iterate).
 * xi holds the last iterate (NaN when the linear part itself is singular). */
int or_newton(int d, const double *P, int max_iter, double tol, double xi[3], int *iters)
{
    double F[3], J[3][3], s[3], zero[3] = {0, 0, 0};
    xi[0] = xi[1] = xi[2] = 0.0;
    *iters = 0;
    map_eval(d, P, zero, F, J); /* F = P_0, J = linear part (columns P_{e_a} - P_0) */
    double det = det_of(d, J);
    if (!(det > 0.0)) {
        xi[0] = xi[1] = xi[2] = NAN;
        return OR_FOLD;
    }
    cramer(d, J, F, det, s);
    for (int a = 0; a < d; ++a) xi[a] = -s[a];
    for (int it = 1; it <= max_iter; ++it) {
        *iters = it;
        map_eval(d, P, xi, F, J);
        det = det_of(d, J);
        if (!(det > 0.0)) return OR_FOLD;
        cramer(d, J, F, det, s);
        double step = 0.0;
        for (int a = 0; a < d; ++a) {
            xi[a] -= s[a];
            step = fmax(step, fabs(s[a]));
        }
        if (step <= tol) return OR_OK;
    }
    return OR_NEWTON;
}

/* Vertices of candidate element c relative to target j, in cell units:
 * P_v = (c + v - j) + D[(c + v) mod n]. */
static void element_vertices(const or_grid *g, const double *D, const int64_t j[3], const int64_t c[3],
                             double *P)
{
    int d = g->dim, nv = 1 << d;
    for (int v = 0; v < nv; ++v) {
        int64_t k[3] = {c[0], c[1], c[2]};
        for (int a = 0; a < d; ++a) k[a] += (v >> a) & 1;
        int64_t idx = node_index(g, k);
        for (int a = 0; a < d; ++a) P[v * d + a] = (double)(k[a] - j[a]) + D[idx * d + a];
    }
}

/* Sec. 2.2, element search: start on the side opposite the velocity, invert, and step into the
 * neighbouring element indicated by each out-of-range local coordinate until it is in range. */
int or_locate(const or_grid *g, const double *D, const int64_t j[3], int64_t c[3], double xi[3], int *hops,
              int *iters)
{
    int d = g->dim;
    int64_t jj = node_index(g, j);
    double P[8 * 3];
    c[0] = c[1] = c[2] = 0;
    for (int a = 0; a < d; ++a) {
        double Dj = D[jj * d + a];
        if (g->start_mode == OR_START_BACKWARD)
            c[a] = (int64_t)floor((double)j[a] - Dj);
        else
            c[a] = j[a] - (Dj > 0.0 ? 1 : 0);
    }
    *hops = 0;
    *iters = 0;
    /* The next element of the walk depends on the current element alone, so a walk that comes
     * back to an element it has already tried goes round that cycle until walk_max and fails.
     * Brent's cycle test stops it at the first repeat: `seen` is the element reached after
     * 1, 2, 4, 8, ... hops and every later element is compared with it.  The status is the one
     * the exhausted walk would return (OR_LOCATE). */
    int64_t seen[3] = {c[0], c[1], c[2]};
    int power = 1, lam = 0;
    for (int hop = 0; hop < g->walk_max; ++hop) {
        int it = 0;
        element_vertices(g, D, j, c, P);
        int st = or_newton(d, P, g->newton_max_iter, g->newton_tol, xi, &it);
        *hops = hop + 1;
        *iters += it;
        int finite = 1, inside = 1;
        for (int a = 0; a < d; ++a) {
            if (!isfinite(xi[a])) finite = 0;
            if (!(xi[a] >= -g->slack && xi[a] <= 1.0 + g->slack)) inside = 0;
        }
        if (!finite) return st == OR_OK ? OR_NEWTON : st;
        if (inside) return st;
        for (int a = 0; a < d; ++a) {
            if (xi[a] < -g->slack) c[a] -= 1;
            else if (xi[a] > 1.0 + g->slack) c[a] += 1;
        }
        if (c[0] == seen[0] && c[1] == seen[1] && c[2] == seen[2]) return OR_LOCATE;
        if (++lam == power) {
            for (int a = 0; a < 3; ++a) seen[a] = c[a];
            power *= 2;
            lam = 0;
        }
    }
    return OR_LOCATE;
}

/* Sec. 2.3, order reduction: lower m from max_order while a flag of field f lies in the stencil
 * [c - m, c + m + 1]^d; stop at linear (m = 0). */
int or_order(const or_grid *g, const uint8_t *flags, const int64_t c[3], int f)
{
    int d = g->dim;
    int m = g->max_order;
    while (m > 0) {
        int found = 0;
        int64_t w = 2 * m + 2, cnt = 1;
        for (int a = 0; a < d; ++a) cnt *= w;
        for (int64_t q = 0; q < cnt && !found; ++q) {
            int64_t k[3] = {0, 0, 0}, r = q;
            for (int a = 0; a < d; ++a) {
                k[a] = c[a] - m + r % w;
                r /= w;
            }
            if (flags[node_index(g, k)] & (1u << f)) found = 1;
        }
        if (!found) break;
        m -= 1;
    }
    return m;
}

/* eq. (multiZ) in the element's logical coordinates: value of field hf at the point c + xi,
 * with order m, summed lexicographically (x innermost). */
double or_interp(const or_grid *g, const double *hf, const int64_t c[3], const double xi[3], int m)
{
    int d = g->dim;
    int64_t w = 2 * m + 2, cnt = 1;
    for (int a = 0; a < d; ++a) cnt *= w;
    double sum = 0.0;
    for (int64_t q = 0; q < cnt; ++q) {
        int64_t k[3] = {0, 0, 0}, r = q;
        double wt = 1.0;
        for (int a = 0; a < d; ++a) {
            k[a] = c[a] - m + r % w;
            r /= w;
            wt *= or_zspline(m, (double)(c[a] - k[a]) + xi[a]);
        }
        sum += hf[node_index(g, k)] * wt;
    }
    return sum;
}

/* ------------------------------------------------------------------------------------------ */
/* Sec. 2 (reset of the Lagrangian grid): reconstruct every field on the reference mesh.        */
/* Optional outputs (NULL to skip): cell (wrapped linear index of the element's lower corner,   */
/* -1 on failure), xi[j*dim + a], order[f*N + j], status[j], hops[j], iters[j].                  */
/* A failed target keeps its old values.  Returns the number of failed targets.                 */
/* ------------------------------------------------------------------------------------------ */
int64_t or_remap(const or_grid *g, const double *D, const uint8_t *flags, const double *h_in, double *h_out,
                 int64_t *cell, double *xi_out, uint8_t *order, uint8_t *status, int32_t *hops_out,
                 int32_t *iters_out)
{
    int64_t N = total_nodes(g);
    int d = g->dim;
    int64_t nfail = 0;
    set_threads(g);
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : nfail)
    for (int64_t jj = 0; jj < N; ++jj) {
        int64_t j[3], c[3];
        double xi[3];
        int hops, iters;
        node_coords(g, jj, j);
        int st = or_locate(g, D, j, c, xi, &hops, &iters);
        if (status) status[jj] = (uint8_t)st;
        if (hops_out) hops_out[jj] = hops;
        if (iters_out) iters_out[jj] = iters;
        if (xi_out)
            for (int a = 0; a < d; ++a) xi_out[jj * d + a] = xi[a];
        if (st != OR_OK) {
            nfail += 1;
            if (cell) cell[jj] = -1;
            for (int f = 0; f < g->nfields; ++f) {
                h_out[(int64_t)f * N + jj] = h_in[(int64_t)f * N + jj];
                if (order) order[(int64_t)f * N + jj] = 0xff;
            }
            continue;
        }
        if (cell) cell[jj] = node_index(g, c);
        for (int f = 0; f < g->nfields; ++f) {
            int m = or_order(g, flags, c, f);
            if (order) order[(int64_t)f * N + jj] = (uint8_t)m;
            h_out[(int64_t)f * N + jj] = or_interp(g, h_in + (int64_t)f * N, c, xi, m);
        }
    }
    return nfail;
}

/* Interpolate every field at one target given an element (used to evaluate a target in an
 * element chosen elsewhere, e.g. on a shared face).  Returns the Newton status in that element. */
int or_eval_in_element(const or_grid *g, const double *D, const uint8_t *flags, const double *h_in,
                       const int64_t j[3], const int64_t c[3], double *out, double xi[3], uint8_t *order)
{
    int64_t N = total_nodes(g);
    double P[8 * 3];
    int it;
    element_vertices(g, D, j, c, P);
    int st = or_newton(g->dim, P, g->newton_max_iter, g->newton_tol, xi, &it);
    for (int f = 0; f < g->nfields; ++f) {
        int m = or_order(g, flags, c, f);
        if (order) order[f] = (uint8_t)m;
        out[f] = or_interp(g, h_in + (int64_t)f * N, c, xi, m);
    }
    return st;
}

/* ------------------------------------------------------------------------------------------ */
/* Sec. 3.3, eq. (nlsw): the non-dimensional shallow-water system on the moving nodes,            */
/*   Dh/Dt = -(1 + h) div u,                                                                       */
/*   Du/Dt = -grad h - f u_perp + nu div[(1 + h)(grad u + grad u^T)],  u_perp = (-u2, u1), f = f0 x2, */
/* with h, u1, u2 the fields 0, 1, 2 (further fields are passive), vel_params = (f0) or (f0, nu). */
/* The viscous term takes two passes per stage: the stress tau = (1 + h)(grad u + grad u^T) at    */
/* every node, then its divergence by the same differences.                                       */
/* Sec. 2: spatial derivatives by finite differences on the reference grid, time by Williamson's */
/* low-storage RK3 over the step, then the reset (remap).  Readings: the step starts with the    */
/* nodes on the reference grid and remaps once; at every stage the derivatives are taken on the */
/* node lattice (the reference grid's stencil applied to the nodes' current values, i.e. in the */
/* reference coordinates X) and turned into physical ones by the chain rule with the Jacobian   */
/* J = dx/dX = I + de/dX of the node positions (de/dX by the same differences), so that          */
/* grad h = J^-T dh/dX and div u = tr(du/dX J^-1); the node moves with its own current velocity; */
/* f is taken at the node's current position.  The                                               */
/* difference is that of the Z-spline basis of order m_max (Sec. 2.1: differentiating a Z-spline  */
/* interpolant at the nodes gives finite differences): the derivative at a node of the interpolant,*/
/* sum_k w_k Z'(-k) / dx, i.e. the second-order centred difference for m <= 1 (Z1'(1) = -1/2) and */
/* the fourth-order one for m = 2 (Z2'(1) = -2/3, Z2'(2) = 1/12).                                */
/* ------------------------------------------------------------------------------------------ */
static double lattice_derivative(const or_grid *g, const double *w, const int64_t k[3], int a, double dxa)
{
    int64_t kp[3] = {k[0], k[1], k[2]}, km[3] = {k[0], k[1], k[2]};
    kp[a] += 1;
    km[a] -= 1;
    const double d1 = w[node_index(g, kp)] - w[node_index(g, km)];
    if (g->max_order < 2) return 0.5 * d1 / dxa;
    kp[a] += 1;
    km[a] -= 1;
    const double d2 = w[node_index(g, kp)] - w[node_index(g, km)];
    return ((2.0 / 3.0) * d1 - (1.0 / 12.0) * d2) / dxa;
}

/* Jacobian J = dx/dX of the node positions at node k (e: displacement planes, physical units)
 * and its inverse, row-major I[0..3] = (J^-1)_00, _01, _10, _11. */
static void node_jacobian_inverse(const or_grid *g, const double *ex, const double *ey, const int64_t k[3],
                                  const double dx[2], double I[4])
{
    const double J00 = 1.0 + lattice_derivative(g, ex, k, 0, dx[0]), J01 = lattice_derivative(g, ex, k, 1, dx[1]);
    const double J10 = lattice_derivative(g, ey, k, 0, dx[0]), J11 = 1.0 + lattice_derivative(g, ey, k, 1, dx[1]);
    const double det = J00 * J11 - J01 * J10;
    I[0] = J11 / det;
    I[1] = -J01 / det;
    I[2] = -J10 / det;
    I[3] = J00 / det;
}

/* One step of the shallow-water system: h (nfields planes) is replaced by the remapped fields.
 * Scratch: W (nfields planes), q (3 planes), e and qx (2 planes each), D (2 per node),
 * flags (N), tmp (nfields planes).  Returns the failed targets of the remap. */
static int64_t or_nlsw_step(const or_grid *g, double *h, double dt, double *W, double *q, double *e, double *qx,
                            double *tau, double *D, uint8_t *flags, double *tmp)
{
    const int64_t N = total_nodes(g);
    const double A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0}, B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    const double f0 = g->vel_params[0];
    const double nu = g->n_vel_params > 1 ? g->vel_params[1] : 0.0;
    double dx[2];
    for (int a = 0; a < 2; ++a) dx[a] = (g->hi[a] - g->lo[a]) / (double)g->n[a];
    memcpy(W, h, sizeof(double) * (size_t)N * (size_t)g->nfields);
    memset(q, 0, sizeof(double) * (size_t)N * 3);
    memset(e, 0, sizeof(double) * (size_t)N * 2);
    memset(qx, 0, sizeof(double) * (size_t)N * 2);
    const double *wh = W, *wu = W + N, *wv = W + 2 * N;
    double *ex = e, *ey = e + N; /* node displacement (physical units), one plane per axis */
    set_threads(g);
    for (int s = 0; s < 3; ++s) {
        if (nu != 0.0) {
            /* pass 1: the stress tau = (1 + h)(grad u + grad u^T) at every node (three planes) */
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < N; ++i) {
                int64_t k[3];
                node_coords(g, i, k);
                double I[4];
                node_jacobian_inverse(g, ex, ey, k, dx, I);
                const double uX = lattice_derivative(g, wu, k, 0, dx[0]), uY = lattice_derivative(g, wu, k, 1, dx[1]);
                const double vX = lattice_derivative(g, wv, k, 0, dx[0]), vY = lattice_derivative(g, wv, k, 1, dx[1]);
                const double ux = I[0] * uX + I[2] * uY, uy = I[1] * uX + I[3] * uY;
                const double vx = I[0] * vX + I[2] * vY, vy = I[1] * vX + I[3] * vY;
                const double d = 1.0 + wh[i];
                tau[i] = d * 2.0 * ux;
                tau[N + i] = d * (uy + vx);
                tau[2 * N + i] = d * 2.0 * vy;
            }
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            int64_t k[3];
            node_coords(g, i, k);
            /* Jacobian of the node positions and its inverse */
            double I[4];
            node_jacobian_inverse(g, ex, ey, k, dx, I);
            const double I00 = I[0], I01 = I[1], I10 = I[2], I11 = I[3];
            /* reference-coordinate derivatives */
            const double hX = lattice_derivative(g, wh, k, 0, dx[0]), hY = lattice_derivative(g, wh, k, 1, dx[1]);
            const double uX = lattice_derivative(g, wu, k, 0, dx[0]), uY = lattice_derivative(g, wu, k, 1, dx[1]);
            const double vX = lattice_derivative(g, wv, k, 0, dx[0]), vY = lattice_derivative(g, wv, k, 1, dx[1]);
            /* physical: grad h = J^-T (hX, hY); div u = du/dX_b (J^-1)_b0 + dv/dX_b (J^-1)_b1 */
            const double hx = I00 * hX + I10 * hY, hy = I01 * hX + I11 * hY;
            const double div = uX * I00 + uY * I10 + vX * I01 + vY * I11;
            const double y = g->lo[1] + (double)k[1] * dx[1] + ey[i];
            const double f = f0 * y;
            double S[3] = {-(1.0 + wh[i]) * div, -hx + f * wv[i], -hy - f * wu[i]};
            if (nu != 0.0) {
                /* pass 2: nu div tau, (div tau)_a = d tau_a0 / dx + d tau_a1 / dy */
                const double *t11 = tau, *t12 = tau + N, *t22 = tau + 2 * N;
                const double aX = lattice_derivative(g, t11, k, 0, dx[0]), aY = lattice_derivative(g, t11, k, 1, dx[1]);
                const double bX = lattice_derivative(g, t12, k, 0, dx[0]), bY = lattice_derivative(g, t12, k, 1, dx[1]);
                const double cX = lattice_derivative(g, t22, k, 0, dx[0]), cY = lattice_derivative(g, t22, k, 1, dx[1]);
                const double t11x = I00 * aX + I10 * aY, t12y = I01 * bX + I11 * bY;
                const double t12x = I00 * bX + I10 * bY, t22y = I01 * cX + I11 * cY;
                S[1] += nu * (t11x + t12y);
                S[2] += nu * (t12x + t22y);
            }
            for (int c = 0; c < 3; ++c) q[(int64_t)c * N + i] = A[s] * q[(int64_t)c * N + i] + dt * S[c];
            qx[i] = A[s] * qx[i] + dt * wu[i];
            qx[N + i] = A[s] * qx[N + i] + dt * wv[i];
        }
        for (int64_t i = 0; i < N; ++i) {
            for (int c = 0; c < 3; ++c) W[(int64_t)c * N + i] += B[s] * q[(int64_t)c * N + i];
            ex[i] += B[s] * qx[i];
            ey[i] += B[s] * qx[N + i];
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        D[2 * i + 0] = ex[i] / dx[0];
        D[2 * i + 1] = ey[i] / dx[1];
    }
    or_flags(g, W, flags);
    const int64_t nfail = or_remap(g, D, flags, W, tmp, NULL, NULL, NULL, NULL, NULL, NULL);
    memcpy(h, tmp, sizeof(double) * (size_t)N * (size_t)g->nfields);
    return nfail;
}

static int64_t or_nlsw_steps(const or_grid *g, double *h, double dt, int nsteps)
{
    const int64_t N = total_nodes(g);
    const size_t F = (size_t)N * (size_t)g->nfields;
    double *W = (double *)malloc(sizeof(double) * F), *tmp = (double *)malloc(sizeof(double) * F);
    double *q = (double *)malloc(sizeof(double) * (size_t)N * 3);
    double *e = (double *)malloc(sizeof(double) * (size_t)N * 2), *qx = (double *)malloc(sizeof(double) * (size_t)N * 2);
    double *D = (double *)malloc(sizeof(double) * (size_t)N * 2);
    double *tau = (double *)malloc(sizeof(double) * (size_t)N * 3);
    uint8_t *flags = (uint8_t *)malloc((size_t)N);
    int64_t nfail = 0;
    if (W && tmp && q && e && qx && D && tau && flags) {
        for (int s = 0; s < nsteps; ++s) nfail += or_nlsw_step(g, h, dt, W, q, e, qx, tau, D, flags, tmp);
    } else {
        nfail = -1;
    }
    free(tau);
    free(W);
    free(tmp);
    free(q);
    free(e);
    free(qx);
    free(D);
    free(flags);
    return nfail;
}

/* One full FSL step sequence: flags of the current fields, trajectories, remap.  h is updated
 * in place (nfields planes).  Returns the total number of failed targets. */
int64_t or_step(const or_grid *g, double *h, double t0, double dt, int nsteps)
{
    if (g->vel_kind == OR_VEL_NLSW) return or_nlsw_steps(g, h, dt, nsteps);
    int64_t N = total_nodes(g);
    double *D = (double *)malloc(sizeof(double) * (size_t)N * (size_t)g->dim);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)N * (size_t)g->nfields);
    uint8_t *flags = (uint8_t *)malloc((size_t)N);
    int64_t nfail = 0;
    if (!D || !tmp || !flags) {
        free(D);
        free(tmp);
        free(flags);
        return -1;
    }
    for (int s = 0; s < nsteps; ++s) {
        double t = t0 + (double)s * dt;
        or_flags(g, h, flags);
        if (g->vel_kind == OR_VEL_CARRIED)
            or_advect_carried(g, h, dt, D);
        else
            or_advect(g, t, dt, D);
        nfail += or_remap(g, D, flags, h, tmp, NULL, NULL, NULL, NULL, NULL, NULL);
        memcpy(h, tmp, sizeof(double) * (size_t)N * (size_t)g->nfields);
    }
    free(D);
    free(tmp);
    free(flags);
    return nfail;
}

/* ------------------------------------------------------------------------------------------ */
/* Sec. 3.1: discrete moments about the box centre c:  m_0 = sum h,                             */
/* m_p = sum_i h_i sum_a (x_a^i - c_a)^p  (p >= 1).  Plain sequential sum.                      */
/* ------------------------------------------------------------------------------------------ */
void or_moments(const or_grid *g, const double *h, int pmax, double *out)
{
    int64_t N = total_nodes(g);
    int d = g->dim;
    double dx[3], cen[3];
    for (int a = 0; a < d; ++a) {
        dx[a] = (g->hi[a] - g->lo[a]) / (double)g->n[a];
        cen[a] = 0.5 * (g->lo[a] + g->hi[a]);
    }
    for (int p = 0; p <= pmax; ++p) out[p] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t k[3];
        node_coords(g, i, k);
        out[0] += h[i];
        for (int p = 1; p <= pmax; ++p) {
            double s = 0.0;
            for (int a = 0; a < d; ++a) {
                double r = g->lo[a] + (double)k[a] * dx[a] - cen[a], rp = 1.0;
                for (int q = 0; q < p; ++q) rp *= r;
                s += rp;
            }
            out[p] += h[i] * s;
        }
    }
}
