"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped or wrong term, a sign, an index, a transposed operand) in
a copy of the oracle's C source, builds that copy into a scratch directory and runs the pin tests
that should reject it.  The copy never touches the real oracle build.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sl_oracle.c")

MUTATIONS = {
    "z1_coefficient": ("1.0 - 2.5 * x2 + 1.5 * x3", "1.0 - 2.5 * x2 + 1.4 * x3", "test_oracle_basis.py"),
    "z2_coefficient": ("(545.0 / 24.0) * x3", "(544.0 / 24.0) * x3", "test_oracle_basis.py"),
    "hat_shape": ("return ax < 1.0 ? 1.0 - ax : 0.0;", "return ax < 1.0 ? 1.0 - ax * ax : 0.0;", "test_oracle_basis.py"),
    "limiter_strictness": ("if (num > g->threshold * den)", "if (num >= g->threshold * den)", "test_oracle_limiter.py"),
    "limiter_denominator": ("double den = fmax(fabs(dp), fabs(dm));", "double den = fmin(fabs(dp), fabs(dm));",
                            "test_oracle_limiter.py"),
    "limiter_axis": ("kp[a] += 1;", "kp[0] += 1;", "test_oracle_limiter.py"),
    "rk4_weight": ("(k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a])", "(k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + 2.0 * k4[a])",
                   "test_oracle_advect.py"),
    "rk4_stage_time": ("or_velocity(g, y, t + 0.5 * dt, k3);", "or_velocity(g, y, t + dt, k3);", "test_oracle_advect.py"),
    "rk4_stage_position": ("y[a] = X[a] + 0.5 * dt * k2[a];", "y[a] = X[a] + 0.5 * dt * k1[a];", "test_oracle_advect.py"),
    "swirl_sign": ("u[1] = -(sy * sy) * or_sinpi(2.0 * x[0]) * ct;", "u[1] = (sy * sy) * or_sinpi(2.0 * x[0]) * ct;",
                   "test_oracle_advect.py"),
    "deform_amplitude": ("u[0] = 2.0 * sx * sx * s2y * s2z * ct;", "u[0] = sx * sx * s2y * s2z * ct;", "test_oracle_advect.py"),
    "fourier_component": ("u[0] += m[1] * dpsi;", "u[0] += m[0] * dpsi;", "test_oracle_advect.py"),
    "cospi_reduction": ("if (a <= 0.75) return sin(M_PI * (0.5 - a));", "if (a <= 0.75) return sin(M_PI * (a - 0.5));",
                        "test_oracle_basis.py"),
    "jacobian_sign": ("double dw = ((v >> b) & 1) ? 1.0 : -1.0;", "double dw = ((v >> b) & 1) ? 1.0 : 1.0;",
                      "test_oracle_mapping.py"),
    "newton_update_sign": ("xi[a] -= s[a];", "xi[a] += s[a];", "test_oracle_mapping.py"),
    "walk_direction": ("if (xi[a] < -g->slack) c[a] -= 1;", "if (xi[a] < -g->slack) c[a] += 1;", "test_oracle_mapping.py"),
    "vertex_displacement_sign": ("P[v * d + a] = (double)(k[a] - j[a]) + D[idx * d + a];",
                                 "P[v * d + a] = (double)(k[a] - j[a]) - D[idx * d + a];", "test_oracle_mapping.py"),
    "interp_argument_sign": ("wt *= or_zspline(m, (double)(c[a] - k[a]) + xi[a]);",
                             "wt *= or_zspline(m, (double)(c[a] - k[a]) - xi[a]);", "test_oracle_remap.py"),
    "interp_transposed_axes": ("wt *= or_zspline(m, (double)(c[a] - k[a]) + xi[a]);",
                               "wt *= or_zspline(m, (double)(c[a] - k[a]) + xi[d - 1 - a]);", "test_oracle_remap.py"),
    "order_stencil_offset": ("k[a] = c[a] - m + r % w;\n                r /= w;\n            }\n            if",
                             "k[a] = c[a] - m + 1 + r % w;\n                r /= w;\n            }\n            if",
                             "test_oracle_limiter.py"),
    "failed_target_value": ("h_out[(int64_t)f * N + jj] = h_in[(int64_t)f * N + jj];", "h_out[(int64_t)f * N + jj] = 0.0;",
                            "test_oracle_remap.py"),
    "wrk3_coefficient": ("q[a] = (-5.0 / 9.0) * q[a] + h * u[a];", "q[a] = (-4.0 / 9.0) * q[a] + h * u[a];",
                         "test_oracle_advect.py"),
    "wrk3_stage_time": ("stage_velocity(g, ucar, x, ts + h / 3.0, u);", "stage_velocity(g, ucar, x, ts + 0.5 * h, u);",
                        "test_oracle_advect.py"),
    "wrk3_update_weight": ("x[a] += (8.0 / 15.0) * q[a];", "x[a] += (7.0 / 15.0) * q[a];", "test_oracle_advect.py"),
    "substep_time": ("const double ts = t + (double)st * h;", "const double ts = t;", "test_oracle_advect.py"),
    "carried_component": ("u[a] = h[(int64_t)carried_field(g, a) * N + i];", "u[a] = h[i];",
                          "test_oracle_burgers.py"),
    "carried_index": ("return g->n_vel_params > a ? (int)g->vel_params[a] : a;", "return a;",
                      "test_oracle_burgers.py"),
    "carried_sign": ("for (int a = 0; a < d; ++a) D[i * d + a] = (x[a] - X[a]) / dx[a];\n    }\n}",
                     "for (int a = 0; a < d; ++a) D[i * d + a] = (X[a] - x[a]) / dx[a];\n    }\n}",
                     "test_oracle_burgers.py"),
    "nlsw_coriolis_sign": ("-hy - f * wu[i]}", "-hy + f * wu[i]}", "test_oracle_nlsw.py"),
    "nlsw_depth_factor": ("-(1.0 + wh[i]) * div", "-div", "test_oracle_nlsw.py"),
    "nlsw_difference": ("return ((2.0 / 3.0) * d1 - (1.0 / 12.0) * d2) / dxa;", "return (0.5 * d1 - (1.0 / 12.0) * d2) / dxa;",
                        "test_oracle_nlsw.py"),
    "nlsw_chain_rule": ("const double hx = I00 * hX + I10 * hY, hy = I01 * hX + I11 * hY;",
                        "const double hx = hX, hy = hY;", "test_oracle_nlsw.py"),
    "nlsw_node_velocity": ("qx[N + i] = A[s] * qx[N + i] + dt * wv[i];", "qx[N + i] = A[s] * qx[N + i] + dt * wu[i];",
                           "test_oracle_nlsw.py"),
    "nlsw_stress_normal": ("tau[i] = d * 2.0 * ux;", "tau[i] = d * ux;", "test_oracle_nlsw.py"),
    "nlsw_stress_shear": ("tau[N + i] = d * (uy + vx);", "tau[N + i] = d * uy;", "test_oracle_nlsw.py"),
    "nlsw_viscous_sign": ("S[1] += nu * (t11x + t12y);", "S[1] -= nu * (t11x + t12y);", "test_oracle_nlsw.py"),
    "nlsw_jacobian_transposed": ("I[1] = -J01 / det;\n    I[2] = -J10 / det;", "I[1] = -J10 / det;\n    I[2] = -J01 / det;",
                                 "test_oracle_nlsw.py"),
    "nlsw_jacobian_axis": ("J01 = lattice_derivative(g, ex, k, 1, dx[1]);", "J01 = lattice_derivative(g, ex, k, 0, dx[1]);",
                           "test_oracle_nlsw.py"),
    "nlsw_difference_fd2": ("if (g->max_order < 2) return 0.5 * d1 / dxa;", "if (g->max_order < 2) return d1 / dxa;",
                            "test_oracle_nlsw.py"),
    "nlsw_coriolis_position": ("const double y = g->lo[1] + (double)k[1] * dx[1] + ey[i];",
                               "const double y = g->lo[1] + (double)k[1] * dx[1];", "test_oracle_nlsw.py"),
    "nlsw_stage_weight": ("B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};", "B[3] = {1.0 / 3.0, 0.5, 8.0 / 15.0};",
                          "test_oracle_nlsw.py"),
    "step_time": ("double t = t0 + (double)s * dt;", "double t = t0;", "test_oracle_step.py"),
    "walk_revisit_one_axis": ("if (c[0] == seen[0] && c[1] == seen[1] && c[2] == seen[2]) return OR_LOCATE;",
                              "if (c[0] == seen[0]) return OR_LOCATE;", "test_oracle_mapping.py"),
    "walk_revisit_never_moves": ("for (int a = 0; a < 3; ++a) seen[a] = c[a];", "(void)0;",
                                 "test_oracle_mapping.py"),
    "cramer_column": ("M[a][b] = (b == c) ? r[a] : J[a][b];", "M[a][b] = (a == c) ? r[b] : J[a][b];",
                      "test_oracle_mapping.py"),
    "moment_power": ("for (int q = 0; q < p; ++q) rp *= r;", "for (int q = 1; q < p; ++q) rp *= r;",
                     "test_oracle_step.py"),
    "moment_centre": ("cen[a] = 0.5 * (g->lo[a] + g->hi[a]);", "cen[a] = 0.5 * (g->hi[a] - g->lo[a]);",
                      "test_oracle_step.py"),
}


WORKERS = max(1, min(4, (os.cpu_count() or 1) // 2))


def _plant_and_run(name, scratch):
    """Build the oracle with mistake `name` planted into `scratch` and run its pin tests there:
    (pattern found, return code, end of the output)."""
    old, new, test_file = MUTATIONS[name]
    base = open(SRC).read()
    if old not in base:
        return False, None, ""
    src = os.path.join(scratch, "sl_oracle.c")
    with open(src, "w") as f:
        f.write(base.replace(old, new, 1))
    env = dict(os.environ, SL_ORACLE_SOURCE=src, SL_ORACLE_BUILD_DIR=scratch, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join("tests", test_file)], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return True, r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(request, tmp_path_factory):
    """The selected mutation cases, run a few at a time in separate processes (each builds its own
    copy of the oracle), so that the whole set costs about a minute."""
    names = sorted({item.callspec.params["name"] for item in request.session.items
                    if getattr(item, "originalname", "") == "test_planted_mistake_is_caught"})
    dirs = {n: str(tmp_path_factory.mktemp(n)) for n in names}
    with ThreadPoolExecutor(max_workers=WORKERS) as ex:
        futures = {n: ex.submit(_plant_and_run, n, dirs[n]) for n in names}
        return {n: f.result() for n, f in futures.items()}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, outcomes):
    found, rc, out = outcomes[name]
    assert found, "mutation pattern no longer matches the oracle source"
    assert rc == 1, f"planted mistake '{name}' was not caught:\n{out}"
