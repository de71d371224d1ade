"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU,
in a temporary directory), compiles it, and runs the pin suite against it
through LBRS_ORACLE_LIB.  The pin suite must fail for every mutant.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbrs_oracle.c")

MUTANTS = {
    "relaxation_weights_swapped": ("fs[idx] = inert ? f[idx] : om1 * f[idx] + om * feq[q * K + k];",
                                   "fs[idx] = inert ? f[idx] : om * f[idx] + om1 * feq[q * K + k];"),
    "energy_flux_drops_pressure": ("F[3] = u * (en + p);", "F[3] = u * en;"),
    "momentum_flux_drops_pressure": ("F[1] = mx * u + p;", "F[1] = mx * u;"),
    "pressure_drops_v_term": ("double p = (g - 1.0) * (en - 0.5 * (mx * u + my * v));",
                              "double p = (g - 1.0) * (en - 0.5 * (mx * u));"),
    "stream_direction_reversed": ("int64_t si = i - sx, sj = j - sy;", "int64_t si = i + sx, sj = j - sy;"),
    "populations_f2_f4_swapped": ("static const int SY2[4] = {-1, -1, +1, +1};",
                                  "static const int SY2[4] = {-1, +1, +1, -1};"),
    "wall_no_sign_flip": ("double sgn = (k == 2) ? -1.0 : 1.0;", "double sgn = 1.0;"),
    "transmissive_clamps_inward": ("else si = si < 0 ? 0 : nx - 1;              /* transmissive */",
                                   "else si = si < 0 ? 1 : nx - 2;              /* transmissive */"),
    "flux_scale_2lambda": ("double c = 1.0 / (4.0 * P->lambda);", "double c = 1.0 / (2.0 * P->lambda);"),
    "d1q2_flux_drops_pressure": ("double G[3] = {m, m * u + p, u * (en + p)};",
                                 "double G[3] = {m, m * u, u * (en + p)};"),
    "gamma_in_place_of_gamma_minus_1": ("return (g - 1.0) * (U[3] - 0.5 * (U[1] * u + U[2] * v));",
                                        "return g * (U[3] - 0.5 * (U[1] * u + U[2] * v));"),
    "ghost_uses_wrong_side": ("profile_ghost(P, side_x, sj, gbuf) : ghost[side_x];",
                              "profile_ghost(P, side_x, sj, gbuf) : ghost[side_x ^ 1];"),
    # D1Q3
    "d1q3_rest_fraction_quarter": ("double a = U[k] / 3.0;", "double a = U[k] / 4.0;"),
    "d1q3_rest_particle_moves": ("static const int SX13[3] = {-1, 0, +1};", "static const int SX13[3] = {-1, +1, +1};"),
    "d1q3_bound_without_factor": ("if (P->lattice == ORC_D1Q3) return sqrt(1.5) * (fabs(U[1] / U[0]) + a);",
                                  "if (P->lattice == ORC_D1Q3) return (fabs(U[1] / U[0]) + a);"),
    # adjoint
    "adjoint_drops_y_flux_jacobian": ("ubar[k] = 0.25 * a[k] + c * sf + c * sg;", "ubar[k] = 0.25 * a[k] + c * sf;"),
    "adjoint_wrong_momentum_jacobian": ("{q2h - u * u, (3.0 - g) * u, -gm1 * v, gm1},",
                                        "{q2h - u * u, (2.0 - g) * u, -gm1 * v, gm1},"),
    "adjoint_pushes_the_wrong_way": ("const int64_t ti = (i - SX2[q] + nx) % nx, tj = (j - SY2[q] + ny) % ny;",
                                     "const int64_t ti = (i + SX2[q] + nx) % nx, tj = (j + SY2[q] + ny) % ny;"),
    # internal walls
    "obstacle_x_wall_keeps_rho_u_sign": ("*sgn_u = mx != sx ? -1.0 : 1.0;", "*sgn_u = 1.0;"),
    "obstacle_walls_classified_crosswise": ("    if (xn && !yn) {\n        mx = -sx;\n    } else if (!xn && yn) {\n        my = -sy;",
                                            "    if (xn && !yn) {\n        my = -sy;\n    } else if (!xn && yn) {\n        mx = -sx;"),
    "obstacle_corner_reflects_in_y": ("    } else {\n        mx = -sx;\n        my = -sy;\n    }",
                                      "    } else {\n        my = -sy;\n    }"),
    "obstacle_solid_cells_relax": ("fs[idx] = inert ? f[idx] : om1 * f[idx] + om * feq[q * K + k];",
                                   "fs[idx] = om1 * f[idx] + om * feq[q * K + k];"),
    # scalar D2Q4 (2-D Burgers)
    "burgers_flux_drops_half": ("double g1 = 0.5 * u * u, g2 = u;", "double g1 = u * u, g2 = u;"),
    "burgers_drops_y_flux": ("double g1 = 0.5 * u * u, g2 = u;", "double g1 = 0.5 * u * u, g2 = 0.0 * u;"),
    "profile_at_cell_edge": ("(((double)m + 0.5) * P->dx)", "(((double)m) * P->dx)"),
    "profile_ghost_wrong_side": ("profile_ghost(P, side_x, sj, gbuf)", "profile_ghost(P, side_x ^ 1, sj, gbuf)"),
    # adaptive lambda
    "adaptive_clock_uses_new_lambda": ("double t_next = last ? t_final : tt + dx / lam_cur;",
                                       "double t_next = last ? t_final : tt + dx / (safety * bound);"),
    "adaptive_collides_with_stream_lambda": ("Qc.lambda = lam_new;", "Qc.lambda = lam_cur;"),
    "adaptive_ignores_dirichlet_states": ("        if (P->bc_kind[s] != ORC_DIRICHLET) continue;\n        double u[4];",
                                          "        if (P->bc_kind[s] != ORC_DIRICHLET || 1) continue;\n        double u[4];"),
    # local wave-speed bound and boundary resolution
    "d2q4_bound_without_sqrt2": ("return (s1 > s2 ? s1 : s2) + sqrt(2.0) * a;", "return (s1 > s2 ? s1 : s2) + a;"),
    "sound_speed_without_gamma": ("double a = sqrt(P->gamma * p / U[0]);", "double a = sqrt(p / U[0]);"),
    "periodic_y_clamps": ("else if (kind == ORC_PERIODIC) sj = (sj + ny) % ny;",
                          "else if (kind == ORC_PERIODIC) sj = sj < 0 ? 0 : ny - 1;"),
    "corner_ghost_from_y_side": (
        "if (kind == ORC_DIRICHLET) g = scalar ? profile_ghost(P, side_x, sj, gbuf) : ghost[side_x];",
        "if (kind == ORC_DIRICHLET && !(side_y >= 0 && P->bc_kind[side_y] == ORC_DIRICHLET))"
        " g = scalar ? profile_ghost(P, side_x, sj, gbuf) : ghost[side_x];"),
    "top_wall_crossed_mapping": (
        "f[(0 * K + k) * N + c] = sgn * f[(3 * K + k) * N + c];\n"
        "                    f[(1 * K + k) * N + c] = sgn * f[(2 * K + k) * N + c];",
        "f[(0 * K + k) * N + c] = sgn * f[(2 * K + k) * N + c];\n"
        "                    f[(1 * K + k) * N + c] = sgn * f[(3 * K + k) * N + c];"),
    # halfway wall
    "halfway_wall_wrong_neighbour": ("const int m = 3 - q;\n                    const double* gm = NULL;",
                                     "const int m = 3 - q;\n                    const double* gm = NULL;\n"
                                     "                    si = i + sx;"),
    "halfway_wall_keeps_rho_v_sign": ("f[(q * K + k) * N + c] = sgn * (gm ? gm[m * K + k]",
                                      "f[(q * K + k) * N + c] = 1.0 * (gm ? gm[m * K + k]"),
    "halfway_wall_same_population": ("const int m = 3 - q;", "const int m = q ^ 1;"),
    # boundary balance
    "balance_outflow_tests_the_source": (
        "if ((!px && (di < 0 || di >= nx)) || (!py && (dj < 0 || dj >= ny)))",
        "if ((!px && (si < 0 || si >= nx)) || (!py && (sj < 0 || sj >= ny)))"),
    "balance_inflow_misses_y_sides": (
        "if ((!px && (si < 0 || si >= nx)) || (!py && (sj < 0 || sj >= ny)))\n                        in +=",
        "if ((!px && (si < 0 || si >= nx)))\n                        in +="),
    "adjoint_relaxation_weights_swapped": ("gout[(q * 4 + k) * N + tj * nx + ti] = om1 * gq[q * 4 + k] + om * ubar[k];",
                                           "gout[(q * 4 + k) * N + tj * nx + ti] = om * gq[q * 4 + k] + om1 * ubar[k];"),
}


PIN_FILES = ("test_oracle_pins.py", "test_oracle_pins_d1q3.py", "test_oracle_adjoint.py", "test_oracle_obstacles.py",
             "test_oracle_burgers.py", "test_oracle_adaptive.py", "test_oracle_halfway.py", "test_oracle_balance.py")
FEATURE_FILES = {"d1q3": "test_oracle_pins_d1q3.py", "adjoint": "test_oracle_adjoint.py",
                 "obstacle": "test_oracle_obstacles.py", "burgers": "test_oracle_burgers.py",
                 "profile": "test_oracle_burgers.py", "adaptive": "test_oracle_adaptive.py",
                 "halfway": "test_oracle_halfway.py", "d2q4_bound": "test_oracle_adaptive.py",
                 "balance": "test_oracle_balance.py"}


def _first_file(name):
    return next((f for prefix, f in FEATURE_FILES.items() if name.startswith(prefix)), PIN_FILES[0])


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = tmp_path / "lbrs_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "liblbrs_oracle_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                    str(mutated), "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, LBRS_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    # the whole pin suite, the pins of the mutant's own feature first (-x stops at the first catch)
    files = [os.path.join(ROOT, "tests", f) for f in sorted(PIN_FILES, key=lambda f: f != _first_file(name))]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"
