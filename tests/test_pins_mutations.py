"""Sensitivity of the oracle's pins: each plausible mistake below (a flipped
sign, a dropped factor, a swapped index or operand) is planted in a copy of
the oracle source on the CPU, compiled, and the pin tests must fail on it.
The mutated copies live in a temporary folder and are loaded through the
oracle loader's override variable; the real oracle is untouched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sph_oracle.c")
PIN_FILES = ["tests/test_oracle_kernel.py", "tests/test_oracle_neighbours.py",
             "tests/test_oracle_physics.py", "tests/test_oracle_variants.py",
             "tests/test_oracle_walls.py", "tests/test_oracle_sampling.py"]

MUTATIONS = {
    "riemann_ustar_sign": ("*Ustar = 0.5 * (UL + UR) + (pL - pR)",
                           "*Ustar = 0.5 * (UL + UR) + (pR - pL)"),
    "riemann_limiter_direction": ("double jump = UL - UR;", "double jump = UR - UL;"),
    "riemann_rho_bar": ("double rho_bar = 0.5 * (rhoL + rhoR);", "double rho_bar = rhoL;"),
    "pressure_volume_index": ("double f = Ps * (s->m / rho[j])",
                              "double f = Ps * (s->m / rho[i])"),
    "pressure_direction": ("for (int k = 0; k < 3; ++k) out[k] = -2.0 / rho[i] * a[k];",
                           "for (int k = 0; k < 3; ++k) out[k] = 2.0 / rho[i] * a[k];"),
    "wall_gravity_sign": ("gdot += (s->xw[w][k] - s->x[i][k]) * (s->g[k] - s->aw[w][k]);",
                          "gdot += (s->x[i][k] - s->xw[w][k]) * (s->g[k] - s->aw[w][k]);"),
    "wall_mirror_velocity": ("d += (2.0 * vw[k] - vi[k]) * e[k];",
                             "d += (2.0 * vw[k] + vi[k]) * e[k];"),
    "wall_mirror_factor": ("d += (2.0 * vw[k] - vi[k]) * e[k];",
                           "d += (vw[k] - vi[k]) * e[k];"),
    "wall_viscous_mirror": ("a[k] += coef * (2.0 * (s->v[i][k] - s->vw[w][k]));",
                            "a[k] += coef * (s->v[i][k] - s->vw[w][k]);"),
    "wall_accel_sign": ("gdot += (s->xw[w][k] - s->x[i][k]) * (s->g[k] - s->aw[w][k]);",
                        "gdot += (s->xw[w][k] - s->x[i][k]) * (s->g[k] + s->aw[w][k]);"),
    "wall_accel_law": ("a[c] = -s->awu[u][c] * s->womega * s->womega * sn;",
                       "a[c] = -s->awu[u][c] * s->womega * sn;"),
    "translate_half_step_time": ("if (s->wtranslate) place_walls(s, s->t + 0.5 * dt);",
                                 "if (s->wtranslate) place_walls(s, s->t + dt);"),
    "translate_speed": ("x[c] = s->xw0[u][c] + t * s->vwu[u][c] + s->awu[u][c] * sn;",
                        "x[c] = s->xw0[u][c] + 0.5 * t * s->vwu[u][c] + s->awu[u][c] * sn;"),
    "translate_not_rebinned": ("if (s->wtranslate) bin_walls(s, s->t);",
                               "if (0) bin_walls(s, s->t);"),
    "wall_viscous_velocity_sign": ("a[k] += coef * (2.0 * (s->v[i][k] - s->vw[w][k]));",
                                   "a[k] += coef * (2.0 * (s->v[i][k] + s->vw[w][k]));"),
    "continuity_sign": ("sum += (s->m / s->rho[j]) * osph_dW(s->dim, s->h, r) * (UL - Us);",
                        "sum += (s->m / s->rho[j]) * osph_dW(s->dim, s->h, r) * (Us - UL);"),
    "viscous_operands": ("a[k] += coef * (s->v[i][k] - s->v[j][k]);",
                         "a[k] += coef * (s->v[j][k] - s->v[i][k]);"),
    "viscous_regulariser": ("osph_dW(s->dim, s->h, r) / (r + eps);\n        for (int k = 0; k < 3; ++k) a[k] += coef * (s->v[i][k]",
                            "osph_dW(s->dim, s->h, r) / (r + eps) / r;\n        for (int k = 0; k < 3; ++k) a[k] += coef * (s->v[i][k]"),
    "half_step_drift": ("for (int k = 0; k < s->dim; ++k) s->x[i][k] += 0.5 * dt * s->v[i][k];\n  }",
                        "for (int k = 0; k < s->dim; ++k) s->x[i][k] += dt * s->v[i][k];\n  }"),
    "kick_prior_sign": ("s->v[i][k] += dt * (s->acc[i][k] + s->aprior[i][k]);",
                        "s->v[i][k] += dt * (s->acc[i][k] - s->aprior[i][k]);"),
    "summation_without_self": (
        "      double r2 = dist2(s->x[i], s->x[j]);\n      if (r2 >= r2max) continue;\n      sig +=",
        "      if (j == i) continue;\n      double r2 = dist2(s->x[i], s->x[j]);\n"
        "      if (r2 >= r2max) continue;\n      sig +="),
    "summation_no_clamp": ("return s->rho0 * (ratio > 1.0 ? ratio : 1.0);",
                           "return s->rho0 * ratio;"),
    "kernel_exponent": ("return osph_alpha(dim, h) * t * t * t * t * (2.0 * q + 1.0);",
                        "return osph_alpha(dim, h) * t * t * t * (2.0 * q + 1.0);"),
    "key_axis_swap": ("return (uint32_t)((c[2] * s->nc[1] + c[1]) * s->nc[0] + c[0]);",
                      "return (uint32_t)((c[2] * s->nc[1] + c[0]) * s->nc[0] + c[1]);"),
    "advection_criterion": ("s->dt_ad = 0.25 * s->h /", "s->dt_ad = 0.35 * s->h /"),
    "no_riemann_average": ("if (!s->density_riemann) Us = 0.5 * (UL + UR);\n        sum += (s->m / s->rho[j])",
                           "if (!s->density_riemann) Us = 0.5 * UL;\n        sum += (s->m / s->rho[j])"),
    "blended_weight": ("return rho_sum + (excess > 0.0 ? excess : 0.0) * s->rho0 / rho_prev;",
                       "return rho_sum + (excess > 0.0 ? excess : 0.0) * rho_prev / s->rho0;"),
    "blended_branch": ("double excess = rho_prev - rho_sum;",
                       "double excess = rho_sum - rho_prev;"),
    "transport_sign": ("const double coef = -0.2 * s->h * s->h;",
                       "const double coef = 0.2 * s->h * s->h;"),
    "transport_support": ("if (s->sigma[i] < 0.95 * s->sigma0) continue;",
                          "if (s->sigma[i] < 0.5 * s->sigma0) continue;"),
    # the sampled first-step evaluations that check the full-size GPU runs
    "sample_neighbour_not_marked": ("if (dist2(s->x[i], s->x[j]) < r2max) need[j] = 1;",
                                    "if (dist2(s->x[i], s->x[j]) < r2max && j == i) need[j] = 1;"),
    "sample_state_density": ("pressure_acc_of(s, slot[user_ids[q]], rho, p, a);",
                             "pressure_acc_of(s, slot[user_ids[q]], s->rho, p, a);"),
    "sample_density_before_clamp": ("rho[k] = density_of_sigma(s, sigma_of(s, k));",
                                    "rho[k] = s->rho0 * sigma_of(s, k) / s->sigma0;"),
    "sample_sigma_slot": ("for (long q = 0; q < m; ++q) sigma[q] = sigma_of(s, slot[user_ids[q]]);",
                          "for (long q = 0; q < m; ++q) sigma[q] = sigma_of(s, user_ids[q]);"),
}


def _run_mutation(name, workdir):
    """Compile the oracle with mutation `name` planted and run the pin files
    against it; returns (anchor found, pytest return code, output tail)."""
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    if src.count(old) < 1:
        return False, None, ""
    mutated = src.replace(old, new, 1).replace(
        '#include "sph_oracle.h"', '#include "%s"' % os.path.join(ROOT, "oracle", "sph_oracle.h"))
    c = os.path.join(workdir, "sph_oracle.c")
    with open(c, "w") as fh:
        fh.write(mutated)
    so = os.path.join(workdir, "liboracle.so")
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    so, c, "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", *PIN_FILES], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    return True, r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutation_results(tmp_path_factory):
    """Every planted mistake, run concurrently (each a compiler and a pytest
    child process of its own)."""
    import concurrent.futures as cf
    names = sorted(MUTATIONS)
    dirs = {n: str(tmp_path_factory.mktemp("mut_" + n)) for n in names}
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {n: ex.submit(_run_mutation, n, dirs[n]) for n in names}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, mutation_results):
    found, code, tail = mutation_results[name]
    assert found, f"mutation anchor for {name} not found"
    assert code == 1, f"pins did not catch {name}:\n{tail}"
