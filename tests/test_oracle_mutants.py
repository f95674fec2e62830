"""The pins are strong enough to catch plausible mistakes in the oracle.

Each case copies the oracle's C source, plants one mistake (a dropped term, a
wrong sign, index or factor, a transposed operand), builds it on the CPU and
runs a fast subset of the pins against it: at least one pin must fail.  The
committed oracle is never modified.
"""
import importlib.util
import os
import shutil
import subprocess
import tempfile

import pytest

import test_oracle_algebra as A
import test_oracle_bruteforce as B
import test_oracle_diagnostics as Dg
import test_oracle_physics as Ph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tlbm_oracle.c")

MUTANTS = {
    "guo_sign": ("Ft[i] = v->w[i] * (3.0 * emuF + 9.0 * eu * eF);", "Ft[i] = v->w[i] * (3.0 * emuF - 9.0 * eu * eF);"),
    "no_half_source": ("src[k] = (1.0 - 0.5 * s->S[k]) * MF[k];", "src[k] = MF[k];"),
    "feq_coefficient": ("4.5 * eu * eu", "4.0 * eu * eu"),
    "bounce_back_direction": ("s->f[i * N + n] = s->fp[s->fs.opp[i] * N + n];", "s->f[i * N + n] = s->fp[i * N + n];"),
    "anti_bounce_back_sign": ("s->g[i * N + n] = -gb + s->omega * Tw;", "s->g[i * N + n] = gb + s->omega * Tw;"),
    "full_force_in_velocity": ("u[a] = (m[a] + 0.5 * F[a]) / r;", "u[a] = (m[a] + F[a]) / r;"),
    "transposed_inverse": ("a += fs->Minv[i][k] * dm[k];", "a += fs->Minv[k][i] * dm[k];"),
    "thermal_equilibrium": ("neq[3] = a_T * T;", "neq[3] = T;"),
    "buoyancy_axis": ("int gax = s->dim == 2 ? 1 : 2;", "int gax = 0;"),
    "pull_sign": ("src[a] = c[a] - s->fs.e[i][a];", "src[a] = c[a] + s->fs.e[i][a];"),
    "viscosity_mapping": ("double snu = 1.0 / (3.0 * s->nu + 0.5);", "double snu = 1.0 / (3.0 * s->nu + 1.0);"),
    "diffusivity_mapping": ("double qj = 1.0 / (s->alpha / s->omega + 0.5);",
                            "double qj = 1.0 / (s->alpha / s->omega + 1.0);"),
    "d3q19_row": ("case 4: return (5.0 * e2 - 9.0) * ex;", "case 4: return (5.0 * e2 - 8.0) * ex;"),
    "energy_half": ("e += 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);",
                    "e += r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);"),
    "mass_sum": ("m += r;", "m += t;"),
    "nusselt_scale": ("return 1.0 + L * (sum / (double)s->N) / (s->alpha * dT);",
                      "return 1.0 + 0.5 * L * (sum / (double)s->N) / (s->alpha * dT);"),
}


def _pins(O):
    """Fast pins (about a second in total); each returns normally or raises."""
    return [
        lambda: A.test_forcing_moments_match_printed_eq6(O, 0, "D2Q9", 9),
        lambda: A.test_forcing_moments_match_printed_eq6(O, 1, "D3Q19", 19),
        lambda: A.test_d2q9_meq_closed_form(O),
        lambda: A.test_d3q19_meq_closed_form(O),
        lambda: A.test_antibounceback_omega_is_twice_moving_weight(O, 0, "D2Q5"),
        lambda: A.test_thermal_equilibrium_moments(O, 0),
        lambda: A.test_relaxation_rates_defaults(O),
        lambda: A.test_moment_matrix_orthogonal_and_inverse(O, 2),
        lambda: Ph.test_pure_conduction_is_exact(O, 0, (8, 32, 1), 0),
        lambda: Ph.test_poiseuille_exact_at_magic_parameter(O, 0, 9),
        lambda: Ph.test_thermal_mode_decay(O, 0),
        lambda: Ph.test_shear_wave_decay(O, 0),
        lambda: Ph.test_mass_conserved_to_roundoff(O, 0, (65, 33, 1)),
        lambda: B.test_one_step_pull_equals_push(O, 0, (4, 5, 1), 0, 0),
        lambda: B.test_one_step_pull_equals_push(O, 1, (5, 4, 3), 0, 0),
        lambda: Ph.test_buoyancy_enters_the_velocity_along_gravity(O, 0, (9, 12, 1)),
        lambda: Ph.test_nusselt_of_a_uniform_flow(O, 0),
        lambda: Dg.test_energy_and_mass_of_a_given_state(O, 0, (23, 17, 1)),
    ]


def _load_mutant(tmp, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation site for {name} not found"
    msrc = os.path.join(tmp, "tlbm_oracle.c")
    with open(msrc, "w") as fh:
        fh.write(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "tlbm_oracle.h"), tmp)
    lib = os.path.join(tmp, f"libmutant_{name}.so")
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", msrc, "-o", lib,
                    "-lm"], check=True)
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", os.path.join(ROOT, "oracle", "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._LIB = lib
    mod.build = lambda force=False: lib
    return mod


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_a_planted_mistake_fails_a_pin(name):
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as tmp:
        Om = _load_mutant(tmp, name, old, new)
        caught = []
        for k, pin in enumerate(_pins(Om)):
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError):
                caught.append(k)
        assert caught, f"no pin caught the mutant {name}"


def test_unmutated_oracle_passes_the_fast_pins(O):
    for pin in _pins(O):
        pin()
