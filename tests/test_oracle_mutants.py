"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of md_oracle.c (on the CPU), loads the
copy in place of the real oracle and runs the fast pins of test_oracle.py: at
least one of them must fail.  The real oracle is restored afterwards.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle as pins
from tests import test_oracle_pow as pow_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "md_oracle.c")

MUTANTS = {
    "force_sign": ("*fs = -24.0 * m->eps", "*fs = 24.0 * m->eps"),
    "dropped_attractive_force_term": ("(2.0 * sr12 - sr6) / r2", "(2.0 * sr12) / r2"),
    "newton_sign_on_j": ("fc->F[3 * j + c] -= fi[c]", "fc->F[3 * j + c] += fi[c]"),
    "minimum_image_floor": ("nearbyint(t / box[c])", "floor(t / box[c])"),
    "transposed_rotation": ("R[0][1] = 2.0 * (x * y - w * z)", "R[0][1] = 2.0 * (x * y + w * z)"),
    "quaternion_product_order": ("quat_mul(dq, q, out)", "quat_mul(q, dq, out)"),
    "energy_shift_dropped": ("- lj_energy(m->eps, m->sigma, rcut * rcut)", "- 0.0"),
    "patch_torque_sign": ("cross(pa[a], fa, tmp)", "cross(fa, pa[a], tmp)"),
    "patch_lever_of_j": ("cross(pb[b], fb, tmp)", "cross(pa[b], fb, tmp)"),
    "full_pair_energy_to_each": ("fc->E[i] += 0.5 * e", "fc->E[i] += e"),
    "half_kick_factor": ("vel[3 * i + c] += 0.5 * dt * F[3 * i + c] / mass;\n        pos",
                         "vel[3 * i + c] += dt * F[3 * i + c] / mass;\n        pos"),
    "stencil_missing_lower_cells": ("lo[c] = cl->nc[c] >= 3 ? -1 : 0", "lo[c] = 0"),
    "patch_exponent_8": ("double q5 = q * q * q * q * q;", "double q5 = q * q * q * q;"),
    "patch_force_prefactor": ("double g = 5.0 * m->eps_p / d2", "double g = 2.5 * m->eps_p / d2"),
    "squared_distance_drops_z": ("d[0] * d[0] + d[1] * d[1] + d[2] * d[2]", "d[0] * d[0] + d[1] * d[1]"),
    "rotation_angle_doubled": ("double half = 0.5 * wn * dt;", "double half = wn * dt;"),
    # the paper-form patchy model and the thermostat
    "pow_core_force_prefactor": ("*fs = -OR_POW_CORE * (*e) / r2;", "*fs = -(OR_POW_CORE - 1) * (*e) / r2;"),
    "pow_core_exponent": ("*e = pow(m->sigma / r, OR_POW_CORE);", "*e = pow(m->sigma / r, OR_POW_CORE / 2);"),
    "patch_cut_ignored": ("if (m->model == OR_PATCHY_POW && !(norm2(s) < m->patch_rc * m->patch_rc)) continue;", ""),
    "pow_uses_wca_core": ("if (m->model == OR_PATCHY_POW) pow_core(m, r2, &eiso, &fs);", "if (0) pow_core(m, r2, &eiso, &fs);"),
    "thermostat_velocity_scale": ("vel[3 * i + c] = sqrt(th->kT / mass) * nrm[c];", "vel[3 * i + c] = sqrt(th->kT * mass) * nrm[c];"),
    "thermostat_angmom_scale": ("angmom[3 * i + c] = sqrt(th->kT * inertia) * nrm[3 + c];",
                                "angmom[3 * i + c] = sqrt(th->kT / inertia) * nrm[3 + c];"),
    "thermostat_every_step": ("step > 0 && step % th->every == 0", "step > 0"),
    "thermostat_selection_inverted": ("if (!(u < th->prob)) continue;", "if (u < th->prob) continue;"),
    "box_muller_radius": ("double r = sqrt(-2.0 * log(unit_open(a)));", "double r = sqrt(-log(unit_open(a)));"),
    "philox_round_count": ("for (int r = 0; r < 10; r++) {\n    uint64_t p0", "for (int r = 0; r < 9; r++) {\n    uint64_t p0"),
    "philox_multiplier": ("(uint64_t)0xD2511F53u * c0", "(uint64_t)0xD2511F55u * c0"),
    "philox_weyl_constant": ("k0 += 0x9E3779B9u;", "k0 += 0x9E3779BBu;"),
    "philox_output_word_order": ("out[0] = c0; out[1] = c1;", "out[0] = c1; out[1] = c0;"),
    "philox_key_word_mixed": ("c2 = hi0 ^ c3 ^ k1;", "c2 = hi0 ^ c3 ^ k0;"),
}

FAST_PINS = [
    lambda: [pins.test_dimer_golden(r) for r in pins._golden_rows()],
    pins.test_lj_energy_continuous_at_cutoff,
    pins.test_lj_force_is_minus_energy_derivative_dimer,
    pins.test_newton_third_law_lj,
    pins.test_patchy_newton_and_angular_momentum_open_cluster,
    pins.test_translation_invariance,
    pins.test_patchy_dimer_closed_form,
    pins.test_patchy_energy_random_orientations_independent_numpy,
    pins.test_patchy_rotated_dimer_torque_closed_form,
    pins.test_patchy_force_and_torque_are_minus_gradients,
    lambda: [pins.test_pair_sets_brute_cells_numpy_agree(c) for c in ("lj", "noncubic")],
    pins.test_forces_brute_equal_cells,
    pins.test_nve_energy_fluctuation_scales_as_dt_squared,
    pins.test_free_rotation_matches_rodrigues,
    pins.test_patchy_nve_dt_squared,
    lambda: [pow_pins.test_core_dimer_closed_form(r) for r in (0.97, 1.03)],
    lambda: [pow_pins.test_facing_patches_closed_form(s) for s in (0.08, 0.15)],
    pow_pins.test_patch_pairs_are_truncated_at_patch_rc,
    pow_pins.test_pow_energy_independent_numpy,
    lambda: [pow_pins.test_refresh_sets_maxwell_boltzmann_momenta_from_the_draws(k) for k in ("lj", "pow")],
    pow_pins.test_refresh_probability_and_schedule,
    pow_pins.test_thermostat_normals_are_standard,
    pow_pins.test_philox_known_answer_vectors,
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(before, after))
    lib = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib),
                           str(mut), "-lm"])
    caught = []
    try:
        oracle.load_library(str(lib))
        for pin in FAST_PINS:
            try:
                pin()
            except (AssertionError, MemoryError, FloatingPointError):
                caught.append(getattr(pin, "__name__", "pin"))
                break
    finally:
        oracle.load_library(None)
    assert caught, f"no pin caught the planted mistake {name!r}"
