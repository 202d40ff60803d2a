"""The oracle's pins catch plausible mistakes: each case plants one mistake in a temporary copy of
the oracle source (CPU only), rebuilds it, and requires at least one pin to fail on it."""
import numpy as np
import pytest

import oracle
import test_oracle_pins as pins
from fractions import Fraction
from paper_1812_07993_gb300 import workloads as W


def _pin_suite():
    return [
        ("lj_exact", lambda: pins.test_lj_matches_exact_rational(Fraction(5, 4), Fraction(3, 2),
                                                                 Fraction(11, 10))),
        ("lj_special", pins.test_lj_special_points),
        ("two_body", lambda: pins.test_two_body_force_vector_and_third_law(1.3)),
        ("two_body_close", lambda: pins.test_two_body_force_vector_and_third_law(0.95)),
        ("wall_pair", pins.test_wall_pair_uses_wall_parameters_and_acts_on_vapor_only),
        ("gradient", pins.test_force_is_minus_gradient_of_energy),
        ("net_force", pins.test_net_force_vanishes_without_walls),
        ("cells", lambda: pins.test_cell_list_equals_all_pairs_and_brute_force(0)),
        ("ballistic", pins.test_ballistic_flight_with_specular_reflection),
        ("reversibility", pins.test_time_reversibility),
        ("second_order", pins.test_velocity_verlet_energy_error_is_second_order),
        ("rescale", pins.test_rescaling_reaches_T0_exactly),
        ("berendsen", pins.test_berendsen_relation_for_general_tau),
        ("occ_cone", lambda: pins.test_occupancy_hand_placed(
            W.Pore(W.PORE_CONE, r0=3.0, r1=8.0), [[2.9, 0, -9.9], [5.4, 0, 0], [0, 7.9, 9.95]],
            [[3.2, 0, -9.9], [5.6, 0, 0], [0, 8.1, 9.95]])),
        ("occ_ink", lambda: pins.test_occupancy_hand_placed(
            W.Pore(W.PORE_INKBOTTLE, r0=3.0, r_cavity=8.0),
            [[7.9, 0, 0], [2.9, 0, 9.9], [0, 4.5, 6.5]], [[4, 0, 7.5], [8.1, 0, 0], [3.1, 0, 9.9]])),
        ("periodic_axis", pins.test_pore_offset_axis_and_periodic_image),
        ("adsorbed", pins.test_adsorbed_threshold_and_group_assignment),
        ("bins", pins.test_profile_bin_edges),
        ("pore_volume", pins.test_pore_volume_closed_forms_and_monte_carlo),
        ("pressure", pins.test_pore_pressure_kinetic_and_pair_terms),
        ("prism_ballistic", pins.test_prism_pore_ballistic_reflections_off_sides_and_floor),
        ("slab_top", pins.test_molecule_above_the_slab_reflects_off_its_top_face),
        ("hard_gas3", lambda: pins.test_hard_walls_keep_molecules_out_of_the_solid_and_conserve_energy(3)),
        ("planar_T", pins.test_planar_thermostat_uses_2n_degrees_of_freedom),
        ("prism_volume", pins.test_prism_volume_area_and_occupancy),
        ("planar_pressure", pins.test_planar_pore_pressure_divides_by_2_area),
    ]


MUTATIONS = {
    "lj force drops the factor 2": ("24.0 * eps * (2.0 * sr12 - sr6) / r2", "24.0 * eps * (sr12 - sr6) / r2"),
    "lj energy sign": ("*u = 4.0 * eps * (sr12 - sr6);", "*u = 4.0 * eps * (sr6 - sr12);"),
    "force accumulated with wrong sign": ("a->fx += fr * dx;", "a->fx -= fr * dx;"),
    "transposed pair offset": ("add_pair(&a, min_image(xi - x[3 * j], p->Lx), min_image(yi - x[3 * j + 1], p->Ly),\n               zi - x[3 * j + 2]",
                               "add_pair(&a, min_image(x[3 * j] - xi, p->Lx), min_image(x[3 * j + 1] - yi, p->Ly),\n               x[3 * j + 2] - zi"),
    "no periodic image": ("if (d > 0.5 * L) return d - L;", "if (d > 0.5 * L) return d;"),
    "energy shift added": ("a->pe_vw += u - ushift;", "a->pe_vw += u + ushift;"),
    "pair energy counted twice": ("a->pe_vv += 0.5 * (u - ushift);", "a->pe_vv += (u - ushift);"),
    "wall uses vapour epsilon": ("zi - w[3 * k + 2], rcw2, p->eps_w, p->sigma_w, usw, 1);\n    }\n    acc[i] = a;\n  }\n}\n\n/* ----",
                                 "zi - w[3 * k + 2], rcw2, p->eps, p->sigma_w, usw, 1);\n    }\n    acc[i] = a;\n  }\n}\n\n/* ----"),
    "cell list skips lower z layer": ("for (int dk = -1; dk <= 1; ++dk)", "for (int dk = 0; dk <= 1; ++dk)"),
    "drift without the half": ("+ 0.5 * a * dt * dt;", "+ a * dt * dt;"),
    "second half-kick full kick": ("v[i] = v[i] + 0.5 * (f[i] / m) * dt;", "v[i] = v[i] + (f[i] / m) * dt;"),
    "first half-kick uses a full kick": ("v[3 * i + c] = v[3 * i + c] + 0.5 * a * dt;", "v[3 * i + c] = v[3 * i + c] + a * dt;"),
    "reflection keeps the velocity": ("r[2] = p->Lz - r[2];\n    v[2] = -v[2];", "r[2] = p->Lz - r[2];\n    v[2] = v[2];"),
    "lambda without square root": ("lambda = sqrt(1.0 + (p->thermostat_every * dt / tauB) * (p->T0 / T - 1.0));",
                                   "lambda = 1.0 + (p->thermostat_every * dt / tauB) * (p->T0 / T - 1.0);"),
    "temperature with 2N degrees of freedom in 3D": ("const double dof = p->dims == 2 ? 2.0 : 3.0;", "const double dof = 2.0;"),
    "planar temperature with 3N degrees of freedom": ("const double dof = p->dims == 2 ? 2.0 : 3.0;", "const double dof = 3.0;"),
    "prism side wall keeps the velocity": ("if (dx >= P->r0) { r[0] += 2.0 * (P->r0 - dx); v[0] = -v[0]; }", "if (dx >= P->r0) { r[0] += 2.0 * (P->r0 - dx); }"),
    "prism reflected about the wrong face": ("else if (dy <= -P->r1) { r[1] += 2.0 * (-P->r1 - dy); v[1] = -v[1]; }", "else if (dy <= -P->r1) { r[1] += 2.0 * (P->r1 - dy); v[1] = -v[1]; }"),
    "prism floor ignored": ("if (r[2] <= fl) { r[2] = 2.0 * fl - r[2]; v[2] = -v[2]; }", "if (0) { r[2] = 2.0 * fl - r[2]; v[2] = -v[2]; }"),
    "slab top face reflects about the wrong side": ("const double face = r_old[2] > 0.0 ? h : -h;", "const double face = r_old[2] > 0.0 ? -h : h;"),
    "prism floor at the wrong depth": ("return (q->width > 0.0 && q->width < 2.0 * h) ? h - q->width : -2.0 * h;", "return (q->width > 0.0 && q->width < 2.0 * h) ? -h + q->width : -2.0 * h;"),
    "planar pressure divides by 3": ("pressure[q] = vol > 0.0 ? sum / ((p->dims == 2 ? 2.0 : 3.0) * vol) : 0.0;", "pressure[q] = vol > 0.0 ? sum / (3.0 * vol) : 0.0;"),
    "prism volume uses half-sides": ("return p->dims == 2 ? 2.0 * q->r0 : 4.0 * q->r0 * q->r1;", "return p->dims == 2 ? q->r0 : q->r0 * q->r1;"),
    "cone narrow end at the top": ("q->r0 + (q->r1 - q->r0) * (z + h) / (2.0 * h)", "q->r0 + (q->r1 - q->r0) * (h - z) / (2.0 * h)"),
    "ink-bottle cavity dropped": ("|| rxy2 + z * z < q->r_cavity * q->r_cavity", "&& rxy2 + z * z < q->r_cavity * q->r_cavity"),
    "adsorbed threshold not squared": ("d2wall[i] < p->r_ads * p->r_ads", "d2wall[i] < p->r_ads"),
    "bins offset by half the box the wrong way": ("floor((zi + 0.5 * p->Lz) / p->bin_width)", "floor((zi - 0.5 * p->Lz) / p->bin_width)"),
    "pressure drops the kinetic term": ("sum += p->mass * (v[3 * i] * v[3 * i]", "sum += 0.0 * (v[3 * i] * v[3 * i]"),
    "molecule virial double-counts vapour pairs": ("if (wvir) wvir[i] = acc[i].vir_vv + acc[i].vir_vw;", "if (wvir) wvir[i] = 2.0 * acc[i].vir_vv + acc[i].vir_vw;"),
    "cone volume uses the radius, not its square": ("return M_PI * R * R;", "return M_PI * R;"),
    "ink-bottle area takes the smaller disc": ("return M_PI * (c > n2 ? c : n2);", "return M_PI * (c < n2 ? c : n2);"),
    "axis distance ignores periodicity": ("double dx = min_image(xi - pores[q].cx, p->Lx), dy = min_image(yi - pores[q].cy, p->Ly);",
                                          "double dx = xi - pores[q].cx, dy = yi - pores[q].cy;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutant = src.replace(old, new, 1)
    path = oracle.build_variant(mutant, str(tmp_path / "liboracle_mutant.so"))
    failed = []
    with oracle.use_library(path):
        for pin_name, fn in _pin_suite():
            try:
                with np.errstate(all="ignore"):
                    fn()
            except (AssertionError, ValueError, FloatingPointError):
                failed.append(pin_name)
    assert failed, f"no pin caught the planted mistake: {name}"


def test_unmodified_oracle_passes_the_suite():
    for _, fn in _pin_suite():
        fn()
