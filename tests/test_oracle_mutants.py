"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/mc_oracle.c (a dropped
factor, a wrong sign, an off-by-one, a missing update), builds it on the CPU
into a temporary library and runs the pin that should catch it in a
subprocess with ORACLE_LIB pointing at the mutant; the pin must fail.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mc_oracle.c")

# (mistake, original text, planted text, occurrence to replace, pin)
MUTANTS = [
    ("Thomson opacity without the Doppler factor", "const double k = g->kappa[s] * D;",
     "const double k = g->kappa[s];", 1,
     "tests/test_oracle_closed_forms.py::test_thomson_opacity_doppler_factor"),
    ("J estimator without D", "res->j_est[s] += (e_cmf * l) * D;", "res->j_est[s] += (e_cmf * l);", 1,
     "tests/test_oracle_closed_forms.py::test_free_streaming_estimators_at_finite_velocity"),
    ("optical depth not reduced by a passed line", "tau_rem = tau_rem - tau_line;",
     "tau_rem = tau_rem;", 1,
     "tests/test_oracle_closed_forms.py::test_second_line_absorbs_with_its_own_depth"),
    ("electron scattering only forward", "const double mu2 = -1.0 + 2.0 * rng_closed0(r);",
     "const double mu2 = rng_closed0(r);", 1,
     "tests/test_oracle_transport.py::test_thin_electron_slab_back_fraction"),
    ("J_blue without 1/nu", "((pk->e_lab * d_res) * d_res) / nu_line[j]",
     "((pk->e_lab * d_res) * d_res)", 1,
     "tests/test_oracle_closed_forms.py::test_j_blue_is_dilute_blackbody_in_free_streaming"),
    ("Boltzmann factor sign", "double b = orc_exp(-(eps / kT));", "double b = orc_exp((eps / kT));", 1,
     "tests/test_oracle_plasma.py::test_populations_sum_and_boltzmann_ratios"),
    ("dilution applied to metastable levels", "(lte_excitation || metastable[a]) ? 1.0 : w[s]",
     "(lte_excitation || !metastable[a]) ? 1.0 : w[s]", 1,
     "tests/test_oracle_plasma.py::test_populations_sum_and_boltzmann_ratios"),
    ("zeta(5) dropped from Eq. 15", "(360.0 * ZETA5)", "(360.0)", 1,
     "tests/test_oracle_plasma.py::test_radiation_field_update_inverts_planck_mean"),
    ("Planck series index off by one", "if (planck_cdf[i] >= z0) { l = i; break; }",
     "if (planck_cdf[i] >= z0) { l = i + 1; break; }", 1,
     "tests/test_oracle_injection.py::test_planck_sampler_mean_and_shape"),
    ("direction after the move flipped", "double mun = pl / xn;", "double mun = -pl / xn;", 1,
     "tests/test_oracle_transport.py::test_events_conserve_comoving_energy_and_hit_sobolev_point"),
    ("spectrum bin off by one", "    spec[b] += e_lab;", "    spec[b > 0 ? b - 1 : 0] += e_lab;", 1,
     "tests/test_oracle_injection.py::test_free_streaming_recovers_injection_exactly"),
    ("lab frequency multiplied instead of divided by D", "pk->nu_lab = nu_cmf / D;",
     "pk->nu_lab = nu_cmf * D;", 1, "tests/test_oracle_injection.py::test_injection_state"),
    ("geometric dilution from the inverse ratio", "double rr = x_i / x_mid;",
     "double rr = x_mid / x_i;", 1,
     "tests/test_oracle_plasma.py::test_geometric_dilution_is_solid_angle_fraction"),
    ("Eq. 19 weight with 1 + mu_min", "(e_cmf * (1.0 - mu_min)) / (2.0 * (double)nv)",
     "(e_cmf * (1.0 + mu_min)) / (2.0 * (double)nv)", 1,
     "tests/test_oracle_virtual.py::test_scattering_model_v_and_r_spectra_agree_and_v_is_less_noisy"),
    ("v-packet energy left in the comoving frame", "(e_v / D) * orc_exp(-tau)", "e_v * orc_exp(-tau)", 1,
     "tests/test_oracle_virtual.py::test_free_streaming_total_matches_closed_form"),
    ("v-packet depth without electron scattering", "        tau += kv * d_shell;",
     "        tau += 0.0 * d_shell;", 1,
     "tests/test_oracle_virtual.py::test_radial_electron_optical_depth"),
    ("v-packet line depth from the neighbouring shell",
     "tau += m->tau[(size_t)s * (size_t)L + (size_t)j];",
     "tau += m->tau[(size_t)(s > 0 ? s - 1 : s + 1) * (size_t)L + (size_t)j];", 1,
     "tests/test_oracle_virtual.py::test_single_line_depth_counts_only_in_its_shell"),
    ("v-packets drawing from the r-packet stream", "transport(m, g, &r, virt ? &rv : NULL,",
     "transport(m, g, &r, virt ? &r : NULL,", 1,
     "tests/test_oracle_virtual.py::test_r_packets_unchanged_by_virtual_packets"),
    ("v-packet directions only outward", "const double mu_min = -sqrt(arg);",
     "const double mu_min = sqrt(arg);", 1,
     "tests/test_oracle_virtual.py::test_scattering_model_v_and_r_spectra_agree_and_v_is_less_noisy"),
    ("macro atom deactivates from the activated level", "        row = next;\n",
     "        (void)next;\n", 1,
     "tests/test_oracle_macroatom.py::test_walks_match_the_absorbing_markov_chain"),
    ("macro-atom jump decision inverted", "if (!(za < m->ma_jump_p[row])) break;",
     "if (za < m->ma_jump_p[row]) break;", 1,
     "tests/test_oracle_macroatom.py::test_walks_match_the_absorbing_markov_chain"),
    ("nebular ratio without (T_e/T_R)^(1/2)", "const double neb = (mode == 2) ? sqrt(0.9) : 1.0;",
     "const double neb = 1.0;", 1,
     "tests/test_oracle_ionization.py::test_hydrogen_like_element_matches_the_saha_quadratic"),
    ("Saha ratio with the partition functions inverted", "((2.0 * Z[j + 1]) / Z[j])",
     "((2.0 * Z[j]) / Z[j + 1])", 1,
     "tests/test_oracle_ionization.py::test_hydrogen_like_element_matches_the_saha_quadratic"),
    ("charge counted one stage low", "for (int32_t j = 1; j < J; ++j) ce += (double)j * f[j];",
     "for (int32_t j = 1; j < J; ++j) ce += (double)(j - 1) * f[j];", 1,
     "tests/test_oracle_ionization.py::test_element_and_charge_conservation"),
    ("macro-atom jump target off by one", "if (zb < m->ma_jump_cdf[k]) { next = m->ma_jump_target[k]; break; }",
     "if (zb < m->ma_jump_cdf[k]) { next = m->ma_jump_target[k > b ? k - 1 : k]; break; }", 1,
     "tests/test_oracle_macroatom.py::test_walks_match_the_absorbing_markov_chain"),
    ("T_inner update with a square root instead of a fourth root",
     "return t_inner * sqrt(sqrt(l_requested / l_emitted));", "return t_inner * sqrt(l_requested / l_emitted);", 1,
     "tests/test_oracle_luminosity.py::test_one_update_reaches_the_requested_luminosity_in_free_streaming"),
    ("Eq. 18 with r instead of r^2", "double x = l_outer / ((((4.0 * PI_D) * r_inner) * r_inner) * SIGMA_SB);",
     "double x = l_outer / (((4.0 * PI_D) * r_inner) * SIGMA_SB);", 1,
     "tests/test_oracle_luminosity.py::test_eq18_inverts_the_inner_luminosity"),
]


@pytest.mark.parametrize("name,orig,planted,count,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(name, orig, planted, count, pin):
    src = open(SRC).read()
    assert src.count(orig) >= 1, f"pattern not found: {orig}"
    mutated = src.replace(orig, planted, count)
    with tempfile.TemporaryDirectory() as d:
        c_path = os.path.join(d, "mutant.c")
        so_path = os.path.join(d, "mutant.so")
        with open(c_path, "w") as f:
            f.write(mutated)
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                        "-o", so_path, c_path, "-lm"], check=True)
        env = dict(os.environ, ORACLE_LIB=so_path)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", pin],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"pin {pin} did not catch: {name}\n{r.stdout[-2000:]}"
