"""The pins are strong enough: each plausible mistake planted in a copy of
the oracle (a dropped term, a wrong sign, index or coefficient, a transposed
operand) is compiled on the CPU and must make a named pin fail.

The mistakes live only in temporary copies of nyx_oracle.c; the oracle in
the tree is never modified."""
import os
import subprocess

import pytest

import oracle
import test_oracle_amr as ta
import test_oracle_flattening as tf
import test_oracle_gravity as tg
import test_oracle_pm as tpm
import test_oracle_poisson as tps
import test_oracle_ppm as tp
import test_oracle_riemann as tr
import test_oracle_step as ts
import test_oracle_trace as tt
import test_oracle_variants as tv

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "nyx_oracle.c")

# name: (text in nyx_oracle.c, replacement, pin that must fail, pin arguments)
MUTANTS = {
    "pdV term dropped from rho e": ("- ahdt * pdivu", "- 0.0 * pdivu",
                                    ts.test_internal_energy_tracks_total_minus_kinetic, ()),
    "gravity source sign in tracing": ("src->hdtp * g3[d]", "src->hdtp * (-g3[d])",
                                       tt.test_gravity_shifts_edge_velocity_by_half_step, ()),
    "corrector without the 1/2": ("rEn = rE_s + s->hdt *", "rEn = rE_s + s->dt *",
                                  ts.test_uniform_gravity_at_rest, ()),
    "PPM interface coefficient": ("(d1 - d0) * SIXTH", "(d1 - d0) * 0.2",
                                  tp.test_unlimited_interface_exact_for_cubic_averages, ()),
    "PPM extremum not flattened": ("if ((sR - si) * (si - sL) <= 0.0)",
                                   "if ((sR - si) * (si - sL) < -1e300)",
                                   tp.test_local_extremum_is_flattened, ()),
    "PPM integral curvature term": ("(1.0 - TWO_THIRDS * sig)", "(1.0 - 0.5 * sig)",
                                    tp.test_integrals_are_averages_of_the_parabola, ()),
    "shock sampled on the wrong side": ("star = (s * S < 0.0);", "star = (s * S > 0.0);",
                                        tr.test_supersonic_upwinding, ()),
    "tangential velocity from the other slot": ("  g[2] = qo[2];", "  g[2] = qo[3];",
                                                tr.test_contact_only, ()),
    "energy flux without p u": ("out[4] = ug * (rhoeg + ke + pg);", "out[4] = ug * (rhoeg + ke);",
                                tr.test_supersonic_upwinding, ()),
    "rarefaction fan weight from the wrong edge (w <-> 1 - w)": (
        "w = (0.0 - H) / (T - H);", "w = (0.0 - T) / (H - T);",
        tr.test_transonic_rarefaction_fan_is_continuous_and_linear, ()),
    "u* = 0 takes the left side instead of the mean": (
        "for (int v = 0; v < 5; ++v) g[v] = 0.5 * (gl[v] + gr[v]);",
        "for (int v = 0; v < 5; ++v) g[v] = gl[v];",
        tr.test_stationary_contact_face_takes_the_mean_of_both_sides, ()),
    "Newton step sign": ("double pn = p - ZL * ZR", "double pn = p + ZL * ZR",
                         tr.test_symmetric_collision_closed_form, (1.4, 1.0)),
    "shock curve constant (gamma+1 -> gamma-1)": (
        "e.kshock = (p->gamma + 1.0) / (2.0 * p->gamma);",
        "e.kshock = (p->gamma - 1.0) / (2.0 * p->gamma);",
        tr.test_symmetric_collision_closed_form, (1.4, 1.0)),
    "expansion drag sign": ("0.5 * adot;", "-0.5 * adot;",
                            tt.test_expansion_sources_on_uniform_state, ()),
    "entropy-wave amplitude sign": ("double b0 = dq[1][0] - dq[1][4] * ic2;",
                                    "double b0 = dq[1][0] + dq[1][4] * ic2;",
                                    tt.test_acoustic_simple_wave_linear_limit, ()),
    "acoustic velocity term sign": ("q[v] = ref[v] - cor * (bp - bm);",
                                    "q[v] = ref[v] - cor * (bp + bm);",
                                    tt.test_acoustic_wave_in_supersonic_flow, ()),
    "corner coupling theta 1/3 -> 1/2": ("cdt = dtp / (3.0 * dx[t])", "cdt = dtp / (2.0 * dx[t])",
                                         ts.test_trilinear_advection_exact, ()),
    "final-state theta 1/2 -> 1/4": ("c1 = 0.5 * dtp / dx[t1], c2 = 0.5 * dtp / dx[t2]",
                                     "c1 = 0.25 * dtp / dx[t1], c2 = 0.25 * dtp / dx[t2]",
                                     ts.test_trilinear_advection_exact, ()),
    "momentum weighted by a_new": ("(a_old * m[c] - dt * div[1 + c]",
                                   "(a_new * m[c] - dt * div[1 + c]",
                                   ts.test_uniform_state_under_expansion, ()),
    "divergence reads the x neighbour": ("(Ff[d][c * V + id + g.st[d]] - Ff[d][c * V + id])",
                                         "(Ff[d][c * V + id + g.st[0]] - Ff[d][c * V + id])",
                                         ts.test_flux_export_reproduces_density_update, ()),
    "dual-energy switch reversed": ("if (rEn - ke > s->eta_de * rEn)",
                                    "if (rEn - ke < s->eta_de * rEn)",
                                    ts.test_dual_energy_switch_direction, (5e-5, True)),
    "pressure from rho E instead of rho e": ("double p = E->gm1 * S[5 * vol + id];",
                                             "double p = E->gm1 * S[4 * vol + id];",
                                             ts.test_dt_closed_form_uniform, ()),
    "CFL step without a": ("double t = a * dx[d] / (fabs(q6[1 + d]) + q6[5]);",
                           "double t = dx[d] / (fabs(q6[1 + d]) + q6[5]);",
                           ts.test_dt_closed_form_uniform, ()),
    "periodic wrap off by one": ("x = dlo[d] + ((x - dlo[d]) % len + len) % len;",
                                 "x = dlo[d] + ((x - dlo[d] + 1) % len + len) % len;",
                                 ts.test_ghost_fill_periodic_outflow_and_tiles, ()),
    # dark matter
    "cloud-in-cell weights swapped": ("  *w0 = 1.0 - (s - fl);", "  *w0 = s - fl;",
                                      tpm.test_deposit_centre_and_corner, ()),
    "deposit without 1/dx^3": ("      rho[id] = rho[id] + m[p] * w * iv;", "      rho[id] = rho[id] + m[p] * w;",
                               tpm.test_deposit_conserves_mass, ()),
    "kick with the whole dt": ("const double uh = (a_old * u[c * np + p] + 0.5 * dt * gp[c]) / a_half;",
                               "const double uh = (a_old * u[c * np + p] + dt * gp[c]) / a_half;",
                               tpm.test_kdk_uniform_field_at_unit_scale_factor, ()),
    "drift divided by a_old": ("double xn = xp[c] + dt / a_half * uh;", "double xn = xp[c] + dt / a_old * uh;",
                               tpm.test_free_streaming_under_expansion_and_periodic_wrap, ()),
    # self-gravity
    "smoother weight 1/7": ("g->phi[id] = (mg_nbsum(g, i, j, k) - g->h2 * g->f[id]) * SIXTH;",
                            "g->phi[id] = (mg_nbsum(g, i, j, k) - g->h2 * g->f[id]) / 7.0;",
                            tps.test_single_mode_closed_form, ()),
    "residual stencil centre 5": ("(mg_nbsum(g, i, j, k) - 6.0 * g->phi[id]) * g->ih2",
                                  "(mg_nbsum(g, i, j, k) - 5.0 * g->phi[id]) * g->ih2",
                                  tps.test_single_mode_closed_form, ()),
    "coarse grid spacing not doubled": ("      h *= 2.0;", "      h *= 1.0;",
                                        tps.test_residual_tolerance_warm_start_and_convergence_rate,
                                        ()),
    "gravity without the 1/2": ("const double hdx = 0.5 / dx;", "const double hdx = 1.0 / dx;",
                                tps.test_single_mode_closed_form, ()),
    # PLM and the linearised solver
    "PLM edge at a quarter slope": ("*sRo = s[2] + 0.5 * d;", "*sRo = s[2] + 0.25 * d;",
                                    tv.test_plm_traced_density_closed_form, ()),
    "PLM slope from the upwind cells": ("double d = mc_slope(s[1], s[2], s[3]);",
                                        "double d = mc_slope(s[0], s[1], s[2]);",
                                        tv.test_plm_traced_density_closed_form, ()),
    "linearised star density sign": ("? qo[0] + (pstar - qo[4]) / (co * co)",
                                     "? qo[0] - (pstar - qo[4]) / (co * co)",
                                     tv.test_sod_with_the_linearised_solver, ()),
    "linearised solver iterates anyway": ("(E->linear ? 0 : E->max_iter)", "(E->max_iter)",
                                          tv.test_linearised_symmetric_collision_closed_form, ()),
    # gravity source variants
    "corrector uses g^n for the new density": ("(rho_s * gn[c] - rho * go[c])",
                                                "(rho_s * go[c] - rho * go[c])",
                                                tg.test_uniform_gas_at_rest_with_new_gravity, (0,)),
    "option (ii) predictor sign": ("0.5 * (ks - kh) / rho_s", "0.5 * (kh - ks) / rho_s",
                                   tg.test_option_two_leaves_internal_energy_to_the_hydro, ()),
    "option (ii) corrector adds the whole kinetic energy": ("rEn = rE_s + 0.5 * (kn - ks) / rho_s;",
                                                            "rEn = rE_s + 0.5 * kn / rho_s;",
                                                            tg.test_uniform_gas_at_rest_with_new_gravity,
                                                            (1,)),
    # coarse-fine coupling
    "reflux sign flipped": ("*U = high ? *U + corr : *U - corr;",
                            "*U = high ? *U - corr : *U + corr;",
                            ta.test_two_level_step_conserves_only_with_reflux, (True,)),
    "reflux against the covered cell's face": ("if (!high) cf[d] += 1;", "if (high) cf[d] += 1;",
                                               ta.test_two_level_step_conserves_only_with_reflux,
                                               (True,)),
    "fine fluxes from the opposite face": ("const int ffi = high ? fn[d] : 0;",
                                           "const int ffi = high ? 0 : fn[d];",
                                           ta.test_two_level_step_conserves_only_with_reflux,
                                           (True,)),
    "interpolation offset 1/2": ("const double xo = o[0] ? 0.25 : -0.25",
                                 "const double xo = o[0] ? 0.5 : -0.5",
                                 ta.test_interp_reproduces_linear_data, ()),
    "one-sided interpolation slope": ("s[d] = mc_slope(um, uc, up);", "s[d] = mc_slope(uc, uc, up);",
                                      ta.test_interp_reproduces_linear_data, ()),
    "extrema limiter off": ("  double alpha = 1.0;\n  if (dev > 0.0) {",
                            "  double alpha = 1.0;\n  if (dev < 0.0) {",
                            ta.test_interp_is_conservative_and_makes_no_new_extrema, ()),
    "average down over 4 cells": ("cstate[cb][c * gc.vol + cid] = 0.125 * s;",
                                  "cstate[cb][c * gc.vol + cid] = 0.25 * s;",
                                  ta.test_average_down_undoes_interpolation, ()),
    "fine ghosts never copied from fine neighbours": ("          if (region == 1) {\n            const int sb",
                                                      "          if (region == 2) {\n            const int sb",
                                                      ta.test_fine_ghosts_take_fine_neighbours_first, ()),
    "flattening takes the high-pressure neighbour": (
        "ptrdiff_t t = (pr[s] - pr[-s] > 0.0) ? -s : s;", "ptrdiff_t t = (pr[s] - pr[-s] > 0.0) ? s : -s;",
        tf.test_two_cell_shock_flattens_the_shock_and_the_cell_behind_it, ()),
    "shock test at half the lower pressure": ("fabs(dp1) > FLAT_EPS * lo", "fabs(dp1) > 0.5 * lo",
                                              tf.test_pressure_jump_threshold_is_a_third,
                                              (0.34, True)),
    "shock test on diverging flow": ("if (!(u[-s] - u[s] > 0.0)) return 0.0;",
                                     "if (!(u[-s] - u[s] < 0.0)) return 0.0;",
                                     tf.test_two_cell_shock_flattens_the_shock_and_the_cell_behind_it,
                                     ()),
    "steepness ramp slope 5": ("double w = FLAT_OMEGA2 * (z - FLAT_OMEGA1);",
                               "double w = 5.0 * (z - FLAT_OMEGA1);",
                               tf.test_partial_flattening_closed_form, ()),
    "curvature not flattened": ("s6[v] = fl * s6[v];", "s6[v] = s6[v];",
                                tf.test_traced_deviation_scales_with_the_coefficient, (0, 0)),
    "flattening from the z direction only": ("if (fd > f) f = fd;", "if (d == 2) f = fd;",
                                             tf.test_each_direction_uses_its_own_line, (0,)),
    "flattening reads u_x in every direction": ("q + (size_t)(1 + d) * V + id", "q + (size_t)1 * V + id",
                                                tf.test_each_direction_uses_its_own_line, (1,)),
}


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(name, mutant_dir):
    old, new, pin, args = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old}"
    tag = str(abs(hash(name)))
    c = os.path.join(mutant_dir, f"m{tag}.c")
    so = os.path.join(mutant_dir, f"m{tag}.so")
    with open(c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-I", os.path.dirname(SRC), "-o", so, c, "-lm"], check=True)
    pin(*args)  # the pin passes on the oracle itself
    with oracle.use_library(so):
        with pytest.raises(AssertionError):
            pin(*args)
