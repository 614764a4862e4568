"""Planted mistakes: the oracle's pins catch plausible errors (no GPU).

Each case copies one of the oracle's sources -- the C file, ``lsm.py`` or
``analytic.py`` -- and plants one mistake of the kind a careful reader could
make: a dropped term, a flipped sign, a wrong index or word, a mistyped digit,
a wrong divisor.  The copy is built on the CPU in a temporary directory,
swapped in for this one test, and the pin named beside the mistake must now
fail.  The shipped oracle is never modified.

Every site is matched verbatim and must occur exactly once, so a later edit of
the oracle that moves a site fails here loudly instead of planting nothing.
"""
from __future__ import annotations

import os
import types

import numpy as np
import pytest

import oracle
from oracle import analytic, lsm
import test_oracle_basket as basket_pins
import test_oracle_lsm as lsm_pins
import test_oracle_pins as pins
import test_oracle_qem as qem_pins

CFG = pins.CFG


def _price_pin(is_put):
    return lambda: pins.test_price_matches_heston_semi_analytic(CFG, 64, is_put)


def _cir_pin(v):
    return lambda: pins.test_qe_step_matches_cir_conditional_moments(v)


def _log_spot_pin():
    return lambda: pins.test_log_spot_mean_and_martingale("cfg", None, pins.cfg_paths())


def _log_spot_hard_pin():
    return lambda: pins.test_log_spot_mean_and_martingale("hard", pins.hard_paths(), None)


# (name, site, planted, pin that must fail) in simr_oracle.c
C_MISTAKES = [
    # Philox4x32-10: round count, key schedule, S-box output words
    ("philox_nine_rounds", "for (int round = 0; round < 10; ++round)", "for (int round = 0; round < 9; ++round)",
     pins.test_philox_matches_triton_library),
    ("philox_key_schedule", "k1 += weyl1;", "k1 += weyl0;", pins.test_philox_matches_triton_library),
    ("philox_sbox_words", "uint32_t y1 = lo1;", "uint32_t y1 = lo0;", pins.test_philox_matches_triton_library),
    # counter -> uniforms
    ("uniform_offset", "((double)(w >> 9) + 0.5) * 0x1p-23", "((double)(w >> 9) + 1.0) * 0x1p-23",
     pins.test_step_uniform_mapping),
    ("odd_step_reuses_even_words", "*u_v = oracle_uniform(w[2]);\n    *u_x = oracle_uniform(w[3]);",
     "*u_v = oracle_uniform(w[0]);\n    *u_x = oracle_uniform(w[1]);", _log_spot_pin()),
    # inverse normal (AS 241)
    ("norminv_coefficient_digits", "4.5921953931549871457e+4", "4.5921953913549871457e+4",
     pins.test_norminv_against_scipy_and_cdf),
    ("norminv_tail_sign", "return (q < 0.0) ? -val : val;", "return (q > 0.0) ? -val : val;",
     pins.test_norminv_against_scipy_and_cdf),
    ("norminv_tail_split", "if (r <= 5.0) {", "if (r <= 2.0) {", pins.test_norminv_against_scipy_and_cdf),
    # QE variance step (Andersen 2008)
    ("qe_decay_over_T", "double E = exp(-m->kappa * dt);", "double E = exp(-m->kappa * m->T);", _cir_pin(0.04)),
    ("qe_c1_drops_E", "out[2] = s2 * E * (1.0 - E) / m->kappa;", "out[2] = s2 * (1.0 - E) / m->kappa;",
     _cir_pin(0.2)),
    ("qe_c2_drops_half", "(1.0 - E) * (1.0 - E) / (2.0 * m->kappa);", "(1.0 - E) * (1.0 - E) / m->kappa;",
     _cir_pin(0.001)),
    ("qe_b2_root_sign", "    double b2 = two_over_psi - 1.0 + sqrt(two_over_psi)",
     "    double b2 = two_over_psi - 1.0 - sqrt(two_over_psi)", _cir_pin(0.04)),
    ("qe_beta_sign", "  double beta = (1.0 - p) / m;", "  double beta = (1.0 + p) / m;", _cir_pin(0.001)),
    ("qe_exponential_inverse", "return log((1.0 - p) / (1.0 - u_v)) / beta;", "return log((1.0 - p) / u_v) / beta;",
     _cir_pin(0.001)),
    ("qe_atom_threshold", "if (u_v <= p) {\n    *branch = 2;", "if (u_v <= 1.0 - p) {\n    *branch = 2;",
     _cir_pin(0.001)),
    # log-spot step constants and update
    ("K0_rho_sign", "out[4] = -m->rho * m->kappa", "out[4] = m->rho * m->kappa", _log_spot_hard_pin()),
    ("K0_drops_rate", "/ m->sigma + m->r * dt;", "/ m->sigma;", _log_spot_pin()),
    ("K1_rho_sign", "- 0.5) - m->rho / m->sigma;", "- 0.5) + m->rho / m->sigma;", _log_spot_pin()),
    ("K3_rho_sign", "out[7] = GAMMA1 * dt * (1.0 - m->rho * m->rho);",
     "out[7] = GAMMA1 * dt * (1.0 + m->rho * m->rho);", _log_spot_pin()),
    ("log_spot_v_for_vnext", "x += k0 + k[5] * v + k[6] * v_next", "x += k0 + k[5] * v + k[6] * v",
     _log_spot_pin()),
    ("log_spot_variance_drops_vnext", "sqrt(k[7] * v + k[8] * v_next) * z_x", "sqrt(k[7] * v) * z_x",
     _log_spot_pin()),
    ("log_spot_normal_from_variance_uniform", "double z_x = oracle_norminv(u_x);\n    const double k0",
     "double z_x = oracle_norminv(u_v);\n    const double k0", _price_pin(False)),
    # payoff, discounting, standard error
    ("payoff_call_put_swapped", "double d = is_put ? (K - s_T) : (s_T - K);",
     "double d = is_put ? (s_T - K) : (K - s_T);", pins.test_put_call_parity_on_common_paths),
    ("price_not_discounted", "price[j] = disc * mean;", "price[j] = mean;", pins.test_put_call_parity_on_common_paths),
    ("stderr_from_first_moment", "s2 += f * f;", "s2 += f;", pins.test_standard_error_matches_the_spread_over_seeds),
    ("stderr_without_sample_size", "(s2 / (double)paths - mean * mean) / (double)(paths - 1)",
     "(s2 / (double)paths - mean * mean)", pins.test_standard_error_matches_the_spread_over_seeds),
    # bump-and-revalue Greeks
    ("fd_one_sided_divisor", "d = (tmp_up[j] - tmp_dn[j]) / (2.0 * h);", "d = (tmp_up[j] - tmp_dn[j]) / h;",
     pins.test_fd_theta_against_semi_analytic),
    ("fd_theta_sign", "double sign = ((1u << b) == G_THETA) ? -1.0 : 1.0;", "double sign = 1.0;",
     pins.test_fd_theta_against_semi_analytic),
    ("fd_gamma_divisor", "g[j] = (up[j] - 2.0 * price[j] + dn[j]) / (h * h);",
     "g[j] = (up[j] - 2.0 * price[j] + dn[j]) / (2.0 * h * h);", pins.test_fd_greeks_against_semi_analytic),
    ("fd_vega_bumps_theta", "static const int field[9] = {0, 0, 3, 2, 1, 4, 5, 6, 7};",
     "static const int field[9] = {0, 0, 5, 2, 1, 4, 3, 6, 7};", pins.test_fd_greeks_against_semi_analytic),
    # reverse-mode adjoint, forward-mode duals, pathwise price sensitivities
    ("adjoint_drops_diffusion_term", "double bar_vcur = K1 + K3 * dsq;", "double bar_vcur = K1;",
     pins.test_reverse_mode_matches_forward_mode_duals),
    ("adjoint_exponential_branch_sign", "double dv_dq = (mm / (q * q)) * (1.0 - L);",
     "double dv_dq = (mm / (q * q)) * (1.0 + L);", pins.test_reverse_mode_matches_forward_mode_duals),
    ("adjoint_sigma_map", "grad5[3] = bar_c1 * 2.0 * c1 / sig", "grad5[3] = bar_c1 * c1 / sig",
     pins.test_reverse_mode_matches_forward_mode_duals),
    ("adjoint_kappa_map_sign", "s2g * ((1.0 - 2.0 * E) * dE_dk / kap - E * (1.0 - E) / (kap * kap))",
     "s2g * ((1.0 - 2.0 * E) * dE_dk / kap + E * (1.0 - E) / (kap * kap))",
     pins.test_reverse_mode_matches_forward_mode_duals),
    ("adjoint_theta_through_mean", "bar_th += bar_m * (1.0 - E);", "bar_th += bar_m * E;",
     pins.test_reverse_mode_matches_forward_mode_duals),
    ("dual_quotient_rule", "(a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v)", "(a.d[i] * b.v + a.v * b.d[i]) / (b.v * b.v)",
     pins.test_reverse_mode_matches_forward_mode_duals),
    ("dual_sqrt_rule", "a.d[i] / (2.0 * r.v)", "a.d[i] / r.v", pins.test_reverse_mode_matches_forward_mode_duals),
    ("adjoint_delta_weight", "s[0] += w / m->S0;", "s[0] += w;", pins.test_adjoint_matches_fd_and_closed_form_delta),
    # the decision taken the other way: the reverse sweep must impose it where the forward did
    ("flip_reverse_keeps_natural_branch", "if (n == f_step && f_kind == 1) quad = f_value;", "",
     lambda: pins.test_flipped_decision_gradient_matches_finite_differences("qe")),
    ("flip_forward_exponential_drops_log", "const double vn = log((1.0 - pp) / (1.0 - u_v)) * mean / (1.0 - pp);",
     "const double vn = 0.0;", lambda: pins.test_flipped_decision_gradient_matches_finite_differences("qe")),
    # QE-M reverse mode: ln M's adjoint in the quadratic branch (b^2 term), in the
    # exponential branch (its A term's sign), and K3's share of the corrected K0*
    ("qem_adjoint_quadratic_b2", "const double db2 = A * a / D;", "const double db2 = A / D;",
     lambda: qem_pins.test_qem_reverse_mode_matches_forward_mode_duals(qem_pins.BASE)),
    ("qem_adjoint_exponential_A_sign", "*bar_A += bM * beta * q / ((beta - A) * (beta - A));",
     "*bar_A -= bM * beta * q / ((beta - A) * (beta - A));",
     lambda: qem_pins.test_qem_reverse_mode_matches_forward_mode_duals(qem_pins.HARD_Q)),
    ("qem_adjoint_drops_K3_share", "bar_K3 -= 0.5 * vc;", "",
     lambda: qem_pins.test_qem_reverse_mode_matches_forward_mode_duals(qem_pins.BASE)),
    # QE-M: the flipped step's reverse mode takes ln M's adjoint in the natural branch
    ("flip_qem_reverse_natural_log_m_branch", "qem_log_m_adjoint(mm, s2, K2 + 0.5 * K4, quad_forced,",
     "qem_log_m_adjoint(mm, s2, K2 + 0.5 * K4, -1,",
     lambda: pins.test_flipped_decision_gradient_matches_finite_differences("qem")),
    ("adjoint_drops_rate_discount", "grad[j * 7 + 6] -= m->T * price[j];", "",
     pins.test_adjoint_matches_fd_and_closed_form_delta),
    # QE-M at a zero mean (v = theta = 0): M = 1 exists; taking the plain step instead
    ("qem_zero_mean_takes_plain_step", "  if (m <= 0.0) return 0.0;", "  if (m <= 0.0) { *ok = 0; return 0.0; }",
     lambda: pins.test_adjoint_at_zero_variance_in_closed_form("qem")),
    # QE-M martingale correction
    ("qem_quadratic_log_sign", "- 0.5 * log(1.0 - 2.0 * A * a);", "+ 0.5 * log(1.0 - 2.0 * A * a);",
     lambda: qem_pins.test_one_step_expectation_is_a_martingale(qem_pins.BASE)),
    ("qem_exponential_branch", "return log(p + beta * (1.0 - p) / (beta - A));",
     "return log(p + beta * (1.0 - p) / (beta + A));",  # psi > 1.5 occurs on the coarse model
     lambda: qem_pins.test_one_step_expectation_is_a_martingale(qem_pins.WILD)),
    ("qem_A_definition", "const double A = k[6] + 0.5 * k[8];", "const double A = k[6] + k[8];",
     lambda: qem_pins.test_one_step_expectation_is_a_martingale(qem_pins.BASE)),
    ("qem_drops_rate", "return m->r * k[0] - lnM", "return -lnM",
     qem_pins.test_multi_step_martingale_within_monte_carlo_error),
    # correlated baskets
    ("basket_qem_plain_constant", "x[a] += step_k0(&models[a], ka, v[a], -1)", "x[a] += ka[4]",
     basket_pins.test_one_asset_is_the_single_asset_scheme_under_qem),
    ("basket_cholesky_transposed", "z += Lc[a * A + j] * eps[j];", "z += Lc[j * A + a] * eps[j];",
     lambda: basket_pins.test_exchange_option_in_the_black_scholes_limit_is_margrabe(0.6)),
    ("basket_shared_draws", "oracle_step_uniforms(seed, (uint32_t)a, path, n, &uv[a], &u_x);",
     "oracle_step_uniforms(seed, 0u, path, n, &uv[a], &u_x);",
     basket_pins.test_identity_correlation_gives_each_asset_its_own_paths),
    ("basket_first_asset_constants", "const double* ka = &k[10 * a];", "const double* ka = &k[0];",
     lambda: basket_pins.test_exchange_option_in_the_black_scholes_limit_is_margrabe(0.6)),
    # exercise-date states for Longstaff-Schwartz
    ("states_without_spot", "xs[j] = m->S0 * exp(xs[j]);", "xs[j] = exp(xs[j]);",
     lsm_pins.test_single_exercise_date_is_the_european_price),
]

# (name, module, site, planted, pin that must fail, [(holder, attribute) to swap])
PY_MISTAKES = [
    ("lsm_exercise_inverted", lsm, "ex = hj > C", "ex = hj < C",
     lsm_pins.test_bermudan_put_black_scholes_limit_matches_lattice),
    ("lsm_discount_from_maturity", lsm, "cash * np.exp(-r * t[np.maximum(stop, 0)]), 0.0)",
     "cash * np.exp(-r * t[-1]), 0.0)", lsm_pins.test_deterministic_paths_deep_put_exercises_at_the_first_date),
    ("lsm_undiscounted_targets", lsm, "Y = np.where(st >= 0, cash[itm] * np.exp(-r * (t[np.maximum(st, 0)] - t[j])), 0.0)",
     "Y = np.where(st >= 0, cash[itm], 0.0)", lsm_pins.test_regression_on_simulated_paths_matches_lstsq),
    ("lsm_regression_on_every_path", lsm, "itm = np.nonzero(h[:, j] > 0.0)[0]", "itm = np.arange(paths)",
     lsm_pins.test_regression_on_simulated_paths_matches_lstsq),
    ("lsm_back_substitution_uses_L", lsm, "sum(L[i][k] * beta[i] for i in range(k + 1, n) if keep[i])",
     "sum(L[k][i] * beta[i] for i in range(k + 1, n) if keep[i])", lsm_pins.test_normal_equation_solve_matches_lstsq),
    ("lsm_pivot_without_earlier_columns", lsm, "d = G[k][k] - sum(L[k][i] ** 2 for i in range(k) if keep[i])",
     "d = G[k][k]", lsm_pins.test_normal_equation_solve_matches_lstsq),
    ("lsm_reported_cross_term", lsm, "b1 * kx - 2.0 * b2 * kx * kx * cx - b4 * kx * ky * cy,",
     "b1 * kx - 2.0 * b2 * kx * kx * cx + b4 * kx * ky * cy,",
     lambda: lsm_pins.test_standardised_and_reported_coefficients_are_the_same_quadratic(0.09)),
    ("cf_rho_sign", analytic, "b = kappa - rho * sigma * iu", "b = kappa + rho * sigma * iu", _price_pin(False)),
    ("lewis_undiscounted", analytic, "return math.exp(-r * T) * (F - math.sqrt(F * K) * val / math.pi)",
     "return (F - math.sqrt(F * K) * val / math.pi)", pins.test_semi_analytic_forms_agree_and_bs_limit),
    ("put_parity_undiscounted_strike", analytic, "return call - S0 + K * math.exp(-r * T)", "return call - S0 + K",
     _price_pin(True)),
    ("cir_mean_sign", analytic, "return theta + (v0 - theta) * math.exp(-kappa * t)",
     "return theta - (v0 - theta) * math.exp(-kappa * t)",
     lambda: pins.test_closed_form_moments_solve_their_moment_equations(pins.HARD)),
    ("cir_var_drops_half", analytic, "theta * sigma ** 2 * (1.0 - e) ** 2 / (2.0 * kappa)",
     "theta * sigma ** 2 * (1.0 - e) ** 2 / kappa",
     lambda: pins.test_closed_form_moments_solve_their_moment_equations(CFG)),
    ("log_mean_sign", analytic, "return r * T - 0.5 * (theta * T", "return r * T + 0.5 * (theta * T",
     lambda: pins.test_closed_form_moments_solve_their_moment_equations(CFG)),
    ("bs_d1_sign", analytic, "d1 = (math.log(S0 / K) + (r + 0.5 * vol * vol) * T) / sd",
     "d1 = (math.log(S0 / K) + (r - 0.5 * vol * vol) * T) / sd",
     pins.test_black_scholes_closed_form_is_the_lognormal_expectation),
]


def _plant_c(monkeypatch, tmp_path, site, planted):
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(site) == 1, f"site not found exactly once: {site!r}"
    mutant = tmp_path / "simr_oracle.c"
    mutant.write_text(src.replace(site, planted))
    out = tmp_path / "_build"
    monkeypatch.setattr(oracle, "_SRC", str(mutant))
    monkeypatch.setattr(oracle, "_OUT_DIR", str(out))
    monkeypatch.setattr(oracle, "_LIB_PATH", str(out / "liboracle.so"))
    monkeypatch.setattr(oracle, "_lib", None)


def _plant_py(monkeypatch, module, site, planted):
    with open(module.__file__) as f:
        src = f.read()
    assert src.count(site) == 1, f"site not found exactly once: {site!r}"
    mod = types.ModuleType(module.__name__)
    mod.__file__ = module.__file__
    mod.__package__ = module.__package__
    exec(compile(src.replace(site, planted), module.__file__, "exec"), mod.__dict__)
    for holder in (pins, lsm_pins, qem_pins, basket_pins):
        for attr, value in list(vars(holder).items()):
            if value is module:
                monkeypatch.setattr(holder, attr, mod)


def test_the_unplanted_copy_passes(monkeypatch, tmp_path):
    # the mechanism itself: a copy with nothing planted builds, loads and passes a pin
    _plant_c(monkeypatch, tmp_path, "k1 += weyl1;", "k1 += weyl1;")
    assert os.path.dirname(oracle.lib()._name) == str(tmp_path / "_build")
    pins.test_step_uniform_mapping()
    pins.test_put_call_parity_on_common_paths()


@pytest.mark.parametrize("name,site,planted,pin", C_MISTAKES, ids=[m[0] for m in C_MISTAKES])
def test_c_oracle_mistake_is_caught(monkeypatch, tmp_path, name, site, planted, pin):
    _plant_c(monkeypatch, tmp_path, site, planted)
    with pytest.raises(AssertionError):
        with np.errstate(all="ignore"):
            pin()


@pytest.mark.parametrize("name,module,site,planted,pin", PY_MISTAKES, ids=[m[0] for m in PY_MISTAKES])
def test_python_oracle_mistake_is_caught(monkeypatch, name, module, site, planted, pin):
    _plant_py(monkeypatch, module, site, planted)
    with pytest.raises(AssertionError):
        with np.errstate(all="ignore"):
            pin()
