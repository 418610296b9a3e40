"""The oracle's pins catch plausible mistakes.  CPU only.

Each case plants one mistake in a copy of an oracle function (a swapped weight pair,
a dropped term, a wrong sign, a transposed operand, an index off by one), installs the
copy in place of the original for the duration of the case, and runs the pins named
beside it: at least one of them must fail.  The same pins are first run on the
unmodified oracle, where all of them must pass.  Mistakes that cannot change any result
(equivalent mutants) are not listed: for instance the finish's bracket (y_L, y_R]
against (y_L, y_R), since y_R always has #(x < y_R) >= k in the oracle's iteration, or
the rho form of LTS summing s <= q instead of s < q, where the tie weight h - #(s <= q)
absorbs the difference.
"""
import importlib.util
import inspect
import os
import textwrap

import pytest

from oracle import bracket as ob
from oracle import knn as oknn
from oracle import philox as oph
from oracle import regression as oreg
from oracle import select as osel

HERE = os.path.dirname(os.path.abspath(__file__))
_PINS = {}


def _pins(name):
    """The pin module tests/<name>.py, loaded once under a private name."""
    if name not in _PINS:
        spec = importlib.util.spec_from_file_location("_pins_" + name, os.path.join(HERE, name + ".py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        _PINS[name] = mod
    return _PINS[name]


def _mutant(module, fname, old, new, count=1):
    """A copy of module.fname with `old` replaced by `new` in its source (which must hold
    `old` exactly `count` times), defined in a copy of the module's namespace."""
    src = textwrap.dedent(inspect.getsource(getattr(module, fname)))
    assert src.count(old) == count, (fname, old, src.count(old))
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant of {module.__name__}.{fname}>", "exec"), ns)
    return ns[fname]


def _run(pin):
    mod, test, kwargs = pin
    getattr(_pins(mod), test)(**kwargs)


S, R, B, K = "test_oracle_select", "test_oracle_regression", "test_oracle_bracket", "test_oracle_knn"

# (id, module, function, old, new, occurrences, pins)
MUTANTS = [
    ("pinball_weights_swapped", osel, "pinball_cost",
     "(k - 0.5) * s, -(n - k + 0.5) * s", "(n - k + 0.5) * s, -(k - 0.5) * s", 1,
     [(S, "test_golden_order_statistics_and_costs", {}),
      (S, "test_pinball_minimiser_is_order_statistic", {"k_frac": 0.01})]),
    ("pinball_lower_branch_sign", osel, "pinball_cost",
     "-(n - k + 0.5) * s", "(n - k + 0.5) * s", 1,
     [(S, "test_golden_order_statistics_and_costs", {}),
      (S, "test_pinball_minimiser_is_order_statistic", {"k_frac": 0.5})]),
    ("median_cost_sign", osel, "median_cost",
     "np.abs(x - float(y))", "(x - float(y))", 1,
     [(S, "test_golden_order_statistics_and_costs", {})]),
    ("subdifferential_counts_transposed", osel, "pinball_subdifferential",
     "n * (c_lt - k + 0.5), n * (c_le - k + 0.5)", "n * (c_le - k + 0.5), n * (c_lt - k + 0.5)", 1,
     [(S, "test_subdifferential_and_minimiser_condition", {})]),
    ("subdifferential_half_dropped", osel, "pinball_subdifferential",
     "- k + 0.5)", "- k)", 2,
     [(S, "test_subdifferential_and_minimiser_condition", {})]),
    ("relative_cost_linear_term_dropped", osel, "relative_cost",
     "(c_le_a - k + 0.5) * (t64 - a64) + ", "", 1,
     [(S, "test_relative_cost_matches_cost_differences", {}),
      (S, "test_relative_cost_ignores_far_outliers", {})]),
    ("relative_cost_slope_from_strict_count", osel, "relative_cost",
     "_, c_le_a = counts(x, a)", "c_le_a, _ = counts(x, a)", 1,
     [(S, "test_relative_cost_at_tied_data_points", {})]),
    ("relative_cost_bracket_closed_at_a", osel, "relative_cost",
     "(x > x.dtype.type(a))", "(x >= x.dtype.type(a))", 1,
     [(S, "test_relative_cost_at_tied_data_points", {})]),
    ("order_key_negatives_not_flipped", osel, "total_order_key",
     "np.where((u & sign) != 0, ~u, u | sign)", "np.where((u & sign) != 0, u, u | sign)", 1,
     [(S, "test_key_roundtrip_and_order", {}), (S, "test_min_max_special_cases", {})]),
    ("select_rank_off_by_one", osel, "select_kth",
     "np.partition(keys, k - 1)[k - 1]", "np.partition(keys, min(k, keys.size - 1))[min(k, keys.size - 1)]", 1,
     [(S, "test_brute_force_all_small_arrays_exhaustive", {}), (S, "test_min_max_special_cases", {})]),
    ("select_rank_reversed", osel, "select_kth",
     "np.partition(keys, k - 1)[k - 1]", "np.partition(keys, keys.size - k)[keys.size - k]", 1,
     [(S, "test_order_statistics_commute_with_monotone_transforms", {})]),
    ("median_rank_rounded_up", osel, "median",
     "(x.size + 1) // 2", "(x.size + 2) // 2", 1,
     [(S, "test_golden_order_statistics_and_costs", {}), (R, "test_lms_brute_force_rank", {})]),
    ("kelley_tangent_slopes_transposed", osel, "kelley_select",
     "(gR * w - dF) / (gR - gL)", "(gL * w - dF) / (gR - gL)", 1,
     [(S, "test_kelley_model_first_step_is_tangent_intersection", {})]),
    ("kelley_cost_difference_sign", osel, "kelley_select",
     "(gR * w - dF)", "(gR * w + dF)", 1,
     [(S, "test_kelley_model_first_step_is_tangent_intersection", {})]),
    ("kelley_right_slope_half_dropped", osel, "kelley_select",
     "gL = cle_L - k + 0.5", "gL = cle_L - k", 1,
     [(S, "test_kelley_model_first_step_is_tangent_intersection", {})]),
    ("kelley_finish_rank_off_by_one", osel, "kelley_select",
     "select_kth(z, k - cle_L)", "select_kth(z, min(k - cle_L + 1, z.size))", 1,
     [(S, "test_kelley_model_matches_definition", {"dist": "normal"}),
      (S, "test_kelley_model_ties_infinities_zeros", {})]),
    ("kelley_lower_end_keeps_strict_count", osel, "kelley_select",
     "new = dict(yL=t, cle_L=c_le, dF=dF - dphi)", "new = dict(yL=t, cle_L=c_lt, dF=dF - dphi)", 1,
     [(S, "test_kelley_model_ties_infinities_zeros", {}),
      (S, "test_kelley_model_integer_ties_every_rank", {})]),
    ("kelley_zero_sign_boundary", osel, "_zero_sign",
     "(k - c_lt_v) <= n_negzero", "(k - c_lt_v) < n_negzero", 1,
     [(S, "test_kelley_model_ties_infinities_zeros", {}),
      (S, "test_kelley_model_exhaustive_small_alphabet", {})]),
    ("lms_rank_off_by_one", oreg, "lms",
     "select_kth(np.asarray(s, dtype=np.float64), k)",
     "select_kth(np.asarray(s, dtype=np.float64), min(k + 1, np.asarray(s).size))", 1,
     [(R, "test_lms_brute_force_rank", {})]),
    ("lts_one_term_short", oreg, "lts",
     "s[:h]", "s[:h - 1]", 1,
     [(R, "test_lts_is_min_over_h_subsets_brute_force", {})]),
    ("lts_rho_tie_weight_dropped", oreg, "lts_rho_form",
     "math.fsum(below.tolist()) + a * q", "math.fsum(below.tolist())", 1,
     [(R, "test_rho_form_with_ties", {}), (R, "test_lts_is_min_over_h_subsets_brute_force", {})]),
    ("residuals_operand_transposed", oreg, "residuals",
     "y[:, None] - X @ theta", "y[:, None] - X[:, ::-1] @ theta", 1,
     [(R, "test_residual_sign_and_shape", {}),
      (R, "test_exact_fit_candidate_has_zero_residuals_on_its_subset", {})]),
    ("rho_tie_share_inverted", oreg, "rho_weights",
     "rho[tie] = a / b", "rho[tie] = b / max(a, 1)", 1,
     [(R, "test_rho_weights_sum_to_h_and_give_the_lts_objective", {})]),
    ("c_step_unweighted_response", oreg, "c_step",
     "b = Xd.T @ (rho * yd)", "b = Xd.T @ yd", 1,
     [(R, "test_c_step_fixed_point_and_recovery_of_the_clean_model", {}),
      (R, "test_c_steps_never_increase_the_objective", {})]),
    ("c_step_gram_transposed_weights", oreg, "c_step",
     "A = Xd.T @ (rho[:, None] * Xd)", "A = Xd.T @ Xd", 1,
     [(R, "test_c_step_fixed_point_and_recovery_of_the_clean_model", {}),
      (R, "test_lts_brute_force_optimum_is_a_c_step_fixed_point", {})]),
    ("f32_residual_fused_in_float64", oreg, "squared_residuals_f32",
     "acc = acc + X[:, j] * theta[j]", "acc = (acc.astype(np.float64) + X[:, j].astype(np.float64) * theta[j]).astype(np.float32)", 1,
     [(R, "test_float32_residuals_follow_their_stated_order", {})]),
    ("c_steps_accepts_increase", oreg, "c_steps",
     "if not Fn < F:", "if False:", 1,
     [(R, "test_c_step_fixed_point_and_recovery_of_the_clean_model", {})]),
    ("knn_tie_weight_full", oknn, "indicator",
     "rho[tie] = a / b", "rho[tie] = 1.0", 1,
     [(K, "test_indicator_is_inclusion_frequency_over_tie_breaks", {})]),
    ("knn_indicator_closed_below", oknn, "indicator",
     "below = d2 < q", "below = d2 <= q", 1,
     [(K, "test_indicator_is_inclusion_frequency_over_tie_breaks", {})]),
    ("knn_weight_on_squared_distance", oknn, "regress_d2",
     "weight(np.sqrt(D2[j]), kind, eps)", "weight(D2[j], kind, eps)", 1,
     [(K, "test_regression_is_the_mean_over_tie_breaks", {"kind": "inverse"})]),
    ("knn_prediction_not_normalised", oknn, "regress_d2",
     "/ math.fsum(w.tolist())", "/ k", 1,
     [(K, "test_regression_is_the_mean_over_tie_breaks", {"kind": "inverse"})]),
    ("knn_distance_operand_dropped", oknn, "squared_distances",
     "diff = Q[:, None, :] - X[None, :, :]", "diff = Q[:, None, :] - 0 * X[None, :, :]", 1,
     [(K, "test_squared_distances_hand_worked", {})]),
    ("knn_f32_distance_accumulated_in_float64", oknn, "squared_distances_f32",
     "acc = acc + diff * diff\n", "acc = (acc.astype(np.float64) + diff.astype(np.float64) ** 2).astype(np.float32)\n", 1,
     [(K, "test_float32_distances_follow_their_stated_order", {})]),
    ("knn_vote_share_inverted", oknn, "exact_votes_d2",
     "share = Fraction(k - int(np.count_nonzero(below)), int(np.count_nonzero(tie)))",
     "share = Fraction(int(np.count_nonzero(tie)), max(1, k - int(np.count_nonzero(below))))", 1,
     [(K, "test_vote_totals_are_exact_fractions", {}), (K, "test_votes_are_the_mean_over_tie_breaks", {})]),
    ("gelu_grad_term_dropped", ob, "gelu_grad",
     "return Phi + u * phi", "return Phi", 1,
     [(B, "test_gelu_closed_forms", {}), (B, "test_backward_matches_central_differences", {})]),
    ("backward_first_layer_transposed", ob, "backward",
     "gW1 = g_u1.T @ F", "gW1 = F.T @ g_u1", 1,
     [(B, "test_backward_matches_central_differences", {})]),
    ("loss_grad_pinball_sign", ob, "loss_grad_o",
     "(-2.0 * d - drho * np.sign(d)) / B", "(-2.0 * d + drho * np.sign(d)) / B", 1,
     [(B, "test_backward_matches_central_differences", {})]),
    ("loss_pinball_tau_mirrored", ob, "loss",
     "rho = u * (tau - (u < 0))", "rho = u * ((1 - tau) - (u < 0))", 1,
     [(B, "test_loss_closed_form", {})]),
    ("adam_bias_correction_dropped", ob, "adam_step",
     "mhat = m / (1 - beta1 ** t)", "mhat = m", 1,
     [(B, "test_adam_first_step_is_lr_times_sign", {})]),
    ("sketch_quantile_offset_dropped", ob, "sketch_features",
     "q = s[16 + 32 * np.arange(N_QUANT)]", "q = s[32 * np.arange(N_QUANT)]", 1,
     [(B, "test_sketch_indexing_and_features", {})]),
    ("philox_multipliers_swapped", oph, "_round",
     "p0 = M0 * c[0]", "p0 = M1 * c[0]", 1,
     [(B, "test_philox_known_answer_vectors", {})]),
]


@pytest.mark.parametrize("case", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(case, monkeypatch):
    _, module, fname, old, new, count, pins = case
    for pin in pins:   # control: the pins hold on the unmodified oracle
        _run(pin)
    monkeypatch.setattr(module, fname, _mutant(module, fname, old, new, count))
    caught = []
    for pin in pins:
        try:
            _run(pin)
        except Exception as e:   # an assertion, or a rank the mistake pushed out of range
            caught.append((pin[1], type(e).__name__))
    assert caught, f"no pin among {[p[1] for p in pins]} caught the mistake {old!r} -> {new!r}"
