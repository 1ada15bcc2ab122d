"""Plant plausible mistakes in a copy of the oracle's walker and check that a
pin catches every one of them (the pins must not be satisfiable by a wrong
oracle).  The planted copies are compiled into a temporary directory; the real
oracle is untouched."""

import numpy as np
import pytest

import oracle
from pw_inputs import barabasi_albert, er_cycle

from . import test_oracle_exact as exact_pins
from . import test_oracle_probe as probe_pins
from . import test_oracle_walker as walker_pins

MUTANTS = {
    # four Feistel rounds (too few for a uniform matching, Lemma 3.2)
    "four_feistel_rounds": ("P->rounds = (b <= 4) ? 12u : 8u;", "P->rounds = 4u;"),
    # X_0 term dropped from a (Algorithm 1 initialises a with z_{X_0}/d_{X_0})
    "drop_x0_term": ("float a = (float)probe_entry(P, (uint64_t)x) / dx;", "float a = 0.0f;"),
    # wrong sign of the t-walk (Eq. hatphi-def subtracts)
    "plus_instead_of_minus": ("return a - b;", "return a + b;"),
    # U-statistic normalised by R^2 instead of R(R-1) (Eq. Q-Ustat)
    "biased_denominator": ("return (S1 * S1 - S2) / (Rd * (Rd - 1.0));", "return (S1 * S1 - S2) / (Rd * Rd);"),
    # both members of a pair get the same sign (Definition 3.1 gives opposite signs)
    "same_sign_pairs": ("return ((hv + pi) % 2 == 0) ? 1 : -1;", "return (hv % 2 == 0) ? 1 : -1;"),
    # always the first neighbour instead of a uniform one (Algorithm 1 samples uniformly)
    "first_neighbour": ("return col_idx[row_ptr[v] + (int64_t)j];", "(void)j; return col_idx[row_ptr[v]];"),
    # smallest block mean instead of the median (Eq. final-estimator)
    "min_not_median": ("double med = (G % 2 == 1) ? means[G / 2]", "double med = (G % 2 == 1) ? means[0]"),
    # even G: the upper middle block mean alone instead of the mean of the two middle ones
    "even_G_upper_middle": ("(means[G / 2 - 1] + means[G / 2]) / 2.0", "means[G / 2]"),
    # pilot variance normalised by R0 instead of R0 - 1 (biased sample variance)
    "pilot_variance_biased": ("sum_var = sum_var + (S2 - S1 * S1 / R0) / (R0 - 1.0);",
                              "sum_var = sum_var + (S2 - S1 * S1 / R0) / R0;"),
    # exact sums: halfway cases rounded up instead of to even
    "sum_ties_up": ("(rem == half && (sticky || (mant & 1)))", "(rem == half)"),
    # exact sums: bits below the kept window ignored when breaking a tie
    "sum_no_sticky": ("(rem == half && (sticky || (mant & 1)))", "(rem == half && (mant & 1))"),
    # S2 accumulated from |U_p| instead of U_p^2
    "s2_not_squared": ("exact_add(&A2, u * u);", "exact_add(&A2, fabs(u));"),
    # ADAPTIVE stopping rule without the pi/2 variance factor of the median
    "adaptive_no_median_factor": ("double x = 1.5707963267948966 * z * z * s2;", "double x = z * z * s2;"),
    # ADAPTIVE stopping rule with the biased (divide by K1) variance
    "adaptive_biased_variance": ("double s2 = K1 > 1 ? ss / (double)(K1 - 1) : 0.0;", "double s2 = ss / (double)K1;"),
    # theta not floored by theta_0 (the floor from the proof of Theorem 3.8)
    "theta_unfloored": ("double theta = q_bar > theta0 ? q_bar : theta0;", "double theta = q_bar;"),
    # zero set one element short (Definition 3.1: |U| = r)
    "zero_set_off_by_one": ("if (pi >= P->n - P->r) return 0; /* i in U */",
                            "if (pi > P->n - P->r) return 0; /* i in U */"),
    # sign hash of the element instead of its pair (pairs must get opposite signs)
    "hash_per_element": ("uint64_t pair = pi / 2;", "uint64_t pair = pi;"),
    # walks one transition short (L transitions, L + 1 terms per side)
    "one_step_short": ("  for (int32_t i = 1; i <= L; ++i) {\n    x = next_node(",
                       "  for (int32_t i = 1; i < L; ++i) {\n    x = next_node("),
    # the t-walk drawing the s-walk's random words (walks must be independent)
    "t_walk_shares_stream": ("uint64_t wid_s = 2 * pair_index, wid_t = 2 * pair_index + 1;",
                             "uint64_t wid_s = 2 * pair_index, wid_t = 2 * pair_index;"),
    # pilot R from 2 sigma^2 / theta instead of Lemma 3.7's 4 sigma^2 / theta
    "pilot_R_factor": ("double R = ceil_tol(c.c_R * 4.0 * sigma2 / theta);",
                       "double R = ceil_tol(c.c_R * 2.0 * sigma2 / theta);"),
    # G with log base 2 instead of the natural log (the proof needs exp(-G/8) <= delta)
    "G_log2": ("uint64_t G = (uint64_t)ceil_tol(8.0 * log(1.0 / c.delta));",
               "uint64_t G = (uint64_t)ceil_tol(8.0 * log2(1.0 / c.delta));"),
    # plain ceiling: exact integers that evaluate a last place high round up
    "ceil_no_tolerance": ("static double ceil_tol(double x) { return ceil(x * (1.0 - 1e-12)); }",
                          "static double ceil_tol(double x) { return ceil(x); }"),
    # strided blocks instead of contiguous ones (block g = probes [gB, (g+1)B))
    "strided_blocks": ("for (uint64_t k = g * B; k < (g + 1) * B; ++k) sum = sum + q[k];",
                       "for (uint64_t k = g; k < G * B; k += G) sum = sum + q[k];"),
    # U-statistic without the square of S1 (Eq. Q-Ustat)
    "s1_not_squared": ("return (S1 * S1 - S2) / (Rd * (Rd - 1.0));", "return (S1 - S2) / (Rd * (Rd - 1.0));"),
    # parity coin stuck at r = 2 for even n (Definition 3.1 draws r in {0, 2})
    "coin_always_two": ("P->r = 2u * (w[0] & 1u);", "P->r = 2u;"),
    # a single Feistel pass, no cycle-walk back into [n]
    "no_cycle_walk": ("  } while (x >= P->n);", "  } while (0);"),
}

# Planted mistakes in a copy of oracle/exact.py, each caught by the closed forms
# of test_oracle_exact.py.
EXACT_MUTANTS = {
    # lambda from the second eigenvalue only (odd cycles have |lambda_n| > lambda_2)
    "lambda_second_only": ("return float(max(abs(ev[1]), abs(ev[-1])))", "return float(abs(ev[1]))"),
    # lambda from the smallest eigenvalue only (circulant C_n(1,2) has lambda_2 > |lambda_n|)
    "lambda_last_only": ("return float(max(abs(ev[1]), abs(ev[-1])))", "return float(abs(ev[-1]))"),
    # R_eff with + instead of - on the cross term
    "reff_cross_sign": ("return float(lp[s, s] + lp[t, t] - 2.0 * lp[s, t])",
                        "return float(lp[s, s] + lp[t, t] + 2.0 * lp[s, t])"),
    # R_eff without the factor 2 on the cross term
    "reff_cross_factor": ("return float(lp[s, s] + lp[t, t] - 2.0 * lp[s, t])",
                          "return float(lp[s, s] + lp[t, t] - lp[s, t])"),
    # (L + J/n)^-1 without subtracting J/n: not the pseudoinverse (beta alone would not notice)
    "pinv_without_j": ("return np.linalg.inv(lap + j) - j", "return np.linalg.inv(lap + j)"),
    # all-pairs beta with + on the cross term
    "beta_matrix_cross_sign": ("return dg[:, None] + dg[None, :] - 2.0 * l2",
                               "return dg[:, None] + dg[None, :] + 2.0 * l2"),
    # beta from L^+ (e_s + e_t)
    "beta_plus": ("x = lp[:, s] - lp[:, t]", "x = lp[:, s] + lp[:, t]"),
    # series without its last term (L terms instead of L + 1)
    "series_last_term_dropped": ("        x = (a @ x) / deg  # (P x)_i = (1/d_i) sum_{j in N(i)} x_j\n    h += x\n",
                                 "        x = (a @ x) / deg  # (P x)_i = (1/d_i) sum_{j in N(i)} x_j\n"),
    # A D^-1 x instead of D^-1 A x (the same on regular graphs only)
    "series_transposed_step": ("x = (a @ x) / deg  # (P x)_i", "x = a @ (x / deg)  # (P x)_i"),
    # series start b_st instead of D^-1 b_st
    "series_start_without_degree": ("x[s] += 1.0 / deg[s]", "x[s] += 1.0"),
    # ||h||^2 without the (1^T h)^2 / n term of Eq. tr-beta-exp-Liu
    "series_no_mean_term": ("return sq - tot * tot / n", "return sq"),
    # the many-pair series without its last term
    "many_last_term_dropped": ("        x = (a @ x) / deg[:, None]\n    h += x\n", "        x = (a @ x) / deg[:, None]\n"),
}


def _pins_fail(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def _run_pins(g_tiny):
    """Fast pins; returns the names of those that fail."""
    failed = []
    checks = [
        ("pairing_uniform_n7", lambda: probe_pins.test_pairing_is_uniform(None, 7)),
        ("probe_structure", lambda: probe_pins.test_probe_structure(None, 10)),
        ("pi_permutation_odd_width", lambda: probe_pins.test_pi_is_permutation(None, 17)),
        ("neighbour_uniform", lambda: walker_pins.test_neighbour_sampling_uniform(None)),
        ("replicas_unbiased", lambda: walker_pins.test_replicas_unbiased_for_phi(None)),
        ("L0_deterministic", lambda: walker_pins.test_L0_replicas_are_deterministic(None, g_tiny)),
        ("pilot_accuracy", lambda: walker_pins.test_pilot_accuracy_problem_1(None, g_tiny)),
        ("median_golden", lambda: walker_pins.test_median_of_means_golden(None)),
        ("theory_budget_golden", lambda: walker_pins.test_theory_budget_golden(None)),
        ("G_for_even_deltas", lambda: walker_pins.test_G_for_even_deltas(None, g_tiny)),
        ("visits_are_walks", lambda: walker_pins.test_visits_are_the_walks_of_every_replica(None, g_tiny)),
        ("exact_sum_ties", lambda: walker_pins.test_exact_sum_ties_and_edges(None)),
        ("adaptive_golden", lambda: walker_pins.test_adaptive_rule_golden(None)),
        ("adaptive_rule", lambda: walker_pins.test_adaptive_budget_stopping_rule(None, g_tiny, 3, 77, 0.2, 32, 12345,
                                                                                 2.0)),
        ("adaptive_rule_2", lambda: walker_pins.test_adaptive_budget_stopping_rule(None, g_tiny, 10, 190, 0.1, 8,
                                                                                   99, 1.0)),
        ("even_G_query", lambda: walker_pins.test_even_G_query_takes_middle_pair(None, g_tiny)),
        ("pilot_statistics", lambda: walker_pins.test_pilot_statistics_from_replicas(None, g_tiny, 3, 77, 32, 12345,
                                                                                     0.2)),
        ("pilot_statistics_far", lambda: walker_pins.test_pilot_statistics_from_replicas(None, g_tiny, 42, 43, 20,
                                                                                         2**63 + 9, 0.05)),
        ("pilot_statistics_hub", lambda: walker_pins.test_pilot_statistics_from_replicas(None, g_tiny, "hub", 0, 32,
                                                                                         2, 0.2)),
    ]
    for name, fn in checks:
        if _pins_fail(fn):
            failed.append(name)
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(oracle_lib, tmp_path, name, tiny_graph):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor not found in walker.c"
    so = oracle.build_variant(src.replace(old, new), str(tmp_path))
    with oracle.use_variant(so):
        failed = _run_pins(tiny_graph)
    assert failed, f"no pin caught the planted mistake {name}"


def test_unmutated_copy_passes_fast_pins(oracle_lib, tmp_path, tiny_graph):
    so = oracle.build_variant(oracle.source_text(), str(tmp_path))
    with oracle.use_variant(so):
        assert _run_pins(tiny_graph) == []


def _load_exact_variant(text, tmp_path, name):
    import importlib.util

    path = tmp_path / f"exact_{name}.py"
    path.write_text(text)
    spec = importlib.util.spec_from_file_location(f"exact_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", sorted(EXACT_MUTANTS))
def test_planted_mistake_in_exact_is_caught(tmp_path, name):
    from oracle import exact

    old, new = EXACT_MUTANTS[name]
    with open(exact.__file__) as f:
        src = f.read()
    assert src.count(old) == 1, "mutation anchor not found in exact.py"
    mod = _load_exact_variant(src.replace(old, new), tmp_path, name)
    failed = [fn.__name__ for fn in (exact_pins.check_effective_resistance, exact_pins.check_mixing_lambda,
                                     exact_pins.check_exact_beta, exact_pins.check_series)
              if _pins_fail(fn, mod)]
    assert failed, f"no pin caught the planted mistake {name}"


def test_unmutated_exact_copy_passes(tmp_path):
    from oracle import exact

    with open(exact.__file__) as f:
        mod = _load_exact_variant(f.read(), tmp_path, "copy")
    exact_pins.check_effective_resistance(mod)
    exact_pins.check_mixing_lambda(mod)
    exact_pins.check_exact_beta(mod)
    exact_pins.check_series(mod)
