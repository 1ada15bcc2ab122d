"""Plant plausible mistakes in a copy of the oracle's walker and check that a
pin catches every one of them (the pins must not be satisfiable by a wrong
oracle).  The planted copies are compiled into a temporary directory; the real
oracle is untouched."""

import numpy as np
import pytest

import oracle
from pw_inputs import barabasi_albert, er_cycle

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
        ("neighbour_uniform", lambda: walker_pins.test_neighbour_sampling_uniform(None)),
        ("replicas_unbiased", lambda: walker_pins.test_replicas_unbiased_for_phi(None)),
        ("L0_deterministic", lambda: walker_pins.test_L0_replicas_are_deterministic(None, g_tiny)),
        ("pilot_accuracy", lambda: walker_pins.test_pilot_accuracy_problem_1(None, g_tiny)),
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
