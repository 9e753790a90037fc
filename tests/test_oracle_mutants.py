"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a copy of ``oracle/oracle.c``
(a dropped factor, a wrong sign or index, a missing penalty), builds it on the
CPU, points the oracle module at the mutant and runs the pins of
``test_oracle.py``: at least one pin must fail for every mutant.  The real
oracle is never modified.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle as O
from tests import test_oracle as T

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")

MUTANTS = {
    "gain_drops_half": ("-(g[i] * di + 0.5 * qii * di * di)", "-(g[i] * di + qii * di * di)"),
    "passive_set_drops_negative_grad": (
        "gb[i] = (!dead[i] && (y[i] > 0.0 || g[i] < 0.0)) ? g[i] : 0.0;",
        "gb[i] = (!dead[i] && (y[i] > 0.0)) ? g[i] : 0.0;"),
    "pg_gradient_update_sign": ("            g[i] += t;\n", "            g[i] -= t;\n"),
    "rescale_one_sided": ("H[i * r + j] / (d[i] * d[j])", "H[i * r + j] / d[i]"),
    "linear_term_times_d": ("q[i] = dead[i] ? 0.0 : h[i] / d[i];", "q[i] = dead[i] ? 0.0 : h[i] * d[i];"),
    "output_not_unscaled": ("x[i] = dead[i] ? 0.0 : y[i] / d[i];", "x[i] = dead[i] ? 0.0 : y[i];"),
    "gram_drops_l2": ("Q[i * r + j] = s + (i == j ? beta : 0.0);", "Q[i * r + j] = s;"),
    "row_drops_l1": ("h[j] = -C[i * r + j] + alpha;\n                double ms", "h[j] = -C[i * r + j];\n                double ms"),
    "stop_rule_absolute": ("if (sk <= o->eps * s0)", "if (sk <= o->eps)"),
    "cd_column_wrong": ("g[i] += Q[i * r + p] * dp;", "g[i] += Q[i * r + i] * dp;"),
    "cross_index_swapped": ("s += A[i * lda + t] * B[t * r + j];", "s += A[i * lda + t] * B[j * r + t % r];"),
    "tie_break_highest": ("if (gain > best) {", "if (gain >= best && gain > 0.0) {"),
    # the structure of Alg. 3's repeat loop
    "line_search_unmasked_gradient": (
        "gb[i] = (!dead[i] && (y[i] > 0.0 || g[i] < 0.0)) ? g[i] : 0.0;",
        "gb[i] = !dead[i] ? g[i] : 0.0;"),
    "line_search_half_step": ("double alpha = s / den;", "double alpha = 0.5 * s / den;"),
    "line_search_not_projected": ("yn[i] = v > 0.0 ? v : 0.0;", "yn[i] = v;"),
    "cd_step_not_projected": ("double di = (v > 0.0 ? v : 0.0) - y[i];", "double di = v - y[i];"),
    "cd_one_step_per_iteration": ("int T = o->cd_steps < 0 ? r : o->cd_steps;",
                                  "int T = o->cd_steps < 0 ? 1 : o->cd_steps;"),
    # the outer loop (Alg. 1/2): the H-update's Gram and cross term
    "m_step_keeps_e_step_gram": ("        oracle_gram(W, m, r, o->beta_h, Q);\n", "\n"),
    "m_step_cross_reads_v": ("oracle_cross_dense(VT, n, m, m, W, r, CH);",
                             "oracle_cross_dense(Vd, n, m, m, W, r, CH);"),
    # the objective (Def. 1, Table 4's 1/2) and the KKT residual (Eq. 2)
    "objective_drops_half": ("return 0.5 * fit + aw * l1w", "return fit + aw * l1w"),
    "objective_csr_cross_sign": ("0.5 * (vv - 2.0 * vwh + whwh)", "0.5 * (vv + 2.0 * vwh + whwh)"),
    "kkt_l1_sign": ("double gj = -C[i * r + j] + alpha;", "double gj = -C[i * r + j] - alpha;"),
    # the plain definitions: Gram X^T X and the CSR cross term
    "gram_outer_index": ("s += X[k * r + i] * X[k * r + j];", "s += X[k * r + i] * X[k * r + i];"),
    "csr_cross_row_end": ("for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)\n                s += vals[p] * B",
                          "for (int64_t p = rowptr[i]; p + 1 < rowptr[i + 1]; ++p)\n                s += vals[p] * B"),
    "csr_objective_drops_square": ("vv += vals[p] * vals[p];", "vv += vals[p];"),
    "rescale_diagonal_unscaled": ("Qt[i * r + j] = 1.0;   /* Q_ii", "Qt[i * r + j] = H[i * r + j];   /* Q_ii"),
    # the fast break (maxStop) of Alg. 2/3 in both readings
    "maxstop_threshold_strict": ("maxstop && sk <= *maxstop)", "maxstop && sk < *maxstop)"),
    "maxstop_same_half_step": ("double ms = maxstop_in, sf = 0.0;",
                               "double ms = sm > maxstop_in ? sm : maxstop_in, sf = 0.0;"),
    "maxstop_other_factor": ("o->nqp.maxstop_mode == 2 ? ms_seq : msw, &ms_next",
                             "o->nqp.maxstop_mode == 2 ? ms_seq : msh, &ms_next"),
    "maxstop_previous_update_dropped": ("        else\n            msw = ms_next;",
                                        "        else\n            msw = 0.0;"),
    "maxstop_sequential_last_not_max": ("if (o->maxstop_mode == 2 && maxstop && sk > *maxstop)",
                                        "if (o->maxstop_mode == 2 && maxstop)"),
    "maxstop_sequential_reset_before_m_step": ("o->nqp.maxstop_mode == 2 ? ms_seq : msh",
                                               "o->nqp.maxstop_mode == 2 ? 0.0 : msh"),
}

PINS = [
    T.test_worked_example_closed_form_and_59_steps,
    lambda: T.test_nqp_matches_brute_force(4, 0.1, 0.05),
    lambda: T.test_nqp_matches_brute_force(3, 0.3, 0.0),
    T.test_nqp_matches_lawson_hanson,
    T.test_rescale_invariants,
    T.test_gram_and_cross_match_numpy,
    T.test_penalties_enter_q_and_linear_term,
    T.test_one_projected_gradient_step_is_exact_line_search,
    T.test_one_coordinate_step_takes_largest_objective_decrease,
    T.test_stop_rule_stops_at_first_qualifying_iteration,
    T.test_diagonal_q_one_iteration_exact,
    T.test_nqp_kkt_at_convergence,
    T.test_outer_objective_monotone_tiny,
    T.test_exact_low_rank_recovery,
    T.test_objectives_agree_and_match_numpy,
    T.test_sparse_solve_equals_dense_solve,
    T.test_maxstop_mode1_fixed_threshold_rows,
    T.test_maxstop_mode1_threshold_of_previous_update_same_factor,
    T.test_maxstop_mode2_running_threshold_row_by_row,
    T.test_maxstop_mode2_reset_each_outer_iteration_carried_into_m_step,
]


def _tie_pin():
    # equal gains on two coordinates: the lower index must move
    import numpy as np
    H = np.eye(3)
    h = np.array([-1.0, -1.0, -0.5])
    x, k, s = O.nqp(H, h, np.zeros(3), O.nqp_opts(max_inner=1, eps=0.0, cd_steps=1, pg=0))
    assert x[0] == 1.0 and x[1] == 0.0


PINS.append(_tie_pin)


def test_tie_break_lowest_index():
    _tie_pin()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_some_pin_catches_mutant(name, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    tmp = tempfile.mkdtemp()
    try:
        path = os.path.join(tmp, "mut.c")
        open(path, "w").write(src.replace(old, new, 1))
        so = os.path.join(tmp, "libmut.so")
        subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", so, path, "-lm"],
                       check=True, capture_output=True)
        monkeypatch.setattr(O, "_lib", O.load(so))
        caught = 0
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                caught += 1
        assert caught >= 1, f"no pin caught mutant {name}"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
