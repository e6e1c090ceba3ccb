"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a private copy of the oracle's C source
(a dropped term, a wrong sign, an off-by-one, a transposed operand ...),
compiles it on the CPU and checks that at least one pin of
``tests/test_oracle.py`` fails against that build.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "sptrsv_oracle.c")

# (name, original text, planted mistake, pins that must notice it)
MUTANTS = [
    ("pick_tie_largest_row", "if (best < 0 || deps < best_deps || (deps == best_deps && i < best)) {",
     "if (best < 0 || deps < best_deps || (deps == best_deps && i > best)) {",
     [lambda: P.test_level_summary_lap2d_closed_form(6)]),
    ("pick_most_deps", "if (best < 0 || deps < best_deps || (deps == best_deps && i < best)) {",
     "if (best < 0 || deps > best_deps || (deps == best_deps && i < best)) {",
     [lambda: P.test_level_summary_brute_force(0)]),
    ("thin_inclusive", "thin[l] = (double)cost[l] < threshold ? 1 : 0;",
     "thin[l] = (double)cost[l] <= threshold ? 1 : 0;",
     [P.test_level_summary_threshold_is_strict]),
    ("solve_sign", "s = s - v[p] * x[(int64_t)ci[p] * k + r];",
     "s = s + v[p] * x[(int64_t)ci[p] * k + r];",
     [lambda: P.test_solve_matches_dense_triangular(1, 1)]),
    ("solve_diag_mul", "x[(int64_t)i * k + r] = s / v[d];", "x[(int64_t)i * k + r] = s * v[d];",
     [lambda: P.test_solve_matches_dense_triangular(2, 3)]),
    ("transpose_sign", "r[(int64_t)ci[p] * k + q] - v[p] * g;", "r[(int64_t)ci[p] * k + q] + v[p] * g;",
     [P.test_solve_transpose_matches_dense]),
    ("grad_sign", "gv[p] = -s;", "gv[p] = s;", [P.test_grad_vals_dense_closed_form]),
    ("grad_transposed", "x[(int64_t)ci[p] * k + q];", "x[(int64_t)i * k + q];",
     [P.test_grad_vals_dense_closed_form]),
    ("levels_offbyone", "lev[front[f]] = round;", "lev[front[f]] = round + (round > 3);",
     [lambda: P.test_levels_brute_force_longest_path(3), P.test_levels_closed_forms]),
    ("cost_drop_one", "cost[lev[i]] += 2 * (int64_t)(rp[i + 1] - rp[i] - 1) + 1;",
     "cost[lev[i]] += 2 * (int64_t)(rp[i + 1] - rp[i] - 1);",
     [P.test_cost_laplacian_closed_form]),
    ("perm_unstable", "for (int32_t i = 0; i < n; ++i) perm[pos[lev[i]]++] = i;",
     "for (int32_t i = n - 1; i >= 0; --i) perm[pos[lev[i]]++] = i;",
     [P.test_partition_definition]),
    ("arl_denominator", "out[1] = (double)n / L;", "out[1] = (double)n / (L + 1.0);",
     [lambda: P.test_stats_reproduce_paper_tuples(P._paper_rows()[1])]),
    ("air_numerator", "out[2] = (double)(nnz - (int64_t)n) / (double)n;",
     "out[2] = (double)(nnz) / (double)n;",
     [lambda: P.test_stats_reproduce_paper_tuples(P._paper_rows()[0])]),
    ("cov_sample_variance", "unsigned __int128 a = (unsigned __int128)(uint64_t)m * S2;",
     "unsigned __int128 a = (unsigned __int128)(uint64_t)(m - 1) * S2;",
     [P.test_cov_population_definition_and_exactness]),
    ("cov_64bit_overflow", "unsigned __int128 d = (a > b) ? (a - b) : 0;",
     "unsigned __int128 d = (uint64_t)((a > b) ? (a - b) : 0);",
     [P.test_cov_population_definition_and_exactness]),
    ("threshold_no_relax", "return alc * (1.0 + alpha * relax);", "return alc * (1.0 + 0.5 * alpha * relax);",
     [lambda: P.test_stats_reproduce_paper_tuples(P._paper_rows()[3])]),
    ("rewrite_update_sign", "w->acc[k] = w->acc[k] - m * v[p];", "w->acc[k] = w->acc[k] + m * v[p];",
     [P.test_rewrite_worked_example, P.test_rewrite_lap2d_closed_form]),
    ("rewrite_wrong_pivot", "double m = w->acc[j] / v[dj];", "double m = w->acc[j] / v[rp[j]];",
     [P.test_rewrite_lap2d_closed_form, lambda: P.test_rewrite_invariants(0)]),
    ("rewrite_target_offbyone", "if (lev[j] >= t && heap_push(&w->h, j)) return ORC_ENOMEM;",
     "if (lev[j] > t && heap_push(&w->h, j)) return ORC_ENOMEM;",
     [P.test_rewrite_worked_example]),
    ("rewrite_T_sign", "w->elim_v[w->nelim] = 0.0 - m;", "w->elim_v[w->nelim] = m;",
     [P.test_rewrite_worked_example, lambda: P.test_rewrite_invariants(1)]),
    ("rewrite_uses_rewritten_rows", "if (tgt[i] < 0 || t < tgt[i]) tgt[i] = t;",
     "if (tgt[i] < 0 || t > tgt[i]) tgt[i] = t;",
     [P.test_rewrite_errors_and_duplicates]),
    ("solve_rewritten_T_sign", "s = s + tv[p] * b[(int64_t)tci[p] * k + r];",
     "s = s - tv[p] * b[(int64_t)tci[p] * k + r];",
     [P.test_rewrite_worked_example]),
    ("validate_allows_repeats", "if (p > a && ci[p] <= ci[p - 1])", "if (p > a && ci[p] < ci[p - 1])",
     [P.test_validate_codes]),
    ("validate_drops_zero_diag", "if (ci[e - 1] != i || v[e - 1] == 0.0)", "if (ci[e - 1] != i)",
     [P.test_validate_codes]),
    ("validate_empty_row_invalid", "return (e < a) ? ORC_EINVAL : ORC_EDIAG;", "return ORC_EINVAL;",
     [P.test_validate_codes]),
    ("validate_sorted_before_range", "if (ci[p] < 0 || ci[p] > i) { *bad_row = i; return ORC_ENOTLOWER; }\n"
     "            if (p > a && ci[p] <= ci[p - 1]) { *bad_row = i; return ORC_EUNSORTED; }",
     "if (p > a && ci[p] <= ci[p - 1]) { *bad_row = i; return ORC_EUNSORTED; }\n"
     "            if (ci[p] < 0 || ci[p] > i) { *bad_row = i; return ORC_ENOTLOWER; }",
     [P.test_validate_codes]),
    ("tt_transposed_operand", "tv[p] * gbp[(int64_t)i * k + r];", "tv[p] * gbp[(int64_t)tci[p] * k + r];",
     [P.test_rewritten_gradient_identity]),
]


@pytest.fixture(scope="module")
def src_text():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,orig,bad,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, src_text, name, orig, bad, pins):
    assert src_text.count(orig) == 1, f"mutation anchor not unique: {orig}"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src_text.replace(orig, bad))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                           "-o", str(lib), str(msrc), "-lm"])
    oracle.use_library(str(lib))
    try:
        caught = 0
        for pin in pins:
            try:
                pin()
            except (AssertionError, oracle.OracleError):
                caught += 1
        assert caught > 0, f"no pin noticed the planted mistake {name}"
    finally:
        oracle.use_library(None)
