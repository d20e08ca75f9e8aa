"""Plant a plausible mistake in a copy of the oracle's C source, build it,
and check that at least one pin fails.  The mistakes are planted in the
oracle on the CPU only; the shipped oracle is never modified."""
import os
import subprocess
import sys

import pytest

import oracle
import test_oracle_omp as omp_pins
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "aqmp_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("unravel_rows", "y[m * b + i] = (double)c->pix", "y[i * b + m] = (double)c->pix"),
    ("atom_transposed", "col[m * b + i] = B[p * b + i] * B[q * b + m]",
     "col[i * b + m] = B[p * b + i] * B[q * b + m]"),
    ("dct_alpha0", "(k == 0) ? sqrt(1.0 / b) : sqrt(2.0 / b)", "sqrt(2.0 / b)"),
    ("dct_half_sample", "(m + 0.5) * k", "(m + 1.0) * k"),
    ("haar_sign", "+ len / 2; ++m) H[row * b + m] = v;", "+ len / 2; ++m) H[row * b + m] = -v;"),
    ("residual_sign", "r[v] -= alpha * pb[v];", "r[v] += alpha * pb[v];"),
    ("argmax_no_abs", "if (fabs(c[j]) > cmax) cmax = fabs(c[j]);", "if (c[j] > cmax) cmax = c[j];"),
    ("tie_highest", "int best = 0;\n        while (fabs(c[best]) < edge) ++best;",
     "int best = M - 1;\n        while (fabs(c[best]) < edge) --best;"),
    ("tie_band_dropped", "const double edge = cmax - tie_c;", "const double edge = cmax;"),
    ("stop_band_dropped", "if (E < eps2 - tie_e) { *converged = 1; break; }",
     "if (E < eps2) { *converged = 1; break; }"),
    ("stop_band_sign", "if (E < eps2 - tie_e) { *converged = 1; break; }",
     "if (E < eps2 + tie_e) { *converged = 1; break; }"),
    ("stop_after_budget_check", "if (E < eps2 - tie_e) { *converged = 1; break; }\n        if (t == k) break;",
     "if (t == k) break;\n        if (E < eps2 - tie_e) { *converged = 1; break; }"),
    ("budget_off_by_one", "if (t == k) break;", "if (t == k + 1) break;"),
    ("child_order", "rec(c, y0, x0 + h, h);\n        rec(c, y0 + h, x0, h);",
     "rec(c, y0 + h, x0, h);\n        rec(c, y0, x0 + h, h);"),
    ("split_no_min_check", "if (!conv && b > c->min_block)", "if (!conv && b >= c->min_block && b > 2)"),
    ("decode_transposed", "out[(long)(y0 + i) * pitch + x0 + m] = s;", "out[(long)(y0 + m) * pitch + x0 + i] = s;"),
    # Orthogonal Matching Pursuit
    ("omp_backsub_transposed", "for (int q = a + 1; q < m; ++q) s -= L[q * m + a] * x[q];",
     "for (int q = a + 1; q < m; ++q) s -= L[a * m + q] * x[q];"),
    ("omp_rhs_from_residual", "for (int v = 0; v < n; ++v) s += pa[v] * y[v];",
     "for (int v = 0; v < n; ++v) s += pa[v] * r[v];"),
    ("omp_residual_sign", "for (int a = 0; a < m; ++a) s -= x[a] * D[(size_t)S[a] * n + v];",
     "for (int a = 0; a < m; ++a) s += x[a] * D[(size_t)S[a] * n + v];"),
    ("omp_pivot_no_sqrt", "L[a * m + a] = sqrt(s);", "L[a * m + a] = s;"),
    ("omp_cholesky_sign", "for (int q = 0; q < b; ++q) s -= L[a * m + q] * L[b * m + q];",
     "for (int q = 0; q < b; ++q) s += L[a * m + q] * L[b * m + q];"),
]

PINS = [
    lambda: pins.test_dct_rows_match_scipy(8),
    lambda: pins.test_haar_rows_match_filter_bank(8),
    lambda: pins.test_dictionary_families_orthonormal(8),
    lambda: pins.test_dct_family_correlations_are_dctn(8),
    lambda: pins.test_haar_family_correlations_are_separable_fast_haar(8),
    lambda: pins.test_mp_on_dct_basis_is_sorted_dctn(4),
    lambda: pins.test_mp_on_haar_basis_is_sorted_fast_haar(4),
    lambda: pins.test_mp_energy_drops_by_alpha_squared(8, 1),
    lambda: [pins.test_mp_steps_are_brute_force_best_fits_4x4(s) for s in range(6)],
    pins.test_mp_stop_rule_is_strict_and_checked_before_each_step,
    lambda: [pins.test_exact_ties_go_to_the_lowest_index(b) for b in (4, 8)],
    pins.test_constant_image_gives_one_dc_atom_per_root,
    pins.test_zero_image_takes_no_step,
    pins.test_huge_tolerance_keeps_roots_without_atoms,
    pins.test_strong_noise_descends_to_min_blocks_with_full_budget,
    lambda: pins.test_quadtree_tiles_and_respects_tolerance(0, 1.0),
    pins.test_depth_first_leaf_order,
    pins.test_decoder_reconstructs_exactly_with_full_orthonormal_budget,
    pins.test_decoder_places_each_leaf_as_d_times_x,
    lambda: [omp_pins.test_matches_scikit_learn(t) for t in (4, 12)],
    omp_pins.test_reduces_to_mp_on_an_orthonormal_dictionary,
    omp_pins.test_each_refit_is_the_least_squares_solution,
]


def run_pins_against(so_path: str) -> int:
    """Run the pins against the build at `so_path`; return the index of the
    first pin that fails, or -1 if all pass."""
    with oracle.use_library(so_path):
        for i, pin in enumerate(PINS):
            try:
                pin()
            except (AssertionError, RuntimeError, ValueError, IndexError):
                return i
    return -1


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, orig, bad):
    src = open(SRC).read()
    assert orig in src, f"mutation site for {name} not found"
    mutant = tmp_path / f"{name}.c"
    mutant.write_text(src.replace(orig, bad, 1))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           str(mutant), "-o", str(so), "-lm"])
    # a child process, so that a mutant that crashes only ends the child
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_oracle_mutations as m; "
            "print('FIRST_FAILING_PIN', m.run_pins_against(%r))" % (here, os.path.dirname(here), str(so)))
    proc = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if proc.returncode == 0:
        line = [l for l in proc.stdout.splitlines() if l.startswith("FIRST_FAILING_PIN")][-1]
        assert int(line.split()[1]) >= 0, f"no pin caught the planted mistake {name}"
    # a non-zero exit (a crash inside the mutant) also means it was caught
