"""Planted mistakes in a copy of the oracle must fail its pins (CPU only).

Each case copies ``oracle/vamp_oracle.c``, changes one expression the way a
plausible slip would (a dropped term, a wrong sign, index or exponent, a
transposed operand), builds the copy in a temporary directory and runs the
pin that should catch it against the copy.  The committed oracle is never
touched.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vamp_oracle.c")

MUTATIONS = [
    ("bw_jacobian_sign",
     "J *= G / (A * (dp * dp + G * G));\n        } else if (m->kind[s] == OR_MAP_POW) {\n            double x2 = x[k] * x[k], x4",
     "J *= G / (A * (dp * dp - G * G));\n        } else if (m->kind[s] == OR_MAP_POW) {\n            double x2 = x[k] * x[k], x4",
     "round_trip_and_jacobian"),
    ("forward_transposed", "x[k] = e[j] + fr * w;", "x[k] = e[j + 1] - fr * w;",
     "forward_map_uniform_grid"),
    ("density_drops_n", "return 1.0 / ((double)o->n * (e[j + 1] - e[j]));",
     "return 1.0 / ((e[j + 1] - e[j]));", "grid_densities_normalised"),
    ("g_drops_alpha_own", "term = o->alpha[c] * g_own * jac_own;", "term = g_own * jac_own;",
     "identical_channels"),
    ("g_drops_alpha_other", "term = o->alpha[c] * gc * J;", "term = gc * J;",
     "multichannel_density_normalised and False"),
    ("dvalue_uses_w", "ks_add(&pp->D[((size_t)c * d + k) * n + jf[k]], w2);",
     "ks_add(&pp->D[((size_t)c * d + k) * n + jf[k]], w);", "pass_sums_brute_force"),
    ("rebin_power_dropped", "else mj = pow((r - 1.0) / log(r), alpha_grid);",
     "else mj = pow((r - 1.0) / log(r), 1.0);", "refine_worked_examples"),
    ("rebin_measure_sign", "else mj = pow((r - 1.0) / log(r), alpha_grid);",
     "else mj = pow((1.0 - r) / log(r), alpha_grid);", "refine_worked_examples"),
    ("omega_not_sqrt", "Dj[j] = sqrt(Dj[j]); S += Dj[j];", "S += Dj[j];", "refine_worked_examples"),
    ("rebin_wrong_edge", "ne[i] = e[j - 1] + fr * (e[j] - e[j - 1]);",
     "ne[i] = e[j - 1] + fr * (e[j + 1] - e[j - 1]);", "refine_worked_examples"),
    ("variance_no_bessel", "V = (m2 - m1 * m1) * Nc / (Nc - 1.0);", "V = (m2 - m1 * m1);",
     "pass_sums_brute_force"),
    ("sum_shift_wrong", "double dv = w - o->shift[c];", "double dv = w - 0.5 * o->shift[c];",
     "pass_sums_brute_force"),
    ("sigma_alpha_once", "ks_add(&V, o->alpha[c] * o->alpha[c] * o->Vc[c] / (double)o->Nc[c]);",
     "ks_add(&V, o->alpha[c] * o->Vc[c] / (double)o->Nc[c]);", "pass_sums_brute_force"),
    ("alpha_beta_dropped", "a = alpha[c] * pow(omega[c], beta) / SU * MU;",
     "a = alpha[c] * omega[c] / SU * MU;", "alpha_update_properties"),
    ("bw_inverse_sign", "x[k] = (atan(dp / G) + m->bwT0[s]) / A;",
     "x[k] = (atan(dp / G) - m->bwT0[s]) / A;", "round_trip_and_jacobian"),
    ("pow_inverse_exponent", "double xx = pow(p[k], 0.2);", "double xx = pow(p[k], 0.25);",
     "round_trip_and_jacobian"),
    ("pow_factor_exponent", "return pow(p + m->b[s], -0.8) / m->powN[s];",
     "return pow(p + m->b[s], -0.75) / m->powN[s];", "integrand_normalised and True"),
    ("gauss_norm_term", "(erf((1.0 - o->gcen) / (o->gsig * M_SQRT2)) + erf(o->gcen / (o->gsig * M_SQRT2)));",
     "(erf((1.0 - o->gcen) / (o->gsig * M_SQRT2)));", "integrand_normalised and False"),
    ("philox_operand", "uint32_t n2 = hi0 ^ c3 ^ k1;", "uint32_t n2 = hi0 ^ c1 ^ k1;",
     "philox_known_answers"),
    ("counter_fields_swapped", "uint32_t ctr[4] = { call, (uint32_t)b, field, o->request }, out[4];",
     "uint32_t ctr[4] = { call, field, (uint32_t)b, o->request }, out[4];", "call_words_layout"),
    ("forward_bin_shift", "j = (int)(t >> 33);", "j = (int)(t >> 34);",
     "forward_map_uniform_grid"),
    ("channel_choice_reflected", "double tgt = u * A[o->K - 1];",
     "double tgt = (1.0 - u) * A[o->K - 1];", "channel_choice_is_inverse_cdf"),
    ("accept_inverted", "if (unif(X[d + 1]) * wm < fabs(w)) {", "if (unif(X[d + 1]) * wm > fabs(w)) {",
     "generation_brute_force"),
    ("alloc_threshold_dropped", "if (nc < n_min) nc = n_min;", "if (nc < 0) nc = n_min;", "test_allocation"),
    ("alloc_rounded", "nc = (int64_t)floor(alpha[c] * (double)N);", "nc = (int64_t)llround(alpha[c] * (double)N);",
     "test_allocation"),
    ("combination_unweighted", "ks_add(&swi, o->hist_I[h] / o->hist_V[h]);", "ks_add(&swi, o->hist_I[h] / o->hist_V[h] * o->hist_V[h]);",
     "combination_inverse_variance"),
    ("chi2_dof_off_by_one", "o->comb_chi2 = ks_val(&chi) / (double)(cnt - 1);", "o->comb_chi2 = ks_val(&chi) / (double)cnt;",
     "combination_inverse_variance"),
    ("power_clamp_dropped", "            if (pk < DBL_MIN) pk = DBL_MIN; /* R15 */", "", "clamp_at_zero"),
    ("smoothing_end_weight", "        t[0] = (Din[0] + Din[1]) / 2.0;", "        t[0] = (Din[0] + Din[1]) / 3.0;",
     "three_point"),
    ("bin_rule_strict", "        if (e[mid] <= x) lo = mid; else hi = mid - 1;", "        if (e[mid] < x) lo = mid; else hi = mid - 1;",
     "bin_rule_at_edges"),
    ("rebin_zero_weight_limit", "if (r == 0.0) mj = 0.0;                    /* R2 */",
     "if (r == 0.0) mj = 1.0;                    /* R2 */", "refine"),
    ("alpha_zero_channel_kept", "else if (Ic[c] == 0.0) a = 0.0; /* all calls gave w = 0: switch off */",
     "else if (Ic[c] == 0.0) a = alpha[c];", "alpha_update_properties"),
    ("wmax_not_raised_between_batches", "        if (bmax > o->wmax) o->wmax = bmax;\n        ++b;",
     "        ++b;", "generation_brute_force"),
    # pseudo-stratified mode (R16, R17): pins in test_oracle_stratified.py
    ("strat_variance_no_bessel", "V = (ks_val(&s2) - ks_val(&qq) / s) / ((double)o->Cc[c] * (s - 1.0));",
     "V = (ks_val(&s2) - ks_val(&qq) / s) / ((double)o->Cc[c] * s);",
     "error_estimate_consistent", "test_oracle_stratified.py"),
    ("strat_cell_sum_not_squared", "ks_add(&pp->Q[c], v * v);", "ks_add(&pp->Q[c], v);",
     "zero_variance", "test_oracle_stratified.py"),
    ("strat_digits_not_shifted",
     "for (int k = 0; k < o->d; ++k) { digit[k] = rest % o->nr[c]; rest /= o->nr[c]; }\n        ksum cs",
     "for (int k = 0; k < o->d; ++k) { digit[k] = rest % o->nr[c]; }\n        ksum cs",
     "unbiased_and_error", "test_oracle_stratified.py"),
    ("strat_fraction_denominator", "fr = (double)(t % den) / (double)den;", "fr = (double)(t % den) / 0x1p33;",
     "points_lie", "test_oracle_stratified.py"),
    # channel equivalences (R18): pins in test_oracle_equiv.py
    ("eq_invert_not_mirrored", "else if (mode == OR_EQ_INVERT) out[j] += src[n - 1 - j];",
     "else if (mode == OR_EQ_INVERT) out[j] += src[j];", "mirror_symmetric", "test_oracle_equiv.py"),
    ("eq_symmetric_half_dropped", "out[j] += 0.5 * (src[j] + src[n - 1 - j]);",
     "out[j] += (src[j] + src[n - 1 - j]);", "mean_of_identity", "test_oracle_equiv.py"),
    ("eq_sequential_in_place", "const double *src = o->D + ((size_t)r[1] * d + r[2 + k]) * n;",
     "const double *src = o->Dp + ((size_t)r[1] * d + r[2 + k]) * n;", "rotation_images",
     "test_oracle_equiv.py"),
    ("eq_permutation_reversed", "const double *src = o->D + ((size_t)r[1] * d + r[2 + k]) * n;",
     "int kq = 0; while (r[2 + kq] != k) ++kq;\n"
     "                const double *src = o->D + ((size_t)r[1] * d + kq) * n;", "rotation_images",
     "test_oracle_equiv.py"),
    ("eq_invariant_adds_one", "for (int j = 0; j < n; ++j) out[j] = 1.0;",
     "for (int j = 0; j < n; ++j) out[j] += 1.0;", "invariant_axis", "test_oracle_equiv.py"),
    # signed integrands (R19): pins in test_oracle_signed.py
    ("signed_wmax_not_abs", "if (fabs(w) > pp->wmax) pp->wmax = fabs(w); /* R19 */",
     "if (w > pp->wmax) pp->wmax = w;", "largest_abs_weight", "test_oracle_signed.py"),
    ("signed_accept_not_abs", "if (unif(X[d + 1]) * wm < fabs(w)) { /* R19: keep the sign */",
     "if (unif(X[d + 1]) * wm < w) {", "follow_abs_f", "test_oracle_signed.py"),
    ("signed_batch_max_not_abs", "if (fabs(w) > bmax) bmax = fabs(w);", "if (w > bmax) bmax = w;",
     "raises_w_max", "test_oracle_signed.py"),
    ("signed_event_loses_sign", "w_out[written] = w;", "w_out[written] = fabs(w);",
     "follow_abs_f", "test_oracle_signed.py"),
]


@pytest.mark.parametrize("name,old,new,selector,pins",
                         [m if len(m) == 5 else m + ("test_oracle_pins.py",) for m in MUTATIONS],
                         ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, selector, pins):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    msrc = tmp_path / "vamp_oracle_mut.c"
    msrc.write_text(src.replace(old, new, 1))
    env = dict(os.environ, VAMP_ORACLE_SRC=str(msrc), VAMP_ORACLE_LIB=str(tmp_path / "libmut.so"))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins),
                        "-x", "-q", "-p", "no:cacheprovider", "-k", selector],
                       env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert "passed" in r.stdout or "failed" in r.stdout, r.stdout + r.stderr
    assert r.returncode == 1, f"planted mistake {name} not caught:\n{r.stdout[-2000:]}"
