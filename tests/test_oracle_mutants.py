"""Planted mistakes: each case compiles a copy of the CPU oracle with one
plausible error in it (a dropped term, a wrong sign or factor, a wrong index,
a strict comparison where the paper's is non-strict ...) and checks that at
least one of the oracle's pins rejects the copy.  The mistakes are planted in
the oracle only, on the CPU."""
import os

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

PIN_CALLS = [
    ("unique brute force", lambda: pins.test_unique_matches_brute_force((16, 16), 4, 3)),
    ("unique numpy", pins.test_unique_matches_numpy_on_plain_image),
    ("splitmix64 vector", pins.test_splitmix64_published_vector),
    ("init valid", pins.test_init_indices_valid),
    ("init uniform", pins.test_init_subsets_uniform),
    ("init on the published stream", pins.test_init_floyd_on_the_published_stream),
    ("init centers", pins.test_init_centers_are_the_drawn_colors),
    ("center distances", pins.test_center_distances_closed_form),
    ("row sort", pins.test_sort_rows_order_and_ties),
    ("hand-worked sort-means", pins.test_assign_hand_worked_cases),
    ("exhaustive minimum", lambda: pins.test_assign_finds_exhaustive_minimum_from_any_start(5)),
    ("exact fractions", pins.test_update_matches_exact_fractions),
    ("K=1 closed form", pins.test_k1_closed_form),
    ("empty cluster and SSE step", pins.test_empty_cluster_keeps_its_center_and_sse_is_taken_before_the_update),
    ("K=N' lossless", pins.test_k_equals_unique_count_is_lossless),
    ("weighted == batch", pins.test_weighted_equals_batch_kmeans),
    ("monotone + termination", pins.test_sse_never_increases_and_termination_rule),
    ("map + mse brute force", pins.test_map_and_mse_brute_force),
    ("indices beyond one byte", pins.test_map_and_mse_with_indices_beyond_one_byte),
    ("large palettes", pins.test_assign_finds_exhaustive_minimum_with_large_palettes),
    ("mse/psnr closed forms", pins.test_mse_psnr_closed_forms),
    ("gradient FD", pins.test_distortion_gradient_finite_differences),
    ("gradient at fixed point", pins.test_gradient_vanishes_at_a_lloyd_fixed_point),
]

# (what the mistake is, exact text in the oracle, replacement)
MUTANTS = [
    ("stop bound uses the running minimum",
     "if (d[(size_t)p * K + t] >= 4.0 * prev_dist) break;",
     "if (d[(size_t)p * K + t] >= 4.0 * min_dist) break;"),
    ("stop bound factor 2 instead of 4 (unsquared rule applied to squares)",
     ">= 4.0 * prev_dist) break;", ">= 2.0 * prev_dist) break;"),
    ("strict stop test", ">= 4.0 * prev_dist) break;", "> 4.0 * prev_dist) break;"),
    ("strict update test", "if (dist <= min_dist) {", "if (dist < min_dist) {"),
    ("scan skips the nearest neighbour", "for (int j = 1; j < K; ++j) {           /*",
     "for (int j = 2; j < K; ++j) {           /*"),
    ("dropped blue term in the distance", "return e0 * e0 + e1 * e1 + e2 * e2;",
     "return e0 * e0 + e1 * e1;"),
    ("unweighted cluster size", "        W[k] += n;\n", "        W[k] += 1;\n"),
    ("green numerator reads the blue channel",
     "S[3 * k + 1] += n * (int64_t)((colors[i] >> 8) & 255u);",
     "S[3 * k + 1] += n * (int64_t)(colors[i] & 255u);"),
    ("rows sorted farthest first", "if (drow[a] != drow[b]) return drow[a] < drow[b];",
     "if (drow[a] != drow[b]) return drow[a] > drow[b];"),
    ("row does not start with its own center", "if (ca != cb) return ca < cb;",
     "if (ca != cb) return ca > cb;"),
    ("SSE without the weights", "sse += ((double)counts[i] / N) * mind[i];",
     "sse += mind[i] / N;"),
    ("frequency counted twice", "counts[n_unique - 1] += 1;", "counts[n_unique - 1] += 2;"),
    ("Floyd draw range off by one", "% (uint64_t)(j + 1);", "% (uint64_t)(j + 2);"),
    ("MSE divided by the channel count too", "return n_pixels > 0 ? acc / (double)n_pixels",
     "return n_pixels > 0 ? acc / (3.0 * (double)n_pixels)"),
    ("relative change measured against the previous SSE",
     "(prev_sse - sse) / sse <= eps", "(prev_sse - sse) / prev_sse <= eps"),
    ("gradient sign flipped", "if (dC) dC[3 * a + c] += -2.0 * w[i] * diff;",
     "if (dC) dC[3 * a + c] += 2.0 * w[i] * diff;"),
    ("mixing constant mistyped", "0xBF58476D1CE4E5B9ull", "0xBF58476D1CE4E5B8ull"),
    ("index image truncated to one byte", "index[p] = labels[at];",
     "index[p] = (uint8_t)labels[at];"),
    ("palette index range check admits K", "if (k < 0 || k >= K) return -1.0;",
     "if (k < 0 || k > K) return -1.0;"),
    ("empty cluster moved to the origin",
     "        if (W[k] > 0)\n            for (int c = 0; c < 3; ++c) centers[3 * k + c] = (double)S[3 * k + c] / (double)W[k];",
     "        for (int c = 0; c < 3; ++c)\n            centers[3 * k + c] = W[k] > 0 ? (double)S[3 * k + c] / (double)W[k] : 0.0;"),
    ("SSE measured after the update instead of at the assignment step",
     "        sse = 0.0;\n        for (int64_t i = 0; i < n_unique; ++i) sse += ((double)counts[i] / N) * mind[i];\n"
     "        wsmo_update(colors, counts, n_unique, labels, K, centers, S_, W_);",
     "        wsmo_update(colors, counts, n_unique, labels, K, centers, S_, W_);\n        sse = 0.0;\n"
     "        for (int64_t i = 0; i < n_unique; ++i) {\n            double x[3], e = 0.0;\n"
     "            unpack(colors[i], x);\n"
     "            for (int c = 0; c < 3; ++c) {\n"
     "                const double t = x[c] - centers[3 * labels[i] + c];\n                e += t * t;\n            }\n"
     "            sse += ((double)counts[i] / N) * e;\n        }"),
    ("Floyd step draws with the candidate top as the counter",
     "uint64_t t = wsmo_splitmix64(seed, (uint64_t)taken) % (uint64_t)(j + 1);",
     "uint64_t t = wsmo_splitmix64(seed, (uint64_t)j) % (uint64_t)(j + 1);"),
]


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_rejected(what, old, new, tmp_path, monkeypatch):
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    lib = oracle.compile_variant(src.replace(old, new), os.path.join(tmp_path, "mutant.so"))
    monkeypatch.setattr(oracle, "_lib", lib)
    rejected = []
    with np.errstate(all="ignore"):
        for name, call in PIN_CALLS:
            try:
                call()
            except (AssertionError, ValueError, ZeroDivisionError, OverflowError, IndexError,
                    pytest.fail.Exception):   # a pytest.raises that saw no error
                rejected.append(name)
    assert rejected, f"no pin rejects the planted mistake: {what}"
