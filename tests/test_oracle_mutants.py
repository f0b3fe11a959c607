"""Planted mistakes in the oracle must fail its pins.

The oracle is pinned by the tests of test_oracle.py: Table 1 of the paper,
closed forms, numpy's correlation, the Random123 known-answer vectors,
brute-force replays of whole walks, the round logic of Algorithm 1, and the
predictive model against Table 1's probabilities.  Each mutant below is one
plausible slip -- a dropped or extra term, a wrong sign or index, an
off-by-one bound, a non-strict comparison, a swapped constant -- planted in a
temporary copy of the oracle package, never in oracle/ itself.  The copy is
built and the pins run against it in a child process (so that a crash or a
hang of a mutant cannot take the test run with it).  Every mutant must make
at least one pin fail, and the unmodified copy must pass them all: this is
what shows that the pins pin the oracle, and not only that the oracle agrees
with itself.
"""
import concurrent.futures
import json
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE_FILES = ("__init__.py", "build.py", "labs_oracle.cpp")

# (name, file of oracle/, original text -- must occur exactly once --, planted text)
MUTANTS = [
    # Eq. 1
    ("eq1_sum_one_term_short", "labs_oracle.cpp",
     "for (int i = 0; i + k < L; ++i) c += (int64_t)s[i] * (int64_t)s[i + k];",
     "for (int i = 0; i + k < L - 1; ++i) c += (int64_t)s[i] * (int64_t)s[i + k];"),
    ("eq1_energy_from_lag_0", "labs_oracle.cpp",
     "for (int k = 1; k < L; ++k) {\n    int64_t c = autocorrelation(s, L, k);",
     "for (int k = 0; k < L; ++k) {\n    int64_t c = autocorrelation(s, L, k);"),
    ("eq1_magnitude_not_square", "labs_oracle.cpp",
     "    e += c * c;", "    e += c < 0 ? -c : c;"),
    # Eq. 2
    ("eq2_sign_pattern", "labs_oracle.cpp",
     "(i & 1) ? -s[c - i] : s[c - i]", "(i & 1) ? s[c - i] : -s[c - i]"),
    ("eq2_mirror_index", "labs_oracle.cpp",
     "s[c + i] = (int8_t)((i & 1) ? -s[c - i] : s[c - i]);",
     "s[c + i] = (int8_t)((i & 1) ? -s[c - i + 1] : s[c - i + 1]);"),
    # Philox4x32-10 and the start layout
    ("philox_multiplier_operand", "labs_oracle.cpp",
     "const uint64_t p0 = (uint64_t)0xD2511F53u * x.v[0];", "const uint64_t p0 = (uint64_t)0xD2511F53u * x.v[1];"),
    ("philox_nine_rounds", "labs_oracle.cpp",
     "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {"),
    ("philox_weyl_constant", "labs_oracle.cpp",
     "k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;"),
    ("philox_output_words", "labs_oracle.cpp",
     "y.v[0] = hi1 ^ x.v[1] ^ k0;", "y.v[0] = hi0 ^ x.v[1] ^ k0;"),
    ("start_block_of_value", "labs_oracle.cpp",
     "(uint32_t)(j / 128)", "(uint32_t)(j / 64)"),
    ("start_word_of_value", "labs_oracle.cpp",
     "r.v[(j / 32) % 4]", "r.v[(j / 32) % 2]"),
    ("start_bit_convention", "labs_oracle.cpp",
     "((word >> (j % 32)) & 1u) ? (int8_t)-1 : (int8_t)1;", "((word >> (j % 32)) & 1u) ? (int8_t)1 : (int8_t)-1;"),
    # the neighbourhood evaluation and the walk (Eq. 3, Algorithm 2)
    ("sidelobe_change_sign", "labs_oracle.cpp",
     "if (a != b) d += -2 * (int64_t)s[i] * (int64_t)s[i + k];", "if (a != b) d += 2 * (int64_t)s[i] * (int64_t)s[i + k];"),
    ("sidelobe_change_pairs", "labs_oracle.cpp",
     "if (a != b) d += -2", "if (a || b) d += -2"),
    ("delta_dropped_square", "labs_oracle.cpp",
     "delta += (C[k] + dC[k]) * (C[k] + dC[k]) - C[k] * C[k];", "delta += 2 * C[k] * dC[k];"),
    ("ties_to_highest_flip", "labs_oracle.cpp",
     "if (best_j < 0 || delta < best_delta) {", "if (best_j < 0 || delta <= best_delta) {"),
    ("first_pivot_not_visited", "labs_oracle.cpp",
     "  visited.insert(key_of(s, D));\n\n  WalkResult res;", "\n  WalkResult res;"),
    ("visited_probe_wrong_bit", "labs_oracle.cpp",
     "nk[j] = (int8_t)-nk[j];", "nk[D - 1 - j] = (int8_t)-nk[D - 1 - j];"),
    ("move_forgets_mirror", "labs_oracle.cpp",
     "    s[p] = (int8_t)-s[p];\n    if (q != p) s[q] = (int8_t)-s[q];\n    for (int k = 1; k < L; ++k) C[k] += best_dC[k];",
     "    s[p] = (int8_t)-s[p];\n    for (int k = 1; k < L; ++k) C[k] += best_dC[k];"),
    ("mirror_off_by_one", "labs_oracle.cpp",
     "int mirror(int j) const { return full ? j : L - 1 - j; }",
     "int mirror(int j) const { return full ? j : L - 2 - j; }"),
    ("walk_best_not_strict", "labs_oracle.cpp",
     "if (E < res.best_E) {", "if (E <= res.best_E) {"),
    ("walk_one_step_short", "labs_oracle.cpp",
     "for (int step = 1; step <= walk_len; ++step) {", "for (int step = 1; step < walk_len; ++step) {"),
    ("evals_d_minus_1_per_step", "labs_oracle.cpp",
     "res.evals += D;", "res.evals += D - 1;"),
    ("full_space_one_flip_short", "labs_oracle.cpp",
     "int free_values() const { return full ? L : (L + 1) / 2; }",
     "int free_values() const { return full ? L - 1 : (L + 1) / 2; }"),
    # the round loop (Algorithm 1)
    ("budget_checked_strictly", "labs_oracle.cpp",
     "if (done >= step_budget) break;", "if (done > step_budget) break;"),
    ("target_checked_strictly", "labs_oracle.cpp",
     "if (target_E >= 0 && cur <= target_E) break;", "if (target_E >= 0 && cur < target_E) break;"),
    ("round_best_ties_to_latest", "labs_oracle.cpp",
     "if (cur < 0 || bE[w] < cur) {", "if (cur < 0 || bE[w] <= cur) {"),
    # the predictive model (Section 4.1, Eq. 6, Eq. 7)
    ("model_rate_base", "__init__.py",
     "return 0.006753 * 0.8617 ** L", "return 0.006753 * 0.8671 ** L"),
    ("model_eq6_without_runs", "__init__.py",
     "return math.log(1.0 - P) / (-model_lambda(L) * N)", "return math.log(1.0 - P) / (-model_lambda(L))"),
    ("model_eq7_rate_of_next_length", "__init__.py",
     "return 1.0 - math.exp(-model_lambda(L) * nses)", "return 1.0 - math.exp(-model_lambda(L + 2) * nses)"),
    ("model_count_conversion_inverted", "__init__.py",
     "return evals * (D - 1) / D", "return evals * D / (D - 1)"),
]


def pins(t, oracle):
    """The pins of test_oracle.py as (name, callable) pairs, cheapest first."""
    rows = t.read_rows("table1_skew_sequences.txt")
    kat = t.read_rows("philox4x32_10_kat.txt")
    return [
        ("table1", lambda: [t.test_table1_energy_and_merit(oracle, r) for r in rows]),
        ("table1_bit_order", lambda: t.test_table1_bit_order_matters(oracle)),
        ("barker", lambda: [t.test_barker_sequences(oracle, L) for L in sorted(t.BARKER)]),
        ("closed_forms", lambda: [t.test_constant_and_alternating(oracle, L) for L in (1, 2, 3, 10, 27, 64)]),
        ("exhaustive", lambda: [t.test_exhaustive_vs_numpy_and_invariants(oracle, L) for L in (5, 7, 9, 11, 13)]),
        ("random_vs_numpy", lambda: [t.test_random_sequences_vs_numpy(oracle, L) for L in (2, 3, 64, 121, 449)]),
        ("philox_kat", lambda: [t.test_philox_known_answers(oracle, r) for r in kat]),
        ("start_layout", lambda: t.test_start_stream_layout(oracle)),
        ("walks_small", lambda: [t.test_walks_vs_bruteforce_small_with_stuck(oracle, L, n)
                                 for L, n in [(5, 12), (7, 40), (9, 300), (11, 64), (13, 200)]]),
        ("walks_L27", lambda: t.test_walks_vs_bruteforce_L27()),
        ("incremental", lambda: t.test_incremental_matches_eq1_every_step(oracle, 61)),
        ("round_logic", lambda: t.test_batch_and_solve_round_logic(oracle)),
        ("round_boundaries", lambda: t.test_round_boundaries_and_ties(oracle)),
        ("model_eq6_eq7", lambda: [t.test_model_eq6_inverts_eq7(oracle, L, P, N)
                                   for L in (71, 223) for P in (0.5, 0.99) for N in (1, 100)]),
        ("model_exponential", lambda: [t.test_model_exponential_properties(oracle, L) for L in (71, 449)]),
        ("model_table1", lambda: t.test_model_matches_table1_probabilities(oracle)),
        ("model_count", lambda: t.test_model_counts_d_minus_1_per_step(oracle)),
        ("full_walks", lambda: [t.test_full_space_walks_vs_bruteforce(oracle, L, n)
                                for L, n in [(2, 5), (3, 10), (5, 40), (8, 300), (13, 600)]]),
        ("full_optimum", lambda: t.test_full_space_reaches_the_brute_force_optimum(oracle)),
        ("full_incremental", lambda: [t.test_full_space_incremental_matches_eq1(oracle, L) for L in (20, 33)]),
    ]


def child(copy_root, stop_at_first):
    """Run the pins against the oracle package under copy_root; print the failures."""
    sys.path.insert(0, copy_root)  # the planted copy's `oracle` before the repository's
    sys.path.insert(1, HERE)
    import oracle
    assert os.path.dirname(os.path.abspath(oracle.__file__)) == os.path.join(copy_root, "oracle")
    import test_oracle as t
    failed = []
    for name, fn in pins(t, oracle):
        try:
            fn()
        except Exception:  # an assertion, or a wrapper refusing a result
            failed.append(name)
            if stop_at_first:
                break
    print(json.dumps({"failed": failed}))


def run_copy(mutant):
    """Build a copy of oracle/ (with `mutant` planted, if any) and run the pins on it."""
    tmp = tempfile.mkdtemp(prefix="oracle_copy_")
    try:
        dst = os.path.join(tmp, "oracle")
        os.makedirs(dst)
        for f in ORACLE_FILES:
            shutil.copy(os.path.join(ROOT, "oracle", f), dst)
        if mutant is not None:
            _, fname, old, new = mutant
            path = os.path.join(dst, fname)
            with open(path) as fh:
                src = fh.read()
            assert src.count(old) == 1, "mutant %s: its original text must occur exactly once" % mutant[0]
            with open(path, "w") as fh:
                fh.write(src.replace(old, new))
        subprocess.run([sys.executable, "-c", "import sys; sys.path.insert(0, sys.argv[1]); "
                        "from oracle.build import build; build(force=True)", tmp],
                       check=True, capture_output=True, timeout=300)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), tmp, "0" if mutant is None else "1"],
                           capture_output=True, text=True, timeout=300)
        if r.returncode != 0:
            return {"crashed": r.returncode, "stderr": r.stderr[-2000:]}
        return json.loads(r.stdout.strip().splitlines()[-1])
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


@pytest.fixture(scope="module")
def outcomes():
    jobs = [("unmodified", None)] + [(m[0], m) for m in MUTANTS]
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {name: ex.submit(run_copy, m) for name, m in jobs}
        return {name: f.result() for name, f in futs.items()}


def test_unmodified_copy_passes_every_pin(outcomes):
    assert outcomes["unmodified"] == {"failed": []}


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    got = outcomes[name]
    assert "crashed" not in got, got  # a pin, not a crash, has to catch it
    assert got["failed"], "the mistake %s passes every pin" % name


def test_mutants_are_distinct_and_compile_in_place():
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, fname, old, new in MUTANTS:
        assert old != new
        with open(os.path.join(ROOT, "oracle", fname)) as fh:
            assert fh.read().count(old) == 1, name


if __name__ == "__main__":
    child(sys.argv[1], sys.argv[2] == "1")
