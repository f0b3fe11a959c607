"""The predictive model behind the C ABI (labs_model_*, Section 4.1, Eq. 6,
Eq. 7) against the oracle's restatement.  Host arithmetic only: these run
without a GPU (the library is loaded, no device call is made)."""
import math

import pytest


@pytest.fixture(scope="module")
def m():
    from paper_2210_15962_gb300 import build
    build.build()
    import paper_2210_15962_gb300 as mod
    mod.load()
    return mod


LS = [5, 27, 71, 117, 121, 171, 223, 247, 301, 449, 511]


@pytest.mark.parametrize("L", LS)
def test_lambda_and_conversion_match_oracle(m, oracle_mod, L):
    assert m.labs_model_lambda(L) == pytest.approx(oracle_mod.model_lambda(L), rel=1e-13)
    for evals in [0, 1, 10 ** 6, 131072 * 8192 * ((L + 1) // 2), 2 ** 62]:
        assert m.labs_model_nses_of_evals(L, evals) == pytest.approx(oracle_mod.model_nses_of_evals(L, evals),
                                                                      rel=1e-13, abs=1e-300)


@pytest.mark.parametrize("L", LS)
@pytest.mark.parametrize("P", [0.0, 0.13, 0.5, 0.99, 0.999999])
@pytest.mark.parametrize("N", [1, 100])
def test_eq6_eq7_match_oracle(m, oracle_mod, L, P, N):
    n = m.labs_model_nses_limit(L, P, N)
    assert n == pytest.approx(oracle_mod.model_nses_limit(L, P, N), rel=1e-12, abs=1e-300)
    # probabilities to 1e-15: the oracle's plain 1 - exp(-x) rounds at that level where x is small
    for x in [0.0, n, 0.5 * n, 3.0 * n + 1.0, 1e3]:
        assert m.labs_model_p_optimal(L, x) == pytest.approx(oracle_mod.model_p_optimal(L, x), rel=1e-12,
                                                              abs=1e-15)


@pytest.mark.parametrize("L", [27, 121, 171, 223, 449])
@pytest.mark.parametrize("P", [0.5, 0.99])
def test_budget_is_the_first_count_reaching_P(m, L, P):
    b = m.labs_model_budget(L, P)
    assert b >= 1
    if b < 2 ** 52:  # exact in double
        assert m.labs_model_p_optimal(L, m.labs_model_nses_of_evals(L, b)) >= P * (1 - 1e-12)
        assert m.labs_model_p_optimal(L, m.labs_model_nses_of_evals(L, b - 1)) < P * (1 + 1e-12)


def test_invalid_arguments(m):
    for L in [4, 3, 513, -1]:
        assert math.isnan(m.labs_model_lambda(L))
        assert m.labs_model_budget(L, 0.5) == 0
    assert math.isnan(m.labs_model_nses_limit(121, 1.0, 1))
    assert math.isnan(m.labs_model_nses_limit(121, -0.1, 1))
    assert math.isnan(m.labs_model_nses_limit(121, 0.5, 0))
    assert math.isnan(m.labs_model_p_optimal(121, -1.0))
    assert m.labs_model_budget(121, 1.0) == 0
    assert m.labs_model_budget(511, 0.999999) == 2 ** 64 - 1  # saturates
