"""The full search space (all length-L sequences; labs_walks_full and
labs_saw_round_full) against the oracle's full-space walks, bit-exact:
trajectories, visited sets, bests, and whole solves."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2210_15962_gb300 import build
    build.build()
    import paper_2210_15962_gb300 as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle._load()
    return oracle


def compare_round(m, orc, L, seed, rnd, n_walks, walk_len, check_walks, trace_walks=(), recheck=0):
    tb, tc = (min(trace_walks), max(trace_walks) - min(trace_walks) + 1) if trace_walks else (0, 0)
    g = m.labs_saw_round(L, seed, rnd, n_walks, walk_len, recheck_every=recheck, trace_begin=tb, trace_count=tc,
                         space="full")
    for w in check_walks:
        o = orc.walk_trace(L, seed, w, rnd, walk_len, full=True)
        assert g["best_E"][w] == o["best_E"], (L, w)
        assert np.array_equal(g["best_seq"][w], o["best_seq"]), (L, w)
        assert g["moves"][w] == o["moves"] and g["stuck"][w] == o["stuck"], (L, w)
        assert g["best_step"][w] == o["best_step"], (L, w)
        if w in trace_walks:
            tr = g["trace"][w - tb]
            assert np.array_equal(tr[:o["moves"]], o["flips"]), (L, w)
            assert np.all(tr[o["moves"]:] == -1)
        assert orc.energy(g["best_seq"][w]) == g["best_E"][w]
    return g


@pytest.mark.parametrize("L", [3, 4, 5, 6, 8, 10])
def test_tiny_spaces_get_stuck(m, orc, L):
    wl = (1 << L) + 3
    g = compare_round(m, orc, L, 3, 1, 40, wl, range(40), trace_walks=range(40))
    assert g["stuck"].sum() == 40


@pytest.mark.parametrize("L", [12, 20, 31, 32, 33, 34, 63, 64, 65, 66, 97, 100, 127, 128, 129, 130, 160, 161,
                               192, 193, 200, 224, 225, 255, 256])
def test_lag_word_classes_and_ragged_tails(m, orc, L):
    # every lag-word class (L - 1 = 32 W and 32 W + 1 edges, both parities of L), every-step full recheck
    wl = 300 if L < 150 else 150
    compare_round(m, orc, L, 5 + L, 2, 70, wl, [0, 1, 31, 32, 33, 69], trace_walks=[0, 1, 31, 32, 33], recheck=1)


@pytest.mark.parametrize("L,wl,w", [(20, 2000, 3), (64, 600, 5), (129, 300, 1), (256, 150, 2)])
def test_visited_set_is_exactly_the_pivots(m, orc, L, wl, w):
    g = m.labs_saw_round(L, 9, 0, 8, wl, visited_walk=w, space="full")
    o = orc.walk_trace(L, 9, w, 0, wl, full=True)
    cur = orc.start_free_values(9, w, 0, L).copy()

    def key(v):
        return sum(1 << j for j, x in enumerate(v) if x < 0)

    want = {key(cur)}
    for j in o["flips"]:
        cur[j] = -cur[j]
        want.add(key(cur))
    got = set()
    for row in g["visited"]:
        v = 0
        for i, wd in enumerate(row):
            v |= int(wd) << (64 * i)
        got.add(v)
    assert g["visited_count"] == len(want) == o["moves"] + 1
    assert got == want


def test_solve_multi_seed_rounds_target_and_cap(m, orc):
    L, walks, wl = 40, 50, 200
    per_round = walks * wl * L
    seeds = [3, 4, 5]
    g = m.labs_walks(L, seeds, walks, wl, 2 * per_round + 1, space="full")
    o = orc.solve(L, seeds, walks, wl, 2 * per_round + 1, threads=8, full=True)
    assert np.array_equal(g["best_E"], o["best_E"]) and np.array_equal(g["best_seq"], o["best_seq"])
    assert np.array_equal(g["evals"].astype(np.int64), o["evals"].astype(np.int64))
    assert list(g["rounds"]) == list(o["rounds"]) == [3, 3, 3]
    tgt = int(o["best_E"].max()) + 6
    g2 = m.labs_walks(L, seeds, walks, wl, 10 ** 12, target_E=tgt, space="full")
    o2 = orc.solve(L, seeds, walks, wl, 10 ** 12, target_E=tgt, threads=8, full=True)
    assert np.array_equal(g2["best_E"], o2["best_E"]) and list(g2["rounds"]) == list(o2["rounds"])
    assert np.array_equal(g2["best_seq"], o2["best_seq"])
    g3 = m.labs_walks(L, seeds, walks, wl, 10 ** 12, max_rounds=2, space="full")
    assert list(g3["rounds"]) == [2, 2, 2]


def test_large_launch_sampled(m, orc):
    # L=128: 65536 walks of 1024 steps in one launch; oracle on sampled walks
    L, n, wl = 128, 65536, 1024
    compare_round(m, orc, L, 1, 0, n, wl, [0, 1, 32767, 65535], trace_walks=[0, 1])


def test_reaches_small_optima(m, orc):
    # the solve reaches the optimum of Eq. 1 found by the oracle's own exhaustive-size solves
    for L in (11, 13, 20):
        o = orc.solve(L, [7], 256, 8 * L, 256 * 8 * L * L * 4, threads=8, full=True)
        g = m.labs_walks(L, [7], 256, 8 * L, 256 * 8 * L * L * 4, space="full")
        assert int(g["best_E"][0]) == int(o["best_E"][0])
