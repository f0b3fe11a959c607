"""Batched persistent path: every problem's result is exactly what labs_walks
gives for it alone (same L, seed, walks, walk length, budget, target), for
mixes of lag-word classes, uneven budgets, targets, stuck walks, CUDA graph
replay and autotuned launch shapes; plus oracle checks on small problems."""
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


def alone(m, p):
    L, walks, wl, seed, budget = p[:5]
    tgt = p[5] if len(p) > 5 else -1
    r = m.labs_walks(L, [seed], walks, wl, budget, target_E=tgt)
    return {"best_E": int(r["best_E"][0]), "best_seq": r["best_seq"][0], "evals": int(r["evals"][0]),
            "rounds": int(r["rounds"][0])}


def check_same(m, probs, results):
    for p, g in zip(probs, results):
        a = alone(m, p)
        assert g["best_E"] == a["best_E"], p
        assert np.array_equal(g["best_seq"], a["best_seq"]), p
        assert g["evals"] == a["evals"] and g["rounds"] == a["rounds"], (p, g["evals"], a["evals"])


MIX = [
    # L, walks, walk_len, seed, budget[, target]
    (27, 64, 300, 1, 64 * 300 * 14 * 3 + 1),          # W=1, 4 rounds
    (61, 100, 250, 2, 1),                              # W=1 edge (m=30), 1 round, ragged chunk
    (65, 70, 200, 3, 70 * 200 * 33 * 2),               # W=1 (m=32)
    (67, 96, 200, 4, 96 * 200 * 34 * 2 + 5),           # W=2 (m=33)
    (121, 128, 300, 5, 128 * 300 * 61 * 2),            # W=2
    (131, 33, 150, 6, 33 * 150 * 66 * 3),              # W=3
    (199, 40, 120, 7, 1, -1),                          # W=4
    (223, 64, 100, 8, 10 ** 12, 4600),                 # W=4, target reached in round 0 (later rounds speculative)
    (301, 32, 80, 9, 32 * 80 * 151 * 2),               # W=5
]


def test_mixed_batch_equals_alone(m):
    with m.Batch(MIX) as b:
        st = b.run()
        check_same(m, MIX, b.results())
        assert st["walk_launches"] >= 1 and st["evals"] == sum(b.result(i)["evals"] for i in range(len(MIX)))
        # a second run of the same batch gives the same results
        b.run()
        check_same(m, MIX, b.results())


def test_graph_replay_and_autotune_equal_alone(m):
    probs = [p for p in MIX if len(p) == 5]  # graphs are used when no problem has a target
    with m.Batch(probs, use_graph=True, autotune=True) as b:
        for _ in range(3):
            b.run()
            check_same(m, probs, b.results())
        for W in {((p[0] - 1) // 2 + 31) // 32 for p in probs}:
            sh = b.shape(W)
            assert sh["block_threads"] in (64, 128, 256) and sh["table_factor_x10"] in (15, 30)
            assert sh["resident_walks"] > 0


def test_stuck_walks_need_continuation_launches(m):
    # tiny spaces: walks get stuck, rounds fall short of the estimate and the
    # batch must launch again to reach the budget
    probs = [(5, 40, 30, 3, 40 * 30 * 3 * 4), (7, 40, 60, 4, 40 * 60 * 4 * 3), (9, 64, 100, 5, 64 * 100 * 5 * 2)]
    with m.Batch(probs, use_graph=True) as b:
        for _ in range(2):
            st = b.run()
            check_same(m, probs, b.results())
        assert st["walk_launches"] > 1


def test_batch_vs_oracle_small(m):
    import oracle
    probs = [(27, 64, 4096, 1, 64 * 4096 * 14), (33, 50, 500, 12, 50 * 500 * 17 * 2)]
    with m.Batch(probs) as b:
        b.run()
        for p, g in zip(probs, b.results()):
            o = oracle.solve(p[0], [p[3]], p[1], p[2], p[4], threads=8)
            assert g["best_E"] == int(o["best_E"][0])
            assert np.array_equal(g["best_seq"], o["best_seq"][0])
            assert g["evals"] == int(o["evals"][0]) and g["rounds"] == int(o["rounds"][0])


def test_many_instances_config3_shape(m):
    # the shape of the batched workload (odd L in [101, 223], walk length 8*D,
    # log-uniform budgets, seed 1000+i), scaled down to 12 instances x 256 walks
    from paper_2210_15962_gb300 import workloads
    wl = workloads.batched_instances(n=12, walks=256, bmin=2e6, bmax=2e7)
    probs = [(p.L, p.walks, p.walk_len, p.seed, p.step_budget) for p in wl.problems]
    with m.Batch(probs, use_graph=True) as b:
        b.run()
        check_same(m, probs, b.results())


def test_full_size_batched_workload_vs_oracle_sampled(m):
    # the batched workload at its full size and in the bench's launch
    # configuration (64 instances of odd L in [101, 223], 2048 walks of 8*D
    # steps, log-uniform budgets, CUDA graph, autotuned shapes); the instance
    # the oracle solves fastest (L=117, two rounds of 2048 walks) is compared
    # with it directly, the next seven with one labs_walks each
    import os
    import oracle
    from paper_2210_15962_gb300 import workloads
    wl = workloads.batched_instances(n=64, walks=2048)
    probs = [(p.L, p.walks, p.walk_len, p.seed, p.step_budget) for p in wl.problems]
    with m.Batch(probs, use_graph=True, autotune=True) as b:
        b.run()
        res = b.results()
    cost = sorted(range(len(probs)), key=lambda i: -(-probs[i][4] // (probs[i][1] * probs[i][2] * ((probs[i][0] + 1) // 2)))
                  * probs[i][1] * probs[i][2] * probs[i][0] ** 2)
    for i in cost[:1]:
        L, walks, wlen, seed, budget = probs[i]
        o = oracle.solve(L, [seed], walks, wlen, budget, threads=os.cpu_count() or 8)
        g = res[i]
        assert g["best_E"] == int(o["best_E"][0]) and np.array_equal(g["best_seq"], o["best_seq"][0]), probs[i]
        assert g["evals"] == int(o["evals"][0]) and g["rounds"] == int(o["rounds"][0]), probs[i]
    for i in cost[1:8]:
        a = alone(m, probs[i])
        assert res[i]["best_E"] == a["best_E"] and res[i]["evals"] == a["evals"], probs[i]


def oracle_result(p, threads=8):
    import oracle
    L, walks, wl, seed, budget = p[:5]
    tgt = p[5] if len(p) > 5 else -1
    o = oracle.solve(L, [seed], walks, wl, budget, target_E=tgt, threads=threads)
    return {"best_E": int(o["best_E"][0]), "best_seq": o["best_seq"][0], "evals": int(o["evals"][0]),
            "rounds": int(o["rounds"][0])}


def check_oracle(probs, results):
    for p, g in zip(probs, results):
        o = oracle_result(p)
        assert g["best_E"] == o["best_E"], (p, g["best_E"], o["best_E"])
        assert np.array_equal(g["best_seq"], o["best_seq"]), p
        assert g["evals"] == o["evals"] and g["rounds"] == o["rounds"], (p, g["evals"], o["evals"])


def target_after_rounds(L, walks, wl, seed, rounds):
    """A target energy the oracle first reaches within `rounds` rounds (its best after them)."""
    D = (L + 1) // 2
    return oracle_result((L, walks, wl, seed, walks * wl * D * rounds))["best_E"]


# one problem per lag-word class W = ceil(((L-1)/2)/32), each with its own
# word edge: L = 61 (m=30, W=1), 67 (m=33, W=2), 129 (m=64, W=2 full), 131 (W=3),
# 161 (W=3), 223 (W=4), 259 (m=129, W=5), 301 (W=5), 383 (W=6), 449 (W=7), 511 (W=8);
# several rounds each, ragged chunks (walks not a multiple of 32)
CLASS_PROBS = [
    (61, 40, 160, 101, 40 * 160 * 31 * 3),
    (67, 33, 150, 102, 33 * 150 * 34 * 2),
    (129, 45, 140, 103, 45 * 140 * 65 * 2 + 1),
    (131, 32, 120, 104, 32 * 120 * 66 * 2),
    (161, 50, 120, 105, 50 * 120 * 81 * 3),
    (223, 37, 110, 106, 37 * 110 * 112 * 2),
    (259, 32, 100, 107, 32 * 100 * 130 * 2),
    (301, 40, 100, 108, 40 * 100 * 151 * 2),
    (383, 32, 80, 109, 32 * 80 * 192 * 2),
    (449, 36, 80, 110, 36 * 80 * 225 * 2),
    (511, 32, 60, 111, 32 * 60 * 256 * 2),
]


def test_batch_vs_oracle_every_class(m):
    # the persistent batch kernel of every lag-word class (its own code: pattern
    # loops, register budgets) against the oracle's Algorithm 1 + Algorithm 2
    with m.Batch(CLASS_PROBS) as b:
        b.run()
        check_oracle(CLASS_PROBS, b.results())


def test_batch_vs_oracle_targets_and_graph(m):
    # target problems (stop at the first round reaching E <= target, later rounds
    # run speculatively and are ignored) beside budget problems, one per class
    # W = 2..5, and the CUDA-graph path for the budget-only mix
    probs = []
    for L, walks, wl, seed in [(121, 40, 150, 201), (161, 33, 120, 202), (223, 32, 100, 203), (301, 32, 80, 204)]:
        tgt = target_after_rounds(L, walks, wl, seed, 2)
        probs.append((L, walks, wl, seed, 10 ** 12, tgt))
    probs.append((121, 64, 200, 205, 64 * 200 * 61 * 3))
    with m.Batch(probs, rounds_per_launch=2) as b:
        b.run()
        res = b.results()
        check_oracle(probs, res)
        assert all(r["rounds"] <= 2 for r in res[:4])
    budget_only = [p for p in CLASS_PROBS[:6]]
    with m.Batch(budget_only, use_graph=True, autotune=True) as b:
        for _ in range(2):
            b.run()
            check_oracle(budget_only, b.results())


def test_batch_warp_mode_vs_oracle_every_class(m):
    # one walk per warp (the lanes split each walk's flips) in every class,
    # budget and target problems, against the oracle
    probs = list(CLASS_PROBS)
    tgt = target_after_rounds(161, 40, 120, 401, 2)
    probs.append((161, 40, 120, 401, 10 ** 12, tgt))
    with m.Batch(probs, walk_mode=2, rounds_per_launch=2) as b:
        b.run()
        check_oracle(probs, b.results())
        for W in {((p[0] - 1) // 2 + 31) // 32 for p in probs}:
            assert b.shape(W)["warp_per_walk"]


def test_batch_cta_mode_vs_oracle_every_class(m):
    # one walk per CTA of 128 threads (its warps split each walk's flips and
    # merge their candidates in shared memory) in every class, budget and
    # target problems, against the oracle
    probs = list(CLASS_PROBS)
    tgt = target_after_rounds(161, 40, 120, 401, 2)
    probs.append((161, 40, 120, 401, 10 ** 12, tgt))
    with m.Batch(probs, walk_mode=3, rounds_per_launch=2) as b:
        b.run()
        check_oracle(probs, b.results())
        for W in {((p[0] - 1) // 2 + 31) // 32 for p in probs}:
            sh = b.shape(W)
            assert sh["cta_per_walk"] and sh["walk_unit"] == "cta"


def test_batch_autotune_offers_warp_mode(m):
    # few walks per class: the autotuner times lane, warp and CTA mode on the
    # first launch's tasks; whatever it picks, the results are the oracle's
    probs = [(301, 64, 300, 501, 64 * 300 * 151), (449, 48, 200, 502, 48 * 200 * 225 * 2)]
    with m.Batch(probs, autotune=True) as b:
        b.run()
        check_oracle(probs, b.results())
        for W in (5, 7):
            sh = b.shape(W)
            assert sh["block_threads"] in (64, 128, 256) and sh["resident_walks"] > 0


def test_batch_rounds_after_a_stop_are_never_counted(m):
    # every problem reaches its target in its first round while 16 of its
    # rounds are issued in the launch: whatever order the chunks finish in
    # around the stopping round's finalization, the later rounds add neither
    # evaluations nor rounds (Algorithm 1), in lane, warp and CTA mode
    probs = []
    for i in range(48):
        L = (61, 121, 161)[i % 3]
        walks, wl, seed = 64, 120, 800 + i
        probs.append((L, walks, wl, seed, 10 ** 12, target_after_rounds(L, walks, wl, seed, 1)))
    for mode in (1, 2, 3):
        with m.Batch(probs, rounds_per_launch=16, walk_mode=mode) as b:
            b.run()
            res = b.results()
        for p, r in zip(probs, res):
            L, walks, wl = p[:3]
            assert r["rounds"] == 1 and r["evals"] == walks * wl * ((L + 1) // 2), (mode, p, r["rounds"], r["evals"])
            assert r["best_E"] == p[5]
