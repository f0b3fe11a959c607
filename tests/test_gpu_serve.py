"""Serving with continuous batching: every request's result is exactly what
labs_walks gives for it alone, whether submitted at once, while others run,
or throttled by memory admission; plus the server's error paths (bad or
oversized requests, unknown tickets, timeouts, shutdown with work in flight).
All failures here are made on the host: no GPU fault is involved."""
import threading
import time

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
    return int(r["best_E"][0]), r["best_seq"][0], int(r["evals"][0]), int(r["rounds"][0])


def check(m, p, res):
    import oracle
    E, seq, ev, rd = alone(m, p)
    assert res["status"] == m.LABS_OK
    assert res["best_E"] == E and np.array_equal(res["best_seq"], seq), p
    assert res["evals"] == ev and res["rounds"] == rd, p
    assert res["t_submit_ns"] <= res["t_admit_ns"] <= res["t_done_ns"]
    # Eq. 7 of the predictive model for the request's evaluations
    L = p[0]
    want = oracle.model_p_optimal(L, oracle.model_nses_of_evals(L, res["evals"]))
    assert res["p_optimal"] == pytest.approx(want, rel=1e-12, abs=1e-15), p


REQS = [
    (27, 64, 216, 1, 64 * 216 * 14 * 3),
    (121, 256, 488, 2, 256 * 488 * 61 * 2),
    (131, 128, 528, 3, 128 * 528 * 66 * 3),
    (223, 96, 896, 4, 1),
    (301, 64, 1208, 5, 64 * 1208 * 151 * 2),
    (161, 200, 648, 6, 10 ** 12, 3300),  # target: stops after the first round reaching E <= 3300
]


def test_requests_same_alone_and_mixed(m):
    with m.Server(max_walks=256) as sv:
        tickets = [sv.submit(*p) for p in REQS]
        results = [sv.wait(t) for t in tickets]
        for p, r in zip(REQS, results):
            check(m, p, r)
        st = sv.stats()
        assert st["completed"] == len(REQS) and st["pending"] == 0 and st["active"] == 0
        assert st["evals"] == sum(r["evals"] for r in results)


def test_requests_arriving_while_others_run(m):
    # the first request runs 40 rounds of 2048 walks at L=301 (several hundred
    # ms on its own), so the others, submitted 10 ms apart, arrive while it is
    # on the GPU
    first = (301, 2048, 1208, 12, 2048 * 1208 * 151 * 40)
    reqs = [first] + REQS
    with m.Server(max_walks=2048, rounds_per_launch=1) as sv:
        tickets = [sv.submit(*first)]
        for p in REQS:
            time.sleep(0.01)
            tickets.append(sv.submit(*p))
        results = [sv.wait(t) for t in tickets]
    for p, r in zip(reqs, results):
        check(m, p, r)
    assert results[0]["rounds"] == 40
    # later requests were admitted, and finished, while the first one was running
    assert any(r["t_admit_ns"] < results[0]["t_done_ns"] for r in results[1:])
    assert any(r["t_done_ns"] < results[0]["t_done_ns"] for r in results[1:])


def launch_bytes(walks, walk_len, L, rounds):
    """Arena bytes of one launch over one request that runs `rounds` rounds: a visited
    table (power-of-two slots >= 3 x pivots, 64-bit words of D + 1 bits) for each
    walk of each round in flight, plus its lists (under 64 KiB here)."""
    slots = 64
    while slots < (walk_len + 1) * 3 + 1:
        slots *= 2
    words = slots * (((L + 1) // 2 + 1 + 63) // 64)
    words += words % 2
    return ((walks + 31) // 32) * 32 * rounds * words * 8


def test_memory_admission_serialises_and_rejects(m):
    big = (121, 256, 488, 7, 256 * 488 * 61 * 3)
    rpl = 4
    one = launch_bytes(256, 488, 121, rpl)
    # each of the two launches in flight gets half of the arena: room for one such request, not two
    mem = 2 * (one + (64 << 10))
    with m.Server(max_walks=256, mem_bytes=mem, rounds_per_launch=rpl) as sv:
        t1 = sv.submit(*big)
        t2 = sv.submit(121, 256, 488, 8, 256 * 488 * 61)
        r1, r2 = sv.wait(t1), sv.wait(t2)
        check(m, big, r1)
        check(m, (121, 256, 488, 8, 256 * 488 * 61), r2)
        assert r2["t_admit_ns"] >= r1["t_done_ns"]  # admitted only once the first left
        st = sv.stats()
        assert 0 < st["mem_peak"] <= mem // 2
        with pytest.raises(m.LabsError) as ei:
            sv.submit(121, 256, 4000, 9, 10 ** 9)  # one launch of it alone exceeds half the arena
        assert ei.value.status == m.LABS_ENOMEM
        with pytest.raises(m.LabsError) as ei:
            sv.submit(401, 64, 100, 9, 10 ** 6)  # above the server's max_L
        assert ei.value.status == m.LABS_ENOMEM
        with pytest.raises(m.LabsError) as ei:
            sv.submit(120, 64, 100, 9, 10 ** 6)  # even L
        assert ei.value.status == m.LABS_EINVAL


def test_device_bytes_stay_within_the_arena_while_requests_queue(m):
    # requests of three classes queue behind a small arena; the bytes any launch
    # uses never exceed its half, every request completes and matches labs_walks
    reqs = [(121, 128, 488, 40 + i, 128 * 488 * 61 * 2) for i in range(3)] + \
           [(161, 96, 648, 50 + i, 96 * 648 * 81 * 2) for i in range(2)] + [(223, 64, 896, 60, 64 * 896 * 112)]
    rpl = 2
    mem = 2 * (launch_bytes(128, 488, 121, rpl) + launch_bytes(64, 896, 223, rpl) + (256 << 10))
    with m.Server(max_walks=128, mem_bytes=mem, rounds_per_launch=rpl) as sv:
        tickets = [sv.submit(*p) for p in reqs]
        seen = []
        while len(seen) < 400:
            st = sv.stats()
            seen.append((st["mem_used"], st["mem_peak"], st["pending"]))
            if st["completed"] == len(reqs):
                break
            time.sleep(0.005)
        results = [sv.wait(t) for t in tickets]
        st = sv.stats()
    assert all(u <= mem // 2 and pk <= mem // 2 for u, pk, _ in seen)
    assert 0 < st["mem_peak"] <= mem // 2
    assert any(q > 0 for _, _, q in seen)  # requests did wait for memory
    for p, r in zip(reqs, results):
        check(m, p, r)


def test_tickets_timeouts_and_shutdown(m):
    sv = m.Server(max_walks=2048, max_active=2)
    with pytest.raises(m.LabsError) as ei:
        sv.poll(12345)
    assert ei.value.status == m.LABS_ENOTFOUND
    long_req = (301, 2048, 1208, 11, 2048 * 1208 * 151 * 4)
    t = sv.submit(*long_req)
    with pytest.raises(m.LabsError) as ei:
        sv.wait(t, timeout_s=0.001)
    assert ei.value.status == m.LABS_ETIMEOUT
    assert sv.poll(t) is None  # still pending
    queued = [sv.submit(121, 2048, 488, 20 + i, 10 ** 10) for i in range(4)]
    # concurrent pollers from other threads while the server runs
    seen = []

    def poller():
        for _ in range(20):
            try:
                seen.append(sv.poll(queued[-1]))
            except m.LabsError:
                pass
            time.sleep(0.005)

    th = threading.Thread(target=poller)
    th.start()
    th.join()
    t0 = time.time()
    sv.close()  # shutdown with work in flight and queued: must not hang
    assert time.time() - t0 < 120


def test_full_size_requests_vs_oracle(m):
    # requests of the serving stream's shape (2048 walks of 8*D steps) in a
    # server configured like the bench's, mixed with other full-size
    # requests; the two the oracle solves fastest (one round at L=121 and
    # L=123, one of them with a target it reaches in that round) are compared
    # with the oracle's Algorithm 1 + Algorithm 2 directly
    import os
    import oracle
    from paper_2210_15962_gb300 import workloads
    cores = os.cpu_count() or 8
    wl121, wl123 = workloads.paper_walk_len(121), workloads.paper_walk_len(123)
    o121 = oracle.solve(121, [5001], 2048, wl121, 2048 * wl121 * 61, threads=cores)
    o123 = oracle.solve(123, [5002], 2048, wl123, 2048 * wl123 * 62, threads=cores)
    checked = [
        ((121, 2048, wl121, 5001, 10 ** 10, int(o121["best_E"][0])), o121),   # target reached in round 1
        ((123, 2048, wl123, 5002, 2048 * wl123 * 62), o123),                   # budget of one round
    ]
    others = [(L, 2048, workloads.paper_walk_len(L), 5100 + L, 2 * 2048 * workloads.paper_walk_len(L) * ((L + 1) // 2))
              for L in (161, 223, 301)]
    with m.Server(max_L=301, max_walks=2048, max_active=64, mem_bytes=16 << 30, rounds_per_launch=4) as sv:
        tickets = [sv.submit(*p) for p, _ in checked] + [sv.submit(*p) for p in others]
        results = [sv.wait(t, timeout_s=600) for t in tickets]
    for (p, o), r in zip(checked, results):
        assert r["status"] == m.LABS_OK
        assert r["best_E"] == int(o["best_E"][0]) and np.array_equal(r["best_seq"], o["best_seq"][0]), p
        assert r["evals"] == int(o["evals"][0]) and r["rounds"] == int(o["rounds"][0]) == 1, p
    for p, r in zip(others, results[len(checked):]):
        check(m, p, r)


def test_probability_target_sets_the_budget(m):
    # the stopping rule of the predictive model: run until Eq. 7 reaches P
    import oracle
    with m.Server(max_walks=256) as sv:
        reqs = [(27, 64, 216, 31, 0.99), (71, 128, 288, 32, 0.5)]
        tickets = [sv.submit(L, w, wl, seed, p_target=P) for L, w, wl, seed, P in reqs]
        for (L, w, wl, seed, P), t in zip(reqs, tickets):
            r = sv.wait(t)
            budget = m.labs_model_budget(L, P)
            # the budget is the model's evaluation count rounded up to a whole evaluation
            assert budget == pytest.approx(oracle.model_nses_limit(L, P, 1) * ((L + 1) // 2) / ((L - 1) // 2),
                                           rel=1e-9, abs=1.0)
            assert r["evals"] >= budget and r["p_optimal"] >= P
            check(m, (L, w, wl, seed, budget), r)


@pytest.mark.parametrize("walk_mode", [0, 1, 2])
def test_served_results_match_oracle_every_class(m, walk_mode):
    # a mixed submission across the lag-word classes W = 1..5 (L = 61, 121, 161,
    # 223, 301), with budgets over several rounds and one target request; every
    # result is compared with the oracle's Algorithm 1 + Algorithm 2 directly,
    # for launches in the mode chosen per launch (0), one walk per lane (1) and
    # one walk per warp (2)
    import oracle
    reqs = [
        (61, 40, 160, 301, 40 * 160 * 31 * 3),
        (121, 50, 150, 302, 50 * 150 * 61 * 2),
        (161, 33, 120, 303, 33 * 120 * 81 * 3),
        (223, 40, 110, 304, 40 * 110 * 112 * 2),
        (301, 32, 100, 305, 32 * 100 * 151 * 2),
    ]
    o = oracle.solve(161, [306], 32, 120, 32 * 120 * 81 * 2, threads=8)
    reqs.append((161, 32, 120, 306, 10 ** 12, int(o["best_E"][0])))  # stops within two rounds
    with m.Server(max_walks=64, rounds_per_launch=2, walk_mode=walk_mode) as sv:
        tickets = [sv.submit(*p) for p in reqs]
        results = [sv.wait(t) for t in tickets]
    for p, r in zip(reqs, results):
        L, walks, wl, seed, budget = p[:5]
        tgt = p[5] if len(p) > 5 else -1
        w = oracle.solve(L, [seed], walks, wl, budget, target_E=tgt, threads=8)
        assert r["status"] == m.LABS_OK
        assert r["best_E"] == int(w["best_E"][0]), (p, r["best_E"], int(w["best_E"][0]))
        assert np.array_equal(r["best_seq"], w["best_seq"][0]), p
        assert r["evals"] == int(w["evals"][0]) and r["rounds"] == int(w["rounds"][0]), p
        if tgt >= 0:
            assert r["reached_target"] == 1 and r["rounds"] <= 2


def test_rounds_after_a_stop_are_never_counted(m):
    # every request reaches its target in its first round while up to 8 (and,
    # on an idle device, more) of its rounds run at once: the rounds issued
    # past the stop must add neither evaluations nor rounds (Algorithm 1 stops
    # at the first round whose best reaches the target), however their chunks
    # finish around the stopping round's finalization
    import oracle
    reqs = []
    for i in range(48):
        L = (61, 121)[i % 2]
        walks, wl, seed = 64, 120, 700 + i
        D = (L + 1) // 2
        o = oracle.solve(L, [seed], walks, wl, walks * wl * D, threads=8)
        reqs.append((L, walks, wl, seed, 10 ** 12, int(o["best_E"][0]), o))
    with m.Server(max_walks=64, rounds_per_launch=8) as sv:
        tickets = [sv.submit(*p[:6]) for p in reqs]
        results = [sv.wait(t) for t in tickets]
    for p, r in zip(reqs, results):
        L, walks, wl, seed, _, tgt, o = p
        assert r["status"] == m.LABS_OK
        assert r["rounds"] == 1 and r["evals"] == walks * wl * ((L + 1) // 2), (p[:6], r["rounds"], r["evals"])
        assert r["best_E"] == tgt and r["reached_target"] == 1
        assert np.array_equal(r["best_seq"], o["best_seq"][0]), p[:6]
