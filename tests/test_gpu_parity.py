"""GPU path vs the CPU oracle, bit-exact (integer search: no tolerance).

Every call goes through the C ABI of liblabs_gb300.so.  Compared per walk:
the whole trajectory (flip chosen at every step), the visited set, moves,
stuck flag, best energy, best sequence and the step where it was reached;
per problem: best energy, best sequence, evaluations and rounds.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def table1():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "table1_skew_sequences.txt")):
        if line.strip() and not line.startswith("#"):
            r = line.split()
            rows.append((int(r[0]), int(r[1]), r[4]))
    return rows


# ------------------------------------------------------------------ Eq. 1
def test_energy_table1(m):
    for L, E, hx in table1():
        assert m.labs_energy(m.from_hex(hx, L)) == E


@pytest.mark.parametrize("L", [1, 2, 3, 5, 31, 32, 33, 64, 65, 121, 449, 511, 1000, 4097])
def test_energy_random_vs_oracle(m, orc, L):
    rng = np.random.default_rng(L)
    for _ in range(3):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=L)
        assert m.labs_energy(s) == orc.energy(s)


def test_energy_batch_and_bad_values(m, orc):
    import torch
    rng = np.random.default_rng(7)
    seqs = rng.choice(np.array([-1, 1], dtype=np.int8), size=(37, 301))
    out = m.labs_energy_batch(torch.from_numpy(seqs).cuda()).cpu().numpy()
    assert [int(x) for x in out] == [orc.energy(s) for s in seqs]
    bad = seqs.copy()
    bad[3, 5] = 0
    with pytest.raises(m.LabsError):
        m.labs_energy_batch(torch.from_numpy(bad).cuda())
    with pytest.raises(m.LabsError):
        m.labs_energy(np.array([1, 2, 1], dtype=np.int8))


# ------------------------------------------------------- one round, per walk
# full scan (lane per walk), incremental, full scan (warp per walk), full scan (CTA per walk): all give the
# oracle's results
KERNELS = [1, 2, 3, 4]


def compare_round(m, orc, L, seed, rnd, n_walks, walk_len, check_walks, trace_walks=(), recheck=0, kernel=1):
    """GPU round of n_walks walks; oracle on the sampled walk indices."""
    tb, tc = (min(trace_walks), max(trace_walks) - min(trace_walks) + 1) if trace_walks else (0, 0)
    g = m.labs_saw_round(L, seed, rnd, n_walks, walk_len, recheck_every=recheck, trace_begin=tb, trace_count=tc,
                         kernel=kernel)
    D = (L + 1) // 2
    for w in check_walks:
        o = orc.walk_trace(L, seed, w, rnd, walk_len)
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


@pytest.mark.parametrize("kernel", KERNELS)
def test_config1_L27_all_walks_and_trajectories(m, orc, kernel):
    # L=27 (D=14), seed 1, 64 walks of 4096 steps: every walk, every step
    L, wl = 27, 4096
    compare_round(m, orc, L, 1, 0, 64, wl, range(64), trace_walks=range(64), kernel=kernel)


def test_config1_solve_matches_oracle(m, orc):
    L, walks, wl = 27, 64, 4096
    budget = walks * wl * 14
    g = m.labs_walks(L, [1], walks, wl, budget)
    o = orc.solve(L, [1], walks, wl, budget, threads=8)
    assert int(g["best_E"][0]) == int(o["best_E"][0]) == 37  # the skew optimum for L=27 (F=9.85)
    assert np.array_equal(g["best_seq"][0], o["best_seq"][0])
    assert int(g["evals"][0]) == int(o["evals"][0]) and int(g["rounds"][0]) == int(o["rounds"][0]) == 1


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("L", [5, 7, 9, 11, 13])
def test_tiny_L_stuck_walks(m, orc, L, kernel):
    # tiny spaces: walks run out of unvisited neighbours (the "stuck" reading)
    wl = 2 ** ((L + 1) // 2) + 3
    g = compare_round(m, orc, L, 3, 1, 40, wl, range(40), trace_walks=range(40), kernel=kernel)
    assert g["stuck"].sum() == 40


@pytest.mark.parametrize("L", [15, 31, 33, 61, 63, 65, 67, 121, 127, 129, 131, 191, 193, 223, 255, 257, 259,
                               301, 383, 385, 449, 511])
@pytest.mark.parametrize("kernel", KERNELS)
def test_lag_word_classes_and_ragged_tails(m, orc, L, kernel):
    # every lag-word class (m = 32W and m = 32W + 1 edges), with an every-step full recheck
    wl = 600 if L < 200 else 250
    n = 70  # more than two warps, last one ragged
    compare_round(m, orc, L, 11 + L, 2, n, wl, [0, 1, 31, 32, 33, 69], trace_walks=[0, 1, 31, 32, 33],
                  recheck=1, kernel=kernel)


@pytest.mark.parametrize("kernel", KERNELS)
def test_visited_set_is_exactly_the_pivots(m, orc, kernel):
    for L, wl, w in [(27, 3000, 5), (121, 700, 3), (449, 200, 1)]:
        D = (L + 1) // 2
        g = m.labs_saw_round(L, 9, 0, 8, wl, visited_walk=w, kernel=kernel)
        o = orc.walk_trace(L, 9, w, 0, wl)
        free = orc.start_free_values(9, w, 0, D).copy()
        want = set()

        def key(f):
            v = 0
            for j, x in enumerate(f):
                if x < 0:
                    v |= 1 << j
            return v

        want.add(key(free))
        for j in o["flips"]:
            free[j] = -free[j]
            want.add(key(free))
        got = set()
        for row in g["visited"]:
            v = 0
            for i, wd in enumerate(row):
                v |= int(wd) << (64 * i)
            got.add(v)
        assert g["visited_count"] == len(want) == o["moves"] + 1
        assert got == want


def test_solve_multi_seed_multi_round_and_target(m, orc):
    L, walks, wl = 41, 50, 300
    D = (L + 1) // 2
    per_round = walks * wl * D
    seeds = [3, 4, 5]
    g = m.labs_walks(L, seeds, walks, wl, 2 * per_round + 1)
    o = orc.solve(L, seeds, walks, wl, 2 * per_round + 1, threads=8)
    assert np.array_equal(g["best_E"], o["best_E"])
    assert np.array_equal(g["best_seq"], o["best_seq"])
    assert np.array_equal(g["evals"].astype(np.int64), o["evals"].astype(np.int64))
    assert list(g["rounds"]) == list(o["rounds"]) == [3, 3, 3]
    # target energy: stop at the first round whose best reaches it
    tgt = int(o["best_E"].max()) + 4
    g2 = m.labs_walks(L, seeds, walks, wl, 10 ** 12, target_E=tgt)
    o2 = orc.solve(L, seeds, walks, wl, 10 ** 12, target_E=tgt, threads=8)
    assert np.array_equal(g2["best_E"], o2["best_E"]) and list(g2["rounds"]) == list(o2["rounds"])
    assert np.array_equal(g2["best_seq"], o2["best_seq"])
    # max_rounds caps every problem
    g3 = m.labs_walks(L, seeds, walks, wl, 10 ** 12, max_rounds=2)
    assert list(g3["rounds"]) == [2, 2, 2]


def test_device_buffer_binding_rejects_bad_buffers(m):
    # the binding refuses device buffers the library would write out of bounds
    import torch
    n, L = 2, 61
    sd = torch.tensor([1, 2], dtype=torch.int64, device="cuda")
    bs = torch.zeros((n, L), dtype=torch.int8, device="cuda")
    be = torch.zeros(n, dtype=torch.int64, device="cuda")
    bad = [
        (sd, bs, torch.zeros(n, dtype=torch.int32, device="cuda")),        # wrong dtype
        (sd, torch.zeros((n, L - 1), dtype=torch.int8, device="cuda"), be),  # too short
        (sd, bs, torch.zeros(n, dtype=torch.int64)),                        # host tensor
        (sd, torch.zeros((L, n), dtype=torch.int8, device="cuda").t(), be),  # not contiguous
        (sd.to(torch.int32), bs, be),                                       # seeds of the wrong width
    ]
    for s_, q_, e_ in bad:
        with pytest.raises(m.LabsError) as ei:
            m.labs_walks_device(L, s_, 32, 50, 10 ** 6, q_, e_)
        assert ei.value.status == m.LABS_EINVAL
    with pytest.raises(m.LabsError):
        m.labs_walks_device(L, sd, 32, 50, 10 ** 6, bs, be, workspace=torch.zeros(1024, dtype=torch.uint8))
    m.labs_walks_device(L, sd, 32, 50, 10 ** 6, bs, be)
    torch.cuda.synchronize()
    ref = m.labs_walks(L, [1, 2], 32, 50, 10 ** 6)
    assert np.array_equal(be.cpu().numpy(), ref["best_E"]) and np.array_equal(bs.cpu().numpy(), ref["best_seq"])


def test_round_boundaries_and_ties_match_oracle(m, orc):
    # a budget of exactly one round's evaluations, a target equal to the first
    # round's best, and several walks tied at the best energy with different
    # sequences (the first wins): the round loop's readings, as in the oracle
    for L, walks, wl, seed in [(19, 16, 8, 4), (121, 64, 100, 6)]:
        b0 = orc.walk_batch(L, seed, 0, 0, walks, wl, threads=8)
        per_round = int(b0["evals"].sum())
        best0 = int(b0["best_E"].min())
        for budget, target in [(per_round, -1), (3 * per_round, best0), (per_round + 1, -1)]:
            g = m.labs_walks(L, [seed], walks, wl, budget, target_E=target)
            o = orc.solve(L, [seed], walks, wl, budget, target_E=target, threads=8)
            assert list(g["rounds"]) == list(o["rounds"]), (L, budget, target)
            assert np.array_equal(g["evals"].astype(np.int64), o["evals"].astype(np.int64))
            assert np.array_equal(g["best_E"], o["best_E"]) and np.array_equal(g["best_seq"], o["best_seq"])
        if L == 19:
            assert list(m.labs_walks(L, [seed], walks, wl, per_round)["rounds"]) == [1]
            tied = [w for w in range(walks) if int(b0["best_E"][w]) == best0]
            assert len(tied) >= 2 and any(not np.array_equal(b0["best_seq"][tied[0]], b0["best_seq"][w])
                                          for w in tied[1:])
            g = m.labs_walks(L, [seed], walks, wl, per_round)
            assert np.array_equal(g["best_seq"][0], b0["best_seq"][tied[0]])


def test_chunked_workspace_and_device_buffers_match(m):
    import torch
    L, walks, wl = 61, 200, 400
    seeds = [21, 22]
    budget = walks * wl * 31 * 2
    ref = m.labs_walks(L, seeds, walks, wl, budget)
    full = m.labs_walks_workspace_size(L, len(seeds), walks, wl)
    small = torch.empty(full // 5, dtype=torch.uint8, device="cuda")  # forces several launches per round
    g = m.labs_walks(L, seeds, walks, wl, budget, workspace=small)
    assert g["stats"]["walk_launches"] > ref["stats"]["walk_launches"]
    assert np.array_equal(g["best_E"], ref["best_E"]) and np.array_equal(g["best_seq"], ref["best_seq"])
    sd = torch.tensor(seeds, dtype=torch.int64, device="cuda")
    bs = torch.zeros((2, L), dtype=torch.int8, device="cuda")
    be = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = m.labs_walks_device(L, sd, walks, wl, budget, bs, be, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(be.cpu().numpy(), ref["best_E"]) and np.array_equal(bs.cpu().numpy(), ref["best_seq"])
    assert st["evals"] == int(ref["evals"].sum())


@pytest.mark.parametrize("kernel", KERNELS)
def test_config2_L121_full_size_sampled(m, orc, kernel):
    # L=121 (D=61), 131072 walks of 8192 steps: the bench's launch shape; oracle on sampled walks
    L, n, wl = 121, 131072, 8192
    compare_round(m, orc, L, 1, 0, n, wl, [0, 1, 4095, 65536, 131071], trace_walks=[0, 1], kernel=kernel)


@pytest.mark.parametrize("L", [27, 121, 223])
def test_variants_agree_on_whole_solves(m, L):
    D = (L + 1) // 2
    wl = 8 * D
    # every variant, and the library's timed choice (kernel 0), solve alike
    res = [m.labs_walks(L, [3, 4], 256, wl, 256 * wl * D * 2, kernel=k) for k in (1, 2, 3, 4, 0)]
    for r in res[1:]:
        for key in ("best_E", "best_seq", "evals", "rounds"):
            assert np.array_equal(res[0][key], r[key]), key


def test_config5_L449_sampled(m, orc):
    # L=449 (D=225), walk length 16384: a smaller batch, sampled walks, full walk length
    L, n, wl = 449, 2048, 16384
    compare_round(m, orc, L, 1, 0, n, wl, [0, 2047], trace_walks=[0])


def test_recheck_mode_runs_clean(m):
    g = m.labs_walks(121, [5], 64, 500, 64 * 500 * 61, recheck_every=1)
    assert g["best_E"][0] > 0
