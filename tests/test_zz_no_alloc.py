"""labs_saw_round_noalloc: the round variant for callers that cannot allocate
device memory (its scratch is the library's fixed static device array).

Each call goes through the C ABI and must give exactly what the allocating
entry point labs_saw_round gives for the same round (integer search: exact),
for calls made one after another that reuse the same scratch.  This file is
collected last so a stop-at-first-failure run has already run the rest.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_2210_15962_gb300 import build
    build.build()
    import paper_2210_15962_gb300 as mod
    mod.load()
    return mod


def run_noalloc(m, L, seed, rnd, n, wl):
    import torch
    E = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    S = torch.zeros((n, L), dtype=torch.int8, device="cuda")
    mv = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    sk = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    m.labs_saw_round_noalloc(L, seed, rnd, n, wl, E, S, mv, sk, stream=torch.cuda.current_stream())
    return E.cpu().numpy(), S.cpu().numpy(), mv.cpu().numpy(), sk.cpu().numpy()


def test_noalloc_round_matches_allocating_round_on_consecutive_calls(m):
    # lag-word classes 1, 2 and 7 (L = 27, 121, 449); the third and last calls
    # reuse a scratch that an earlier, different round left filled
    cases = [(27, 1, 0, 64, 4096), (121, 7, 3, 100, 1500), (449, 5, 2, 40, 600), (27, 1, 0, 64, 4096)]
    for L, seed, rnd, n, wl in cases:
        E, S, mv, sk = run_noalloc(m, L, seed, rnd, n, wl)
        ref = m.labs_saw_round(L, seed, rnd, n, wl)
        assert np.array_equal(E, ref["best_E"]), (L, seed)
        assert np.array_equal(S, ref["best_seq"]), (L, seed)
        assert np.array_equal(mv, ref["moves"]) and np.array_equal(sk, ref["stuck"]), (L, seed)


def test_noalloc_rejects_rounds_larger_than_its_scratch(m):
    import torch
    n, L, wl = 1000, 121, 8192  # ~128 MiB of visited tables > the fixed scratch
    E = torch.zeros(n, dtype=torch.int64, device="cuda")
    S = torch.zeros((n, L), dtype=torch.int8, device="cuda")
    with pytest.raises(m.LabsError) as ei:
        m.labs_saw_round_noalloc(L, 1, 0, n, wl, E, S)
    assert ei.value.status == m.LABS_ENOMEM
    # a rejected call leaves the entry point usable
    E2, S2, _, _ = run_noalloc(m, 27, 2, 0, 8, 300)
    ref = m.labs_saw_round(27, 2, 0, 8, 300)
    assert np.array_equal(E2, ref["best_E"]) and np.array_equal(S2, ref["best_seq"])


def test_noalloc_binding_rejects_bad_buffers(m):
    # the binding refuses buffers the library would write out of bounds
    import torch
    n, L = 8, 27
    good_E = torch.zeros(n, dtype=torch.int64, device="cuda")
    good_S = torch.zeros((n, L), dtype=torch.int8, device="cuda")
    bad = [
        (torch.zeros(n, dtype=torch.int32, device="cuda"), good_S),   # wrong dtype
        (torch.zeros(n - 1, dtype=torch.int64, device="cuda"), good_S),  # too short
        (torch.zeros(n, dtype=torch.int64), good_S),                   # host tensor
        (good_E, torch.zeros((L, n), dtype=torch.int8, device="cuda").t()),  # not contiguous
        (good_E, None),
    ]
    for E, S in bad:
        with pytest.raises(m.LabsError) as ei:
            m.labs_saw_round_noalloc(L, 1, 0, n, 100, E, S)
        assert ei.value.status == m.LABS_EINVAL
    E, S, mv, sk = run_noalloc(m, L, 3, 0, n, 100)
    ref = m.labs_saw_round(L, 3, 0, n, 100)
    assert np.array_equal(E, ref["best_E"]) and np.array_equal(S, ref["best_seq"])
