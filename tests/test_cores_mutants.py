"""Planted mistakes in the CUDA path's walk cores must fail the host-core check.

`walk_core.cuh`, `full_core.cuh` and `walk_incr.cuh` hold the kernels'
arithmetic as host+device functions, and test_cores_on_host.py walks with them
on the host against the oracle.  Each mutant below is one plausible slip in
that arithmetic -- the Philox rounds, the start's word choice, Eq. 2's sign,
the correlation count, the digit offset, the plane-count choice, the top-4
list, the key's constant part or its step, the doubled-lag coefficient, the
top plane's index, the move's carry or pair lag, the sign fold, the full
space's even-lag correction or key step, the incremental variant's delta
update or correlation update -- planted in a temporary copy of the three
headers, never in the sources themselves.  The host-core program is built
against the copy (unoptimised, to keep the build short) and its walks are
compared with the oracle's: every mutant must change a trajectory, an energy,
a best E or a stuck flag, or fail the full recheck of the digit planes, and
the unmodified copy must match everywhere.  This runs without a GPU.

Not every slip changes a walk: a top-4 list that keeps only copies of its
smallest key gives the same walks, since a step whose listed candidates are
all visited rescans above the list's last key, so the list only saves time;
such equivalent changes are not in the list below.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2210_15962_gb300", "csrc")
SRC = os.path.join(HERE, "host_core", "walk_cores_on_host.cpp")
CORE_HEADERS = ("walk_core.cuh", "full_core.cuh", "walk_incr.cuh")

sys.path.insert(0, HERE)
import test_cores_on_host as hc  # noqa: E402  (the case format and comparison of the host-core check)

# (name, header, original text -- must occur exactly once --, planted text)
MUTANTS = [
    ("philox_nine_rounds", "walk_core.cuh",
     "for (int r = 0; r < 10; ++r) {\n    const uint32_t lo0", "for (int r = 0; r < 9; ++r) {\n    const uint32_t lo0"),
    ("start_word_choice", "walk_core.cuh",
     "st.key[w] = blk[w & 3] & low_mask_word(g.D, w);", "st.key[w] = blk[w & 1] & low_mask_word(g.D, w);"),
    ("eq2_sign", "walk_core.cuh",
     "b = get_bit(st.key, g.c - i) ^ (uint32_t)(i & 1);", "b = get_bit(st.key, g.c - i) ^ (uint32_t)((i + 1) & 1);"),
    ("correlation_disagreements_once", "walk_core.cuh",
     "      C += pairs - 2 * dis;\n    }\n  }\n  return C;", "      C += pairs - dis;\n    }\n  }\n  return C;"),
    ("digit_offset", "walk_core.cuh",
     "const uint32_t e = (uint32_t)((C + (1 << T) - 1) >> 1);\n#pragma unroll\n    for (int t = 0; t < T; ++t) xor_bit(st.ep[t], i - 1, (e >> t) & 1u);\n  }\n  st.E = E;",
     "const uint32_t e = (uint32_t)((C + (1 << T) + 1) >> 1);\n#pragma unroll\n    for (int t = 0; t < T; ++t) xor_bit(st.ep[t], i - 1, (e >> t) & 1u);\n  }\n  st.E = E;"),
    ("plane_count_one_short", "walk_core.cuh",
     "    if (!all) break;\n    tp = u + 1;", "    if (!all) break;\n    tp = u;"),
    ("top_list_keeps_largest", "walk_core.cuh",
     "    const uint32_t lo = top[r] < x ? top[r] : x;", "    const uint32_t lo = top[r] < x ? x : top[r];"),
    ("key_constant_count", "walk_core.cuh",
     "(16u + 8u * K1) * (uint32_t)n - (32u + 16u * K1) * (uint32_t)nxy) +",
     "(16u + 8u * K1) * (uint32_t)(n + 1) - (32u + 16u * K1) * (uint32_t)nxy) +"),
    ("key_step", "walk_core.cuh",
     "kbase += 2u - 256u * (32u + 16u * K1);", "kbase += 2u - 256u * (32u + 8u * K1);"),
    ("doubled_lag_coefficient", "walk_core.cuh",
     "imad(mcnt, 4096u * (K1 + 4u), kbase)", "imad(mcnt, 4096u * (K1 + 2u), kbase)"),
    ("top_plane_index", "walk_core.cuh",
     "const uint32_t e1 = st.ep[tt < TP - 1 ? tt : T - 1][w];", "const uint32_t e1 = st.ep[tt][w];"),
    ("move_drops_carry", "walk_core.cuh",
     "const uint32_t d1 = xs ^ ys ^ c1;", "const uint32_t d1 = xs ^ ys;"),
    ("move_keeps_pair_lag", "walk_core.cuh",
     "low_mask_word(Nq - 1 - t, w);\n    if (!centre && ((i0 - 1) >> 5) == w) vy &= ~(1u << ((i0 - 1) & 31));",
     "low_mask_word(Nq - 1 - t, w);\n"),
    ("scan_mask_keeps_pair_lag", "walk_core.cuh",
     "low_mask_word(g.N[q] - 1 - t, w);\n      if (!centre && ((i0 - 1) >> 5) == w) vy &= ~(1u << ((i0 - 1) & 31));",
     "low_mask_word(g.N[q] - 1 - t, w);\n"),
    ("sign_not_folded", "walk_core.cuh",
     "const uint32_t bm = kFold ? 0u - ba : 0u;", "const uint32_t bm = 0u;"),
    ("full_even_lag_count", "full_core.cuh",
     "qev += 2 * (int)popc32(m2 & evm);", "qev += (int)popc32(m2 & evm);"),
    ("full_key_step_second_half", "full_core.cuh",
     "j < half ? 1u - 256u * (8u + 8u * K1) : 1u + 256u * (8u + 8u * K1);",
     "j < half ? 1u - 256u * (8u + 8u * K1) : 1u - 256u * (8u + 8u * K1);"),
    ("incr_delta_scale", "walk_incr.cuh",
     "int dnew = v.getD(a) + 32 * sa * sstar * (ncnt - 2 * (int)xcnt);",
     "int dnew = v.getD(a) + 16 * sa * sstar * (ncnt - 2 * (int)xcnt);"),
    ("incr_correlation_sign", "walk_incr.cuh",
     "if (u) vv.setC(i, v.getC(i) - 4 * u);", "if (u) vv.setC(i, v.getC(i) + 4 * u);"),
]


def cases():
    """The host-core check's walks: every lag-word class of both spaces, forced and free plane counts,
    pattern runs at three words and one class narrower and wider, long walks that rescan and get stuck,
    and the incremental variant."""
    out = []
    for L in hc.SKEW_L:
        W = ((L - 1) // 2 + 31) // 32
        for walk in range(2):
            for force_tp in (0, 1):
                for pmax in ((3, 4, 2) if 2 <= W <= 4 else (3,)):
                    out.append(("skew", L, 11, 2, walk, hc.walk_len_for(L), force_tp, pmax))
    out += [("skew", L, 5, 0, walk, wl, 0, 4) for L, wl in [(5, 40), (7, 80), (13, 4000)] for walk in range(2)]
    out += [("incr", L, 11, 2, walk, hc.walk_len_for(L)) for L in hc.SKEW_L for walk in range(2)]
    out += [("full", L, 7, 1, walk, hc.walk_len_for(L), force_tp)
            for L in hc.FULL_L for walk in range(2) for force_tp in (0, 1)]
    return out


def mismatches(got_all, want_all):
    """Number of walks whose result differs from the oracle's (or fails the recheck)."""
    bad = 0
    for got, want in zip(got_all, want_all):
        same = (got["recheck_ok"] and got["moves"] == want["moves"] and got["stuck"] == want["stuck"]
                and list(got["flips"]) == list(want["flips"]) and list(got["energies"]) == list(want["energies"])
                and got["best_E"] == want["best_E"])
        bad += not same
    return bad


def run_copy(mutant, case_list, cxx):
    """Build the host-core program against a copy of the core headers (with `mutant` planted) and run the walks."""
    tmp = tempfile.mkdtemp(prefix="cores_copy_")
    try:
        for h in CORE_HEADERS:
            shutil.copy(os.path.join(CSRC, h), tmp)
        if mutant is not None:
            name, header, old, new = mutant
            path = os.path.join(tmp, header)
            with open(path) as fh:
                src = fh.read()
            assert src.count(old) == 1, "mutant %s: its original text must occur exactly once" % name
            with open(path, "w") as fh:
                fh.write(src.replace(old, new))
        exe = os.path.join(tmp, "walk_cores_on_host")
        b = subprocess.run([cxx, "-O0", "-std=c++17", "-I", tmp, SRC, "-o", exe], capture_output=True, text=True,
                           timeout=600)
        if b.returncode != 0:
            return {"build_failed": b.stderr[-2000:]}
        try:
            return {"results": hc.run_cases(exe, case_list)}
        except (subprocess.CalledProcessError, ValueError, AssertionError) as e:
            return {"crashed": repr(e)[-2000:]}
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


@pytest.fixture(scope="module")
def outcomes(oracle_mod):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    case_list = cases()
    want = []
    for c in case_list:
        L, seed, rnd, walk, wl = c[1:6]
        want.append(oracle_mod.walk_trace(L, seed, walk, rnd, wl, full=(c[0] == "full")))
    jobs = [("unmodified", None)] + [(m[0], m) for m in MUTANTS]
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {name: ex.submit(run_copy, m, case_list, cxx) for name, m in jobs}
        res = {name: f.result() for name, f in futs.items()}
    return {name: (dict(r, bad=mismatches(r["results"], want)) if "results" in r else r) for name, r in res.items()}


def test_unmodified_cores_match_the_oracle(outcomes):
    got = outcomes["unmodified"]
    assert "results" in got, got
    assert got["bad"] == 0


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_changes_a_walk(outcomes, name):
    got = outcomes[name]
    assert "build_failed" not in got, got
    assert "crashed" not in got, got  # a wrong walk, not a crash, has to show it
    assert got["bad"] > 0, "the mistake %s leaves every walk unchanged" % name


def test_core_mutants_are_distinct_and_present():
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, header, old, new in MUTANTS:
        assert old != new
        with open(os.path.join(CSRC, header)) as fh:
            assert fh.read().count(old) == 1, name
