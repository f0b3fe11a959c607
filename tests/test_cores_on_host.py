"""The CUDA path's walk cores, compiled for the host, against the oracle.

`walk_core.cuh`, `full_core.cuh` and `walk_incr.cuh` hold the walk kernels'
arithmetic as host+device functions: the start (Philox draw, Eq. 2
expansion, Eq. 1 correlations into digit planes), the bit-sliced
neighbourhood scan of Algorithm 2 with its pattern runs, sign fold, stepped
key and plane-count choice, the move's bit-sliced update, the incremental
variant's stored correlations and deltas, and the visited table.
`host_core/walk_cores_on_host.cpp` compiles them with g++ and walks with them;
every walk's flips, energies, best E and stuck flag must equal the oracle's,
and the digit planes must pass the full recheck after every move.  This runs
without a GPU; the `-m gpu` tests check the kernels themselves."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2210_15962_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "host_core", "walk_cores_on_host.cpp")

# every lag-word class of the skew space (W = 1..8) with the lengths at its edges
SKEW_L = [5, 7, 9, 13, 27, 63, 65, 67, 121, 129, 131, 161, 193, 195, 223, 257, 259, 301, 321, 383, 385, 449, 511]
# every class of the full space (W = 1..8), both word edges of L-1
FULL_L = [3, 4, 5, 8, 12, 13, 20, 31, 32, 33, 34, 63, 64, 65, 100, 127, 128, 129, 160, 192, 193, 200, 224, 225,
          255, 256]


def walk_len_for(L):
    return 120 if L <= 64 else (60 if L <= 260 else 24)


@pytest.fixture(scope="module")
def cores(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("host_core") / "walk_cores_on_host")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, SRC, "-o", exe], check=True)
    return exe


def run_cases(exe, cases):
    text = "".join(" ".join(str(x) for x in c) + "\n" for c in cases)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
    assert len(out) == len(cases)
    res = []
    for line in out:
        head, flips, energies = line.split("|")
        moves, stuck, best_E, recheck_ok = (int(x) for x in head.split())
        res.append({"moves": moves, "stuck": stuck, "best_E": best_E, "recheck_ok": recheck_ok == 1,
                    "flips": np.array(flips.split(), dtype=np.int64),
                    "energies": np.array(energies.split(), dtype=np.int64)})
    return res


def compare(oracle_mod, case, got, full):
    L, seed, rnd, walk, wl = case[1:6]
    want = oracle_mod.walk_trace(L, seed, walk, rnd, wl, full=full)
    assert got["recheck_ok"], case
    assert got["moves"] == want["moves"] and got["stuck"] == want["stuck"], case
    assert np.array_equal(got["flips"], want["flips"]), case
    assert np.array_equal(got["energies"], want["energies"]), case
    assert got["best_E"] == want["best_E"], case


def test_skew_cores_match_the_oracle(cores, oracle_mod):
    cases = []
    for L in SKEW_L:
        W = ((L - 1) // 2 + 31) // 32
        for walk in range(2):
            for force_tp in (0, 1):
                # the kernels' pattern runs (pmax 3) and the same templates one class narrower and wider
                for pmax in ((3, 4, 2) if 2 <= W <= 4 else (3,)):
                    cases.append(("skew", L, 11, 2, walk, walk_len_for(L), force_tp, pmax))
    for case, got in zip(cases, run_cases(cores, cases)):
        compare(oracle_mod, case, got, full=False)


def test_skew_cores_long_walks_with_rescans(cores, oracle_mod):
    # long walks at small L revisit neighbourhoods: rescans above the 4th key and stuck walks
    cases = [("skew", L, 5, 0, walk, wl, 0, 4) for L, wl in [(5, 40), (7, 80), (9, 300), (13, 4000), (27, 4096)]
             for walk in range(3)]
    res = run_cases(cores, cases)
    for case, got in zip(cases, res):
        compare(oracle_mod, case, got, full=False)
    assert any(r["stuck"] for r in res)


def test_incremental_cores_match_the_oracle(cores, oracle_mod):
    # the incremental neighbourhood (stored C and Delta, updated by each move), every class, with the
    # kernel's storage widths; short walks at small L revisit and rescan
    cases = [("incr", L, 11, 2, walk, walk_len_for(L)) for L in SKEW_L for walk in range(2)]
    cases += [("incr", L, 5, 0, walk, wl) for L, wl in [(7, 80), (13, 4000)] for walk in range(2)]
    for case, got in zip(cases, run_cases(cores, cases)):
        compare(oracle_mod, case, got, full=False)


def test_full_cores_match_the_oracle(cores, oracle_mod):
    cases = []
    for L in FULL_L:
        for walk in range(2):
            for force_tp in (0, 1):
                cases.append(("full", L, 7, 1, walk, walk_len_for(L), force_tp))
    for case, got in zip(cases, run_cases(cores, cases)):
        compare(oracle_mod, case, got, full=True)
