"""Plain CPU oracle for the skew-symmetric LABS self-avoiding-walk solver.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
(``paper_2210_15962_gb300``) never does and has no CPU fallback.

The arithmetic lives in ``labs_oracle.cpp`` (C++17, ``std::set`` visited set);
this module only loads it with ctypes and marshals arguments.  Every function
cites the passage of the paper (Bošković, Herzog, Brest, arXiv 2210.15962) it
restates:

* ``energy``, ``autocorrelations`` -- Eq. 1;
* ``skew_expand`` -- Eq. 2;
* ``philox4x32_10``, ``start_free_values`` -- the random first pivot of Eq. 3
  (``rand{-1,+1}``), drawn from Philox4x32-10 (Salmon et al., SC'11);
* ``walk_trace``, ``walk_batch`` -- one contiguous self-avoiding walk, Eq. 3
  and Algorithm 2 (with ``full=True`` over all length-L sequences, the search
  space the paper leaves to future work in Section 5: L flips of one position
  each, the whole sequence as key);
* ``solve`` -- the round loop of Algorithm 1 with a neighbour-evaluation budget;
* ``model_lambda``, ``model_nses_limit``, ``model_p_optimal``,
  ``model_nses_of_evals`` -- the predictive model of Section 4.1 (the fitted
  trend of the exponential rate lambda(L), Eq. 6 and Eq. 7), plain Python in
  double precision.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from .build import LIB_PATH, build

_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            build()
        lib = ctypes.CDLL(LIB_PATH)
        i8p = ctypes.POINTER(ctypes.c_int8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_energy.restype = ctypes.c_int64
        lib.oracle_energy.argtypes = [i8p, ctypes.c_int32]
        lib.oracle_autocorrelations.restype = ctypes.c_int32
        lib.oracle_autocorrelations.argtypes = [i8p, ctypes.c_int32, i64p]
        lib.oracle_skew_expand.restype = ctypes.c_int32
        lib.oracle_skew_expand.argtypes = [i8p, ctypes.c_int32, i8p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.oracle_start_free_values.restype = None
        lib.oracle_start_free_values.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                                 ctypes.c_int32, i8p]
        lib.oracle_walk_trace.restype = ctypes.c_int32
        lib.oracle_walk_trace.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int32, ctypes.c_int32, i32p, i64p, i8p, i64p, i32p, i32p,
                                          i32p]
        lib.oracle_walk_batch.restype = ctypes.c_int32
        lib.oracle_walk_batch.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, i64p, i8p, i32p,
                                          i32p, i64p]
        lib.oracle_solve.restype = ctypes.c_int32
        lib.oracle_solve.argtypes = [ctypes.c_int32, u64p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, i64p, i8p, u64p, i32p]
        for space_fn, twin in [("oracle_full_walk_trace", lib.oracle_walk_trace),
                               ("oracle_full_walk_batch", lib.oracle_walk_batch),
                               ("oracle_full_solve", lib.oracle_solve)]:
            fn = getattr(lib, space_fn)
            fn.restype, fn.argtypes = twin.restype, twin.argtypes
        _lib = lib
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def energy(seq) -> int:
    """Eq. 1: E = sum_{k=1}^{L-1} C_k^2 of a +-1 sequence."""
    s = np.ascontiguousarray(seq, dtype=np.int8)
    e = _load().oracle_energy(_p(s, ctypes.c_int8), s.size)
    if e < 0:
        raise ValueError("sequence must be non-empty and contain only +1/-1")
    return int(e)


def autocorrelations(seq) -> np.ndarray:
    """Eq. 1: C_k for k = 0..L-1 (C_0 = L)."""
    s = np.ascontiguousarray(seq, dtype=np.int8)
    out = np.zeros(s.size, dtype=np.int64)
    if _load().oracle_autocorrelations(_p(s, ctypes.c_int8), s.size, _p(out, ctypes.c_int64)) != 0:
        raise ValueError("bad sequence")
    return out


def skew_expand(free_vals, L: int) -> np.ndarray:
    """Eq. 2: the length-L skew-symmetric sequence with the given D=(L+1)/2 free values."""
    f = np.ascontiguousarray(free_vals, dtype=np.int8)
    out = np.zeros(L, dtype=np.int8)
    if f.size < (L + 1) // 2 or _load().oracle_skew_expand(_p(f, ctypes.c_int8), L, _p(out, ctypes.c_int8)) != 0:
        raise ValueError("L must be odd and >= 3 with (L+1)/2 free values")
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def start_free_values(seed: int, walk: int, round_: int, D: int) -> np.ndarray:
    """Random first pivot P_1 (Eq. 3) of walk `walk` in round `round_` as D +-1 values."""
    out = np.zeros(D, dtype=np.int8)
    _load().oracle_start_free_values(seed, walk, round_, D, _p(out, ctypes.c_int8))
    return out


def walk_trace(L: int, seed: int, walk: int, round_: int, walk_len: int, check: bool = False,
               full: bool = False) -> dict:
    """One contiguous SAW (Eq. 3, Algorithm 2) with its full trajectory; `full`
    walks the whole space of length-L sequences instead of the skew-symmetric one."""
    flips = np.full(max(walk_len, 1), -1, dtype=np.int32)
    energies = np.full(walk_len + 1, -1, dtype=np.int64)
    best_seq = np.zeros(L, dtype=np.int8)
    best_E = np.zeros(1, dtype=np.int64)
    moves = np.zeros(1, dtype=np.int32)
    stuck = np.zeros(1, dtype=np.int32)
    best_step = np.zeros(1, dtype=np.int32)
    fn = _load().oracle_full_walk_trace if full else _load().oracle_walk_trace
    rc = fn(L, seed, walk, round_, walk_len, int(check), _p(flips, ctypes.c_int32),
            _p(energies, ctypes.c_int64), _p(best_seq, ctypes.c_int8), _p(best_E, ctypes.c_int64),
            _p(moves, ctypes.c_int32), _p(stuck, ctypes.c_int32), _p(best_step, ctypes.c_int32))
    if rc < 0:
        raise ValueError("bad arguments")
    m = int(moves[0])
    return {
        "check_failed": rc == 1,
        "flips": flips[:m].copy(),
        "energies": energies[:m + 1].copy(),
        "best_seq": best_seq,
        "best_E": int(best_E[0]),
        "moves": m,
        "stuck": int(stuck[0]),
        "best_step": int(best_step[0]),
    }


def walk_batch(L: int, seed: int, round_: int, walk_begin: int, n_walks: int, walk_len: int,
               threads: int = 1, full: bool = False) -> dict:
    """Walks [walk_begin, walk_begin + n_walks) of one round, per-walk results."""
    best_E = np.zeros(n_walks, dtype=np.int64)
    best_seq = np.zeros((n_walks, L), dtype=np.int8)
    moves = np.zeros(n_walks, dtype=np.int32)
    stuck = np.zeros(n_walks, dtype=np.int32)
    evals = np.zeros(n_walks, dtype=np.int64)
    fn = _load().oracle_full_walk_batch if full else _load().oracle_walk_batch
    rc = fn(L, seed, round_, walk_begin, n_walks, walk_len, threads, _p(best_E, ctypes.c_int64),
            _p(best_seq, ctypes.c_int8), _p(moves, ctypes.c_int32), _p(stuck, ctypes.c_int32),
            _p(evals, ctypes.c_int64))
    if rc != 0:
        raise ValueError("bad arguments")
    return {"best_E": best_E, "best_seq": best_seq, "moves": moves, "stuck": stuck, "evals": evals}


def solve(L: int, seeds, walks: int, walk_len: int, step_budget: int, target_E: int = -1,
          threads: int = 1, full: bool = False) -> dict:
    """Algorithm 1: rounds of `walks` SAWs per seed until the evaluation budget (or target) is met."""
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    n = sd.size
    best_E = np.zeros(n, dtype=np.int64)
    best_seq = np.zeros((n, L), dtype=np.int8)
    evals = np.zeros(n, dtype=np.uint64)
    rounds = np.zeros(n, dtype=np.int32)
    fn = _load().oracle_full_solve if full else _load().oracle_solve
    rc = fn(L, _p(sd, ctypes.c_uint64), n, walks, walk_len, step_budget, target_E, threads,
            _p(best_E, ctypes.c_int64), _p(best_seq, ctypes.c_int8), _p(evals, ctypes.c_uint64),
            _p(rounds, ctypes.c_int32))
    if rc != 0:
        raise ValueError("bad arguments")
    return {"best_E": best_E, "best_seq": best_seq, "evals": evals, "rounds": rounds}


# ---------------------------------------------------------------- Section 4.1
def model_lambda(L: int) -> float:
    """Rate of the exponential distribution of the solution evaluations one run
    needs to reach an optimal skew-symmetric sequence: the authors' trend fitted
    on L = 71..119, lambda(L) = 0.006753 * 0.8617^L (Section 4.1; used beyond
    that range, as the paper does, as an extrapolation)."""
    return 0.006753 * 0.8617 ** L


def model_nses_limit(L: int, P: float, N: int) -> float:
    """Eq. 6: evaluations per run so that N independent runs reach an optimum
    with probability P, ln(1 - P) / (-lambda(L) N)."""
    return math.log(1.0 - P) / (-model_lambda(L) * N)


def model_p_optimal(L: int, nses: float) -> float:
    """Eq. 7: probability that an optimum was reached after nses evaluations in
    total (the runs taken together as one), 1 - exp(-lambda(L) nses)."""
    return 1.0 - math.exp(-model_lambda(L) * nses)


def model_nses_of_evals(L: int, evals: int) -> float:
    """The paper's evaluation count from this project's: the paper adds D - 1
    per walk step (the previous pivot is never re-evaluated), this project
    counts all D flips of a step."""
    D = (L + 1) // 2
    return evals * (D - 1) / D
