"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

The paper's workloads are random +-1 starting pivots (Eq. 3, ``rand{-1,+1}``)
drawn inside the solver from a per-problem seed, so a workload here is just the
list of problems: sequence length L, seed, walks per round, walk length, the
neighbour-evaluation budget and, for serving, arrival times and energy targets.
All of it comes from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) seeded with a fixed constant, so
the oracle, the tests and the benchmark see identical problems.

Both the CUDA path's callers and the oracle's callers use this module; it holds
no energy, walk or selection code.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

MANIFEST_SEED = 20221028

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (64-bit state, Weyl increment + finaliser)."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by rejection."""
        n = hi - lo + 1
        limit = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next_u64()
            if x < limit:
                return lo + x % n


def odd_uniform(rng: SplitMix64, lo: int, hi: int) -> int:
    """Odd L uniform over the odd values of [lo, hi]."""
    first = lo if lo % 2 else lo + 1
    last = hi if hi % 2 else hi - 1
    return first + 2 * rng.randint(0, (last - first) // 2)


def paper_walk_len(L: int) -> int:
    """Walk length n = 8 * D used by the paper (Section 4.1), D = (L + 1) / 2."""
    return 8 * ((L + 1) // 2)


@dataclass
class Problem:
    L: int
    seed: int
    walks: int
    walk_len: int
    step_budget: int
    target_E: int = -1
    arrival_s: float = 0.0


@dataclass
class Workload:
    name: str
    problems: List[Problem] = field(default_factory=list)
    note: str = ""


def plain_small() -> Workload:
    """L=27 (D=14), seed 1, 64 walks of 4096 steps, one round: fully enumerable."""
    L, walks, wl = 27, 64, 4096
    return Workload("plain_L27_64x4096", [Problem(L, 1, walks, wl, walks * wl * ((L + 1) // 2))],
                    "brute-force enumerable parity case")


def plain_l121(walks: int = 131072, walk_len: int = 8192, budget: int = 10 ** 11) -> Workload:
    """L=121 (D=61), seed 1, 131072 walks of 8192 steps, budget 1e11 evaluations."""
    return Workload("plain_L121_131072x8192_budget1e11", [Problem(121, 1, walks, walk_len, budget)])


def batched_instances(n: int = 64, walks: int = 2048, lmin: int = 101, lmax: int = 223,
                      bmin: float = 1e8, bmax: float = 1e10) -> Workload:
    """n instances, odd L uniform in [lmin, lmax], log-uniform budgets, seed 1000+i."""
    rng = SplitMix64(MANIFEST_SEED)
    probs = []
    for i in range(n):
        L = odd_uniform(rng, lmin, lmax)
        budget = int(math.exp(math.log(bmin) + rng.uniform() * (math.log(bmax) - math.log(bmin))))
        probs.append(Problem(L, 1000 + i, walks, paper_walk_len(L), budget))
    return Workload("batched_%dx_L%d-%d_%dwalks" % (n, lmin, lmax, walks), probs)


def serving_stream(duration_s: float = 120.0, rate_per_s: float = 20.0, lmin: int = 121, lmax: int = 301,
                   walks: int = 2048, budget: int = 10 ** 10, seed0: int = 5000) -> Workload:
    """Poisson arrivals (exponential gaps, mean 1/rate), odd L uniform in [lmin, lmax]."""
    rng = SplitMix64(MANIFEST_SEED ^ 0x5E7F)
    t = 0.0
    probs = []
    i = 0
    while True:
        t += -math.log(1.0 - rng.uniform()) / rate_per_s
        if t >= duration_s:
            break
        L = odd_uniform(rng, lmin, lmax)
        probs.append(Problem(L, seed0 + i, walks, paper_walk_len(L), budget, -1, t))
        i += 1
    return Workload("serving_poisson%g_L%d-%d" % (rate_per_s, lmin, lmax), probs)


def plain_large(walks: int = 65536, walk_len: int = 16384) -> Workload:
    """L=449 (D=225), 65536 walks of 16384 steps per round."""
    L = 449
    return Workload("plain_L449_65536x16384", [Problem(L, 1, walks, walk_len, walks * walk_len * ((L + 1) // 2))])
