"""Seeded synthetic inputs: mod-2 characteristic maps for the enumeration workloads.

This module only draws inputs. It holds none of the enumeration's arithmetic
(no candidate facets, ridges or search); both the CPU oracle and the CUDA path
consume what it produces, so neither regenerates anything itself.

Randomness comes from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out below from its
published definition so that a draw is reproducible on any machine.

Map forms (Section 3.1, the characteristic matrix and its dual):
  * primal: m columns lambda(i) in Z2^n, column i stored as an int whose bit k is row k;
  * dual:   m rows of the dual map lambda-bar in Z2^(m-n) (Picard number m-n, 4 here),
            row i stored as an int (bit k = coordinate k).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import List, Sequence

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator (Steele-Lea-Flood 2014): a 64-bit counter advanced by the
    golden-ratio increment, then finalised by two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, k: int) -> int:
        """An integer in [0, k) (modulo reduction; the bias is below 2^-58 for k < 64)."""
        return self.next_u64() % k

    def uniform01(self) -> float:
        """A float in (0, 1): the top 53 bits, offset by half a step so it is never 0."""
        return ((self.next_u64() >> 11) + 0.5) / float(1 << 53)

    def shuffle(self, xs: list) -> list:
        """Fisher-Yates shuffle in place, drawing from the end of the list down."""
        for i in range(len(xs) - 1, 0, -1):
            j = self.below(i + 1)
            xs[i], xs[j] = xs[j], xs[i]
        return xs


def _spans(vectors: Sequence[int], p: int) -> bool:
    """True when the vectors span Z2^p, tested as: no nonzero functional a vanishes
    on all of them (a spanning set lies in none of the 2^p - 1 hyperplanes a.x = 0)."""
    for a in range(1, 1 << p):
        if all(bin(a & v).count("1") % 2 == 0 for v in vectors):
            return False
    return True


@dataclass
class Instance:
    """One enumeration problem: n, m, the map, its form and the facet-count cap."""
    n: int
    m: int
    kind: str                  # "primal" or "dual"
    cols: List[int]            # m ints (see module docstring)
    seed: int = 0
    label: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def picard(self) -> int:
        return self.m - self.n


def ubt_cap(n: int) -> int:
    """Facets of the cyclic polytope C^n(n+4), the upper bound of Section 4.2:
    C(n+4-ceil(n/2), 4) + C(n+3-floor(n/2), 4)."""
    return math.comb(n + 4 - (n + 1) // 2, 4) + math.comb(n + 3 - n // 2, 4)


def fano_primal(seed: int) -> Instance:
    """n=3, m=7 primal map: the 7 nonzero vectors of Z2^3 as columns, in seeded order.
    Its 3-subsets that are bases are the 35 triples minus the 7 lines of the Fano plane."""
    rng = SplitMix64(seed)
    cols = rng.shuffle(list(range(1, 8)))
    return Instance(n=3, m=7, kind="primal", cols=cols, seed=seed, label=f"fano-s{seed}")


def random_dual(n: int, rng: SplitMix64, p: int = 4) -> List[int]:
    """m = n+p distinct nonzero rows of Z2^p, drawn as the first m of a seeded shuffle of
    all 2^p - 1 nonzero vectors, redrawn until they span Z2^p (rank p)."""
    m = n + p
    if m > (1 << p) - 1:
        raise ValueError(f"m={m} distinct nonzero vectors do not exist in Z2^{p}")
    while True:
        rows = rng.shuffle(list(range(1, 1 << p)))[:m]
        if _spans(rows, p):
            return rows


def single_dual(n: int, seed: int) -> Instance:
    """A single Picard-4 instance: dual rows = m distinct nonzero vectors of Z2^4 of rank 4."""
    rng = SplitMix64(seed)
    return Instance(n=n, m=n + 4, kind="dual", cols=random_dual(n, rng), seed=seed,
                    label=f"dual-n{n}-s{seed}")


def batch_duals(count: int = 4096, n_lo: int = 3, n_hi: int = 8, seed: int = 0) -> List[Instance]:
    """The batched workload: `count` instances, n uniform in {n_lo..n_hi}, each a dual map
    drawn as in `single_dual`, all from one seeded stream."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        n = n_lo + rng.below(n_hi - n_lo + 1)
        out.append(Instance(n=n, m=n + 4, kind="dual", cols=random_dual(n, rng), seed=seed,
                            label=f"batch-{i}"))
    return out


def poisson_jobs(rate: float = 200.0, duration: float = 60.0, n_lo: int = 5, n_hi: int = 9,
                 seed: int = 0) -> List[Instance]:
    """The serving workload: arrival times of a Poisson process of the given rate over
    `duration` seconds (exponential gaps -ln(U)/rate), each job a dual map with n uniform
    in {n_lo..n_hi}. The arrival time is stored in `extra['t_arrival']`."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    while True:
        t += -math.log(rng.uniform01()) / rate
        if t >= duration:
            return out
        n = n_lo + rng.below(n_hi - n_lo + 1)
        out.append(Instance(n=n, m=n + 4, kind="dual", cols=random_dual(n, rng), seed=seed,
                            label=f"job-{len(out)}", extra={"t_arrival": t}))


def full_dual_n11(seed: int) -> Instance:
    """The largest Picard-4 instance: n=11, m=15, the dual rows are all 15 nonzero vectors
    of Z2^4 in seeded order."""
    rng = SplitMix64(seed)
    return Instance(n=11, m=15, kind="dual", cols=rng.shuffle(list(range(1, 16))), seed=seed,
                    label=f"n11-s{seed}")


def simplex_boundary_primal(n: int) -> Instance:
    """lambda = [I_n | 1]: every n-subset of [n+1] is a basis, so the candidates are all
    facets of the boundary of the n-simplex (Picard number 1)."""
    cols = [1 << k for k in range(n)] + [(1 << n) - 1]
    return Instance(n=n, m=n + 1, kind="primal", cols=cols, label=f"simplex-n{n}")


# --- IDCM orbit representatives (Section 4.2, Proposition 4.3) ---------------------------

def _permute_coords(v: int, perm: Sequence[int]) -> int:
    """Apply a coordinate permutation of Z2^4: bit k of v moves to bit perm[k]."""
    out = 0
    for k in range(4):
        if (v >> k) & 1:
            out |= 1 << perm[k]
    return out


def idcm_orbit_reps(n: int, p: int = 4) -> List[List[int]]:
    """One representative per orbit of Lambda(n, p) under S_n x S_p (Proposition 4.3).

    An element of Lambda(n, p) is [M; I_p] with no repeated rows. Its rows for vertices
    n+1..n+p are the unit vectors, so the rows of M are n distinct vectors that are
    neither a unit vector nor zero (a zero row would put that vertex in every facet, a
    cone; the orbit counts of Table 1 are those of the weight >= 2 vectors). S_n reorders
    the rows of M, so M is an n-subset; S_p permutes coordinates. A representative is the
    lexicographically least sorted tuple of its orbit. Returned as dual rows: the n rows
    of M (ascending), then e_1..e_p."""
    if p != 4:
        raise ValueError("orbit generation is written for Picard number 4")
    allowed = [v for v in range(1, 16) if bin(v).count("1") >= 2]
    perms = list(itertools.permutations(range(4)))
    seen = set()
    reps = []
    for sub in itertools.combinations(allowed, n):
        if sub in seen:
            continue
        orbit = {tuple(sorted(_permute_coords(v, pr) for v in sub)) for pr in perms}
        seen |= orbit
        rep = min(orbit)
        reps.append(list(rep) + [1, 2, 4, 8])
    reps.sort()
    return reps
