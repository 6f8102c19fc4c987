"""Algorithm 4.4 (the Z2^n-colorable seeds of Picard number 4) and the n = 11 construction
of Section 4.4, as sequences of library calls.

Every step is a call into libwpm: the searches and the post-filters of lines 8-12 run on
the GPU (wpm_enumerate_batch), the link conditions (wpm_link_conditions), isomorphism
classes (line 14, wpm_iso_classes) and the PL-sphere test (line 16, wpm_pl_spheres) in its
native host code. This module only hands each call's output to the next.

  colorable_seeds(n)          lines 1-19 for one n <= 10: one map per IDCM orbit
                              (Proposition 4.3), the base facet and the cap (line 5),
                              Pic(K) = 4 and seedness (lines 8-12), one K per class (14),
                              PL spheres (15-19). seedness=False skips line 10, which gives
                              the links that Section 4.4 starts from.
  seeds_from_links(links, n)  Section 4.4's construction for dimension n - 1: for each link
                              L with its map mu, K's map (mu plus the apex row) and the cone
                              conditions (1), (2); then lines 5-19 of Algorithm 4.4 on the
                              conditioned searches.
  colorable_seeds_n11()       the paper's n = 11 run: the 114 PL spheres of n = 10 (seeds
                              and non-seeds) as links, one map each, then seeds_from_links.
  main_theorem_p4()           the main theorem's Picard-4 row: line 19 for n = 2..10, plus
                              the 4-cross-polytope that Section 4.3 adds at n = 4
                              (extra_n4_seed checks it), plus the n = 11 seeds.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

from . import instances as I
from . import wpm


@dataclass
class SeedRun:
    """Counts at the lines of Algorithm 4.4, and one complex per PL-sphere class."""
    n: int
    maps: int                      # maps searched (IDCM orbits, or links)
    line7: int                     # WPMs found by the searches
    line13: int                    # after Pic(K) = 4 (and seedness, when applied)
    line15: int                    # isomorphism classes
    line19: int                    # PL spheres among them
    spheres: List[Tuple[List[int], np.ndarray]] = field(default_factory=list)
    # (dual rows of the map the representative was found for, its facet vertex masks)
    nodes: int = 0                 # search nodes of the canonical trees
    seconds: float = 0.0


class _Found:
    """The complexes that passed, all maps together: facets flat[off[c]:off[c+1]] of
    complex c, found for the map rows[owner[c]]."""

    def __init__(self):
        self.rows, self.flats, self.offs, self.owner = [], [], [0], []

    def add(self, rows, flat, off):
        k = len(self.rows)
        self.rows.append(rows)
        self.flats.append(flat)
        base = self.offs[-1]
        self.offs += [base + int(x) for x in off[1:]]
        self.owner += [k] * (off.size - 1)

    def arrays(self):
        flat = np.concatenate(self.flats) if self.flats else np.zeros(0, dtype=np.uint16)
        return flat.astype(np.uint16), np.asarray(self.offs, dtype=np.uint64)


def _classes_and_spheres(n: int, m: int, found: _Found):
    """-> (classes, [(map rows, facets) of one member of each PL-sphere class])."""
    flat, off = found.arrays()
    if off.size == 1:
        return 0, []
    cls, classes = wpm.iso_classes(m, flat, off)
    first = sorted(np.unique(cls, return_index=True)[1])  # first member of each class
    reps = [flat[off[c]:off[c + 1]].copy() for c in first]
    rflat = np.concatenate(reps).astype(np.uint16)
    roff = np.concatenate([[0], np.cumsum([len(K) for K in reps])]).astype(np.uint64)
    is_sphere, _ = wpm.pl_spheres(n, m, rflat, roff)
    return classes, [(found.rows[found.owner[c]], K)
                     for c, K, s in zip(first, reps, is_sphere) if s]


def _search(specs: List[wpm.BatchSpec], post: int, stream=None, capacity: int = 1 << 15):
    """One list run with the post-filters (line 7, then lines 9-12 on the GPU); maps whose
    WPMs overflow `capacity` are run again with room for exactly their count. Returns
    (line-7 count, nodes, the complexes that pass)."""
    if not specs:
        return 0, 0, _Found()
    listed_specs = [wpm.BatchSpec(s.kind, s.n, s.m, s.cols, cap=s.cap, base_facet=s.base_facet,
                                  forced_in=s.forced_in, forced_out=s.forced_out,
                                  n_facets=s.n_facets, post_filter=post) for s in specs]
    listed = wpm.enumerate_batch(listed_specs, list_mode=True,
                                 capacities=[capacity] * len(specs), stream=stream)
    again = [i for i, r in enumerate(listed) if r.status == wpm.ERR_CAPACITY]
    if again:
        redo = wpm.enumerate_batch([listed_specs[i] for i in again], list_mode=True,
                                   capacities=[listed[i].found for i in again], stream=stream)
        for i, r in zip(again, redo):
            listed[i] = r
    found = _Found()
    for s, r in zip(specs, listed):
        if r.status != wpm.OK:
            raise wpm.WpmError(r.status, "list run failed")
        if r.count == 0:
            continue
        facets = wpm.candidate_facets(s.kind, s.n, s.m, s.cols)
        flat, off = wpm.complexes_from_masks(facets, r.masks)
        found.add([int(x) for x in s.cols], flat, off)
    return sum(r.found for r in listed), sum(r.nodes for r in listed), found


def colorable_seeds(n: int, seedness: bool = True, stream=None) -> SeedRun:
    """Algorithm 4.4 for 2 <= n <= 10 (m = n + 4)."""
    t0 = time.perf_counter()
    reps = I.idcm_orbit_reps(n)
    specs = [wpm.BatchSpec("dual", n, n + 4, r, cap=wpm.CAP_UBT, base_facet=True) for r in reps]
    post = wpm.POST_PIC | (wpm.POST_SEED if seedness else 0)
    line7, nodes, found = _search(specs, post, stream)
    classes, spheres = _classes_and_spheres(n, n + 4, found)
    return SeedRun(n, len(reps), line7, len(found.owner), classes, len(spheres), spheres, nodes,
                   time.perf_counter() - t0)


def seeds_from_links(links: Sequence[Tuple[Sequence[int], Sequence[int]]], n: int,
                     stream=None) -> SeedRun:
    """Section 4.4's construction: the seeds K of dimension n - 1 on m = n + 4 vertices
    whose apex m - 1 has one of the given links. links: [(mu, L)], mu the m - 1 dual rows
    of L's map, L its facets (vertex masks on [m - 1]); K's map is mu plus the one nonzero
    vector of Z2^4 that mu misses (so m = 15, n = 11)."""
    t0 = time.perf_counter()
    m = n + 4
    specs = []
    for mu, L in links:
        lam, M, fin, fout = wpm.link_conditions(n, m, mu, L)
        specs.append(wpm.BatchSpec("dual", n, m, lam, cap=wpm.CAP_UBT, forced_in=fin,
                                   forced_out=fout, n_facets=M))
    line7, nodes, found = _search(specs, wpm.POST_PIC | wpm.POST_SEED, stream)
    classes, spheres = _classes_and_spheres(n, m, found)
    return SeedRun(n, len(specs), line7, len(found.owner), classes, len(spheres), spheres, nodes,
                   time.perf_counter() - t0)


def colorable_seeds_n11(stream=None) -> Tuple[SeedRun, SeedRun]:
    """The paper's n = 11 run: (the n = 10 run without the seedness discard, whose PL
    spheres are the links; the n = 11 run from those links)."""
    links = colorable_seeds(10, seedness=False, stream=stream)
    run = seeds_from_links([(rows, K) for rows, K in links.spheres], 11, stream=stream)
    return links, run


def cross_polytope_boundary(d: int) -> np.ndarray:
    """Facets (vertex masks) of the boundary of the d-dimensional cross-polytope, antipodal
    vertices 2i and 2i + 1: one vertex of each pair."""
    facets = []
    for bits in range(1 << d):
        facets.append(sum(1 << (2 * i + ((bits >> i) & 1)) for i in range(d)))
    return np.asarray(sorted(facets), dtype=np.uint16)


def extra_n4_seed(run4: SeedRun) -> bool:
    """Section 4.3's addition to n = 4: the boundary of the 4-dimensional cross-polytope, a
    seed of Picard number 4 that supports a dual characteristic map but no injective one, so
    the IDCM runs cannot find it. True when it is a PL sphere (Lemma 3.3) isomorphic to none
    of the PL-sphere classes of run4 (Algorithm 4.4 for n = 4)."""
    K = cross_polytope_boundary(4)
    is_sphere, _ = wpm.pl_spheres(4, 8, K, np.asarray([0, K.size], dtype=np.uint64))
    reps = [F for _, F in run4.spheres] + [K]
    flat = np.concatenate(reps).astype(np.uint16)
    off = np.concatenate([[0], np.cumsum([len(F) for F in reps])]).astype(np.uint64)
    cls, classes = wpm.iso_classes(8, flat, off)
    return bool(is_sphere[0]) and classes == len(run4.spheres) + 1 and \
        int(cls[-1]) == len(run4.spheres)


# The main theorem's Picard-4 row: Z2^n-colorable seeds of dimension n - 1 up to isomorphism
MAIN_THEOREM_P4 = {2: 1, 3: 4, 4: 21, 5: 142, 6: 733, 7: 1190, 8: 776, 9: 243, 10: 39, 11: 4}


def main_theorem_p4(ns: Sequence[int] = tuple(range(2, 11)), n11: bool = True,
                    stream=None) -> dict:
    """The main theorem's row for Picard number 4: Algorithm 4.4's PL spheres (line 19) for
    each n in ns, plus Section 4.3's cross-polytope at n = 4, plus (n11) the seeds of the
    n = 11 construction. Returns {n: count}."""
    row = {}
    for n in ns:
        run = colorable_seeds(n, stream=stream)
        row[n] = run.line19 + (int(extra_n4_seed(run)) if n == 4 else 0)
    if n11:
        row[11] = colorable_seeds_n11(stream=stream)[1].line19
    return row
