"""Pins for the oracle's route through Section 4.4 ("Enumeration for n = 11").

The route: links L (n = 10 WPMs that use all 14 vertices), the cone conditions (1) and (2)
that fix the link of the apex, the conditioned searches, and Algorithm 4.4's filters on
what they find. Checked here against
  - the paper: its Theorem for n = 11 (exactly 4 seeds up to isomorphism) and Table 2's
    n = 10 count at line 7, for the stored results of make_n11_seeds.py;
  - the definition of the conditions: a conditioned search returns exactly the WPMs of the
    unconditioned search whose apex link is L (on small maps, every link of every output);
  - invariants of every stored class and sample (seedness, PL sphereness, the apex link);
  - the paper's own initialization for these runs (the kernel sweep with the leading
    coordinates fixed by a column echelon form), which must give the same WPMs.
"""
import numpy as np
import pytest

import oracle as O
from conftest import load_n11_seeds
from paper_2301_00806_gb300 import instances as I

TOTALS, CLASSES, SAMPLES = load_n11_seeds()
N, M = 11, 15
APEX = 1 << (M - 1)


def _mask_bits(words, count):
    return [j for j in range(count) if (int(words[j // 64]) >> (j % 64)) & 1]


def _apex_link(K, apex):
    return sorted(int(s) ^ apex for s in K if int(s) & apex)


def _link(orbit, words):
    rep = I.idcm_orbit_reps(10)[orbit]
    f10 = O.candidate_facets("dual", 10, 14, rep)
    return rep, [int(f10[j]) for j in _mask_bits(words, len(f10))]


def test_paper_theorem_n11_four_seeds():
    # the paper's Theorem for n = 11: exactly 4 Z2^11-colorable seeds of Picard number 4
    assert TOTALS["spheres"] == 4
    assert sum(1 for c in CLASSES if c[1]) == 4
    assert len(CLASSES) == TOTALS["classes"]
    assert sum(c[0] for c in CLASSES) == TOTALS["pic_seed"]
    # Table 2, n = 10, line 7 (the run the links come from)
    assert TOTALS["line7_n10"] == 99374
    assert TOTALS["links"] <= TOTALS["line7_n10"]
    # the paper's own initialization of the sweep found the same WPMs for every link
    assert TOTALS["sweep_fixed_wpms"] == TOTALS["conditioned_wpms"]
    assert TOTALS["sweep_fixed_pic_seed"] == TOTALS["pic_seed"]


@pytest.mark.parametrize("idx", range(len(CLASSES)))
def test_stored_classes_are_seeds_with_the_stated_sphereness(idx):
    members, sphere, K = CLASSES[idx]
    assert len(K) <= O.ubt_cap(N)
    assert O.pic_seed(N, M, K)
    assert O.pl_sphere(N, M, K) == sphere
    assert list(O.canonical_form(M, K)) == sorted(K)   # stored as canonical forms
    others = [c[2] for j, c in enumerate(CLASSES) if j != idx]
    assert all(sorted(K) != sorted(o) for o in others)


@pytest.mark.parametrize("idx", range(len(SAMPLES)))
def test_sample_link_conditions_and_search(idx):
    orbit, words, count, nodes, probes, kept = SAMPLES[idx]
    rep, L = _link(orbit, words)
    assert O.pic_full(14, L)
    lam, f, fin, fout = O.link_conditions(N, M, rep, L)
    assert sorted(lam) == list(range(1, 16))        # K's map: all 15 nonzero rows
    fin_set = {int(f[j]) for j in _mask_bits(fin, len(f))}
    fout_set = {int(f[j]) for j in _mask_bits(fout, len(f))}
    assert fin_set == {s | APEX for s in L}         # condition (1)
    assert not fin_set & fout_set
    assert fin_set | fout_set == {int(s) for s in f if int(s) & APEX}  # condition (2)
    c, nd, pr, masks = O.enumerate_dfs(N, M, f, cap=O.CAP_UBT, forced_in=fin, forced_out=fout,
                                       list_mode=True, capacity=64)
    assert (c, nd, pr) == (count, nodes, probes)
    keep = O.filter_pic_seed(N, M, f, masks) if c else []
    assert int(np.sum(keep)) == kept
    for i in range(c):
        K = O.masks_to_facets(f, masks[i])
        assert _apex_link(K, APEX) == sorted(L)


@pytest.mark.parametrize("idx", range(len(SAMPLES)))
def test_sample_links_by_the_papers_initialization(idx):
    """Section 4.4's own route: conditions (1), (2) fix the leading coordinates of X in a
    column echelon form of the kernel basis and only the rest is swept; same WPMs as the
    conditioned search."""
    orbit, words, count = SAMPLES[idx][:3]
    rep, L = _link(orbit, words)
    _, f, fin, fout = O.link_conditions(N, M, rep, L)
    c, swept, n_free, masks = O.enumerate_sweep_fixed(N, M, f, cap=O.CAP_UBT, forced_in=fin,
                                                      forced_out=fout, capacity=64)
    c2, _, _, masks2 = O.enumerate_dfs(N, M, f, cap=O.CAP_UBT, forced_in=fin,
                                       forced_out=fout, capacity=64)
    assert c == c2 == count
    assert np.array_equal(masks, masks2)
    assert n_free < O.kernel_dim(N, f) == 64 and swept == 1 << n_free


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_conditioned_search_is_the_definition(seed):
    """Picard number 3, n = 4, m = 7 = 2^3 - 1 (the apex row is then fixed by mu, as for
    n = 11 with Picard number 4): every output K of the unconditioned search, grouped by
    its apex link L; the search conditioned on (mu, L) returns exactly that group."""
    n, m = 4, 7
    rows = I.SplitMix64(seed).shuffle(list(range(1, 8)))
    apex = 1 << (m - 1)
    f = O.candidate_facets("dual", n, m, rows)
    c, _, _, masks = O.enumerate_dfs(n, m, f, list_mode=True, capacity=1 << 16)
    groups = {}
    for i in range(c):
        K = O.masks_to_facets(f, masks[i])
        groups.setdefault(tuple(_apex_link(K, apex)), set()).add(tuple(sorted(K)))
    links = [L for L in groups if L]                # the empty link: K avoids the apex
    assert len(links) > 3
    for L in links:
        lam, f2, fin, fout = O.link_conditions(n, m, rows[:-1], list(L))
        assert lam == rows and np.array_equal(f2, f)
        c2, _, _, masks2 = O.enumerate_dfs(n, m, f2, forced_in=fin, forced_out=fout,
                                           list_mode=True, capacity=1 << 12)
        got = {tuple(sorted(O.masks_to_facets(f2, masks2[i]))) for i in range(c2)}
        assert got == groups[L]
        c3, _, _, masks3 = O.enumerate_sweep_fixed(n, m, f2, forced_in=fin, forced_out=fout,
                                                   capacity=1 << 12)
        assert c3 == c2 and np.array_equal(masks3, masks2)


def test_papers_initialization_with_unsatisfiable_conditions():
    """Forced sets that no WPM meets (a facet forced in with every other parent of one of
    its ridges forced out): the fixed sweep finds nothing, as the search does."""
    n, m = 4, 7
    rows = I.SplitMix64(5).shuffle(list(range(1, 8)))
    f = O.candidate_facets("dual", n, m, rows)
    W = (len(f) + 63) // 64
    a = 0
    r = int(f[a]) & ~(int(f[a]) & -int(f[a]))          # a ridge of facet 0
    fin = np.zeros(W, dtype=np.uint64)
    fout = np.zeros(W, dtype=np.uint64)
    fin[0] |= np.uint64(1)
    for j, s in enumerate(f):
        if j != a and (int(s) & r) == r:
            fout[j // 64] |= np.uint64(1 << (j % 64))
    c, _, _, _ = O.enumerate_sweep_fixed(n, m, f, forced_in=fin, forced_out=fout)
    c2, _, _, _ = O.enumerate_dfs(n, m, f, forced_in=fin, forced_out=fout)
    assert c == c2 == 0


def test_conditioned_search_brute_force_pic4_n2():
    """Picard number 4 at n = 2 (m = 6, so the apex row is given explicitly): the
    conditioned searches against the brute force over all 2^M subsets, grouped by the
    apex link."""
    n, m = 2, 6
    mu = [1, 2, 4, 8, 3]
    apex_row = 12
    f = O.candidate_facets("dual", n, m, mu + [apex_row])
    apex = 1 << (m - 1)
    c, _, _, masks = O.enumerate_brute(n, m, f, list_mode=True, capacity=1 << 12)
    groups = {}
    for i in range(c):
        K = O.masks_to_facets(f, masks[i])
        groups.setdefault(tuple(_apex_link(K, apex)), set()).add(tuple(sorted(K)))
    links = [L for L in groups if L]
    assert len(links) >= 3
    for L in links:
        _, f2, fin, fout = O.link_conditions(n, m, mu, list(L), apex_row=apex_row)
        c2, _, _, masks2 = O.enumerate_dfs(n, m, f2, forced_in=fin, forced_out=fout,
                                           list_mode=True, capacity=1 << 12)
        got = {tuple(sorted(O.masks_to_facets(f2, masks2[i]))) for i in range(c2)}
        assert got == groups[L]
