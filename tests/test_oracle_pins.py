"""Pins for the CPU oracle: values the paper prints, closed forms, independent methods.

Every test here runs on the CPU. Each checks the oracle against something other than
itself, chosen so that a plausible slip (a dropped condition, a wrong order, a missing
parent, a wrong rank test) fails at least one of them.
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest

import oracle as O
from conftest import load_table
from paper_2301_00806_gb300 import instances as I

T1 = load_table("table1_picard4.txt")
T2 = load_table("table2_line7.txt")


def all_nsubsets(n, m):
    return np.array([sum(1 << v for v in c) for c in itertools.combinations(range(m), n)],
                    dtype=np.uint16)


def masks_to_sets(masks, M):
    out = []
    for row in masks:
        s = set()
        for j in range(M):
            if (int(row[j // 64]) >> (j % 64)) & 1:
                s.add(j)
        out.append(frozenset(s))
    return out


def ridge_degrees(facet_vmasks):
    """Degrees of every (n-1)-face among the given facets, from vertex masks directly."""
    deg = Counter()
    for f in facet_vmasks:
        f = int(f)
        v = f
        while v:
            low = v & -v
            deg[f ^ low] += 1
            v ^= low
    return deg


# --------------------------------------------------------------------------------------
# Table 1 (Section 4.2)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("row", T1, ids=[f"n{r[0]}" for r in T1])
def test_table1_idcm_orbit_count(row):
    n, _, orbits, _ = row
    assert len(I.idcm_orbit_reps(n)) == orbits


@pytest.mark.parametrize("row", T1, ids=[f"n{r[0]}" for r in T1])
def test_table1_max_kernel_dim(row):
    """max over IDCM orbits of dim ker_Z2 A(F(lambda)): pins the candidate facets
    (Proposition 4.2), the ridges and the GF(2) rank together."""
    n, _, _, want = row
    got = max(O.kernel_dim(n, O.candidate_facets("dual", n, n + 4, r))
              for r in I.idcm_orbit_reps(n))
    assert got == want


@pytest.mark.parametrize("row", T1, ids=[f"n{r[0]}" for r in T1])
def test_table1_kernel_dim_all_subsets(row):
    n, want, _, _ = row
    assert O.kernel_dim(n, all_nsubsets(n, n + 4)) == want
    assert want == math.comb(n + 3, n)  # the closed form C(m-1, n)


# --------------------------------------------------------------------------------------
# The upper-bound-theorem cap (Section 4.2) against other closed forms
# --------------------------------------------------------------------------------------

def test_ubt_cap_against_cyclic_polytope_closed_forms():
    # polygon: m edges; simplicial 3-polytope: 2m - 4 facets (Euler); neighborly
    # 4-polytope: m(m-3)/2 facets
    assert O.ubt_cap(2) == 6
    assert O.ubt_cap(3) == 2 * 7 - 4
    assert O.ubt_cap(4) == 8 * 5 // 2
    # McMullen's formula for the cyclic d-polytope on m vertices:
    #   d = 2k: m/(m-k) C(m-k, k);  d = 2k+1: 2 C(m-k-1, k)
    for n in range(2, 12):
        m, k = n + 4, n // 2
        want = (m * math.comb(m - k, k)) // (m - k) if n % 2 == 0 else 2 * math.comb(m - k - 1, k)
        assert O.ubt_cap(n) == want
        assert I.ubt_cap(n) == want


# --------------------------------------------------------------------------------------
# Candidate facets
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(16))
def test_fano_candidates_are_the_non_lines(seed):
    inst = I.fano_primal(seed)
    f = O.instance_facets(inst)
    # three distinct nonzero vectors of Z2^3 are dependent exactly when they are a line
    # of the Fano plane: a ^ b ^ c == 0
    want = sorted(
        sum(1 << v for v in t) for t in itertools.combinations(range(7), 3)
        if inst.cols[t[0]] ^ inst.cols[t[1]] ^ inst.cols[t[2]] != 0)
    assert f.size == 28 == 35 - 7
    assert sorted(int(x) for x in f) == want


def _primal_from_dual_normal_form(rows, n):
    """lambda = [I_n | M] from the dual [M; I_4] (Section 3.1): primal column n+k collects
    bit k of the rows of M."""
    cols = [1 << i for i in range(n)]
    for k in range(4):
        cols.append(sum(1 << i for i in range(n) if (rows[i] >> k) & 1))
    return cols


@pytest.mark.parametrize("n", range(2, 12))
def test_gale_duality_primal_equals_dual(n):
    """Proposition 4.2: the facets read from the dual map (complement is a basis of
    Z2^4) equal those read from the primal map (the facet is a basis of Z2^n)."""
    for rows in I.idcm_orbit_reps(n)[:6]:
        fd = O.candidate_facets("dual", n, n + 4, rows)
        fp = O.candidate_facets("primal", n, n + 4, _primal_from_dual_normal_form(rows, n))
        assert np.array_equal(fd, fp)


def test_full_n11_sizes():
    inst = I.full_dual_n11(0)
    f = O.instance_facets(inst)
    # one facet per 4-subset of rows forming a basis: |GL(4,2)| / 4! ordered bases
    gl42 = (16 - 1) * (16 - 2) * (16 - 4) * (16 - 8)
    assert f.size == gl42 // 24 == 840
    r, npar = O.ridges(11, f)
    # ridges = 10-subsets inside some candidate, counted here from the vertex masks
    inside = {int(x) & ~(1 << v) for x in f for v in range(15) if (int(x) >> v) & 1}
    assert r.size == len(inside)
    assert max(npar) <= 5


def test_candidates_lexicographic_order():
    inst = I.single_dual(6, 3)
    f = O.instance_facets(inst)
    tuples = [tuple(v for v in range(16) if (int(x) >> v) & 1) for x in f]
    assert tuples == sorted(tuples)
    r, _ = O.ridges(6, f)
    rt = [tuple(v for v in range(16) if (int(x) >> v) & 1) for x in r]
    assert rt == sorted(rt)


# --------------------------------------------------------------------------------------
# Table 2, first row (Algorithm 4.4 line 7): sums over IDCM orbit representatives
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("row", [r for r in T2 if r[0] <= 7], ids=[f"n{r[0]}" for r in T2 if r[0] <= 7])
def test_table2_line7_counts(row):
    n, want = row
    total = 0
    for rows in I.idcm_orbit_reps(n):
        f = O.candidate_facets("dual", n, n + 4, rows)
        c, _, _, _ = O.enumerate_dfs(n, n + 4, f, cap=O.CAP_UBT, base_facet=True, list_mode=False)
        total += c
    assert total == want


def test_table2_n2_by_cycle_families():
    """n = 2 by an independent route: a 1-dimensional WPM is a family of vertex-disjoint
    cycles. Families through the base edge {0,1} = all families minus those of the graph
    without that edge; capped at 6 edges (the bound for n = 2)."""
    total = 0
    for rows in I.idcm_orbit_reps(2):
        f = O.candidate_facets("dual", 2, 6, rows)
        without = np.array([x for x in f if int(x) != 0b11], dtype=np.uint16)
        assert without.size == f.size - 1
        total += O.n2_cycle_sets(f, 6) - O.n2_cycle_sets(without, 6)
    assert total == 90


# --------------------------------------------------------------------------------------
# Independent routes agree: brute force (the definition), kernel sweep, search
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("cap", [O.CAP_NONE, O.CAP_UBT])
def test_fano_three_routes(cap):
    inst = I.fano_primal(5)
    f = O.instance_facets(inst)
    b = O.enumerate_brute(3, 7, f, cap=cap)
    s = O.enumerate_sweep(3, 7, f, cap=cap)
    d = O.enumerate_dfs(3, 7, f, cap=cap)
    assert b[0] == s[0] == d[0] == (666 if cap == O.CAP_UBT else 1303)
    assert np.array_equal(b[3], s[3]) and np.array_equal(b[3], d[3])


@pytest.mark.parametrize("seed", range(6))
def test_n5_sweep_equals_search(seed):
    inst = I.single_dual(5, seed)
    f = O.instance_facets(inst)
    s = O.enumerate_sweep(5, 9, f, cap=O.CAP_UBT, capacity=1 << 14)
    d = O.enumerate_dfs(5, 9, f, cap=O.CAP_UBT, capacity=1 << 14)
    assert s[0] == d[0] and np.array_equal(s[3], d[3])


def _random_case(rng, n):
    m = rng.integers(n + 1, min(16, n + 5) + 1)
    allf = all_nsubsets(n, int(m))
    M = int(min(allf.size, rng.integers(6, 19)))
    pick = np.sort(rng.choice(allf.size, size=M, replace=False))
    facets = allf[pick]
    return int(m), facets


@pytest.mark.parametrize("seed", range(40))
def test_random_conditions_brute_equals_search(seed):
    """Random facet sets and random properties: forced-in/out sets, a cap and general
    affine functions with mixed-sign coefficients."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 5))
    m, facets = _random_case(rng, n)
    M = facets.size
    kw = {}
    if seed % 2:
        kw["cap"] = int(rng.integers(0, M + 1))
    if seed % 3 == 0:
        kw["forced_in"] = [int(1 << int(rng.integers(0, M)))]
    if seed % 5 == 0:
        kw["forced_out"] = [int(rng.integers(0, 1 << M))]
    if seed % 4 in (1, 2):
        kw["affine"] = [(int(rng.integers(-3, 6)), rng.integers(-2, 3, size=M).tolist())
                        for _ in range(int(rng.integers(1, 3)))]
    b = O.enumerate_brute(n, m, facets, **kw)
    d = O.enumerate_dfs(n, m, facets, **kw)
    s = O.enumerate_sweep(n, m, facets, **kw)
    assert b[0] == d[0] == s[0]
    assert np.array_equal(b[3], d[3]) and np.array_equal(b[3], s[3])


# --------------------------------------------------------------------------------------
# Proposition 2.1 invariant and closed forms
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("inst", [I.fano_primal(1), I.single_dual(4, 2), I.single_dual(5, 7)],
                         ids=["fano", "n4", "n5"])
def test_every_output_is_a_wpm_and_every_wpm_is_output(inst):
    f = O.instance_facets(inst)
    c, _, _, masks = O.enumerate_dfs(inst.n, inst.m, f, cap=O.CAP_UBT, capacity=1 << 14)
    sets = masks_to_sets(masks, f.size)
    assert len(set(sets)) == c  # no duplicates
    cap = I.ubt_cap(inst.n)
    for s in sets:
        deg = ridge_degrees([f[j] for j in s])
        assert all(d == 2 for d in deg.values())  # each present ridge in exactly two facets
        assert len(s) <= cap
    # sorted ascending as multiword integers
    keys = [sum(int(w) << (64 * i) for i, w in enumerate(row)) for row in masks]
    assert keys == sorted(keys)


@pytest.mark.parametrize("n", range(2, 12))
def test_simplex_boundary_closed_form(n):
    """All n-subsets of [n+1]: the only WPMs are the empty complex and the boundary of
    the n-simplex (a facet forces its neighbour across every ridge)."""
    inst = I.simplex_boundary_primal(n)
    f = O.instance_facets(inst)
    assert f.size == n + 1
    c, nodes, probes, masks = O.enumerate_dfs(n, n + 1, f)
    assert c == 2
    assert [int(x) for x in masks[:, 0]] == [0, (1 << (n + 1)) - 1]


def test_empty_complex_reading():
    """Reading: the empty complex satisfies Proposition 2.1; it is output exactly when
    every property holds at K = 0 (yes under the cap alone, no with the base facet)."""
    rows = I.idcm_orbit_reps(3)[0]
    f = O.candidate_facets("dual", 3, 7, rows)
    _, _, _, a = O.enumerate_dfs(3, 7, f, cap=O.CAP_UBT)
    _, _, _, b = O.enumerate_dfs(3, 7, f, cap=O.CAP_UBT, base_facet=True)
    assert not a[0].any()
    assert b[:, 0].min() & 1  # facet 0 = {0,1,2} is in every output


def test_n2_cycles_match_search_on_all_orbits():
    for rows in I.idcm_orbit_reps(2):
        f = O.candidate_facets("dual", 2, 6, rows)
        for cap in (6, -1):
            d = O.enumerate_dfs(2, 6, f, cap=cap, list_mode=False)
            assert d[0] == O.n2_cycle_sets(f, cap)


def test_k4_cycle_families_closed_form():
    """K_4: the empty family, 4 triangles and 3 four-cycles (no two disjoint)."""
    f = all_nsubsets(2, 4)
    assert O.n2_cycle_sets(f) == 8
    assert O.enumerate_dfs(2, 4, f, list_mode=False)[0] == 8


def test_n11_subtree_golden_file_reproduces():
    """Two lines of tests/golden/n11_subtrees.txt re-derived by the oracle (walk + search)."""
    import os
    from conftest import GOLDEN
    inst = I.full_dual_n11(0)
    f = O.instance_facets(inst)
    lines = [l.split() for l in open(os.path.join(GOLDEN, "n11_subtrees.txt")) if not l.startswith("#")]
    for t in (lines[4], lines[5]):
        seed = int(t[0])
        a, b = O.walk(11, 15, f, seed, 6, cap=O.CAP_UBT)
        assert [f"{int(x):016x}" for x in a] + [f"{int(x):016x}" for x in b] == t[1:29]
        c, nodes, probes, _ = O.enumerate_dfs(11, 15, f, cap=O.CAP_UBT, forced_in=a, forced_out=b,
                                              list_mode=False)
        assert (c, nodes, probes) == (int(t[29]), int(t[30]), int(t[31]))


# ---------------------------------------------------------------------------------------
# Algorithm 4.4 lines 8-12: Pic(K) = 4 (every vertex used) and the seedness condition of
# Proposition 3.1
# ---------------------------------------------------------------------------------------

TABLE2_LINE13 = {2: 22, 3: 578, 4: 13679, 5: 47012, 6: 204714}  # Table 2, line 13


@pytest.mark.parametrize("n", sorted(TABLE2_LINE13))
def test_table2_line13_post_filters(n):
    total = 0
    for rows in I.idcm_orbit_reps(n):
        f = O.candidate_facets("dual", n, n + 4, rows)
        _, _, _, masks = O.enumerate_dfs(n, n + 4, f, cap=-2, base_facet=True,
                                         capacity=1 << 17)
        total += int(O.filter_pic_seed(n, n + 4, f, masks).sum())
    assert total == TABLE2_LINE13[n]


def _mask(vs):
    return sum(1 << v for v in vs)


def test_simplex_boundary_is_not_a_seed():
    # the boundary of a simplex has one minimal non-face, all its vertices: no edge is split
    import itertools
    for n in range(2, 7):
        facets = [_mask(c) for c in itertools.combinations(range(n + 1), n)]
        assert O.pic_seed(n, n + 1, facets) is False


def _hexagon():
    return [_mask((i, (i + 1) % 6)) for i in range(6)]


def _wedge(facets, v, m):
    """Wedge (J-construction) at vertex v: v becomes v and a new vertex m; a facet through v
    takes both, a facet missing v is joined with each of them."""
    out = []
    for F in facets:
        if (F >> v) & 1:
            out.append(F | (1 << m))
        else:
            out += [F | (1 << v), F | (1 << m)]
    return out


def _suspension(facets, m):
    return [F | (1 << m) for F in facets] + [F | (1 << (m + 1)) for F in facets]


def test_hexagon_and_two_triangles_are_seeds():
    assert O.pic_seed(2, 6, _hexagon()) is True
    tri = [_mask(e) for e in ((0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5))]
    assert O.pic_seed(2, 6, tri) is True


def test_a_wedge_is_not_a_seed():
    # the two vertices a wedge makes from one lie in the same minimal non-faces
    for v in range(6):
        assert O.pic_seed(3, 7, _wedge(_hexagon(), v, 6)) is False


def test_suspension_keeps_seedness():
    # the suspension of a seed is a seed (Section 4.4); of a non-seed, a non-seed
    assert O.pic_seed(3, 8, _suspension(_hexagon(), 6)) is True
    w = _wedge(_hexagon(), 0, 6)
    assert O.pic_seed(4, 9, _suspension(w, 7)) is False


def test_unused_vertex_fails_pic():
    assert O.pic_seed(2, 7, _hexagon()) is False


# ---------------------------------------------------------------------------------------
# Algorithm 4.4 line 14: one representative per isomorphism class (canonical forms)
# ---------------------------------------------------------------------------------------

TABLE2_LINE15 = {2: 2, 3: 5, 4: 49, 5: 256}  # Table 2, |K°(n,4)| at line 15


def _line13_complexes(n):
    out = []
    for rows in I.idcm_orbit_reps(n):
        f = O.candidate_facets("dual", n, n + 4, rows)
        _, _, _, masks = O.enumerate_dfs(n, n + 4, f, cap=-2, base_facet=True,
                                         capacity=1 << 17)
        keep = O.filter_pic_seed(n, n + 4, f, masks)
        out += [O.masks_to_facets(f, row) for row, k in zip(masks, keep) if k]
    return out


TABLE2_LINE19 = {2: 1, 3: 4, 4: 20, 5: 142}  # Table 2, |K°(n,4)| at line 19


@pytest.fixture(scope="module")
def line15_representatives():
    """For n = 2..5: one line-13 complex per canonical form."""
    reps = {}
    for n in sorted(TABLE2_LINE15):
        forms = {}
        for K in _line13_complexes(n):
            forms.setdefault(O.canonical_form(n + 4, K), K)
        reps[n] = list(forms.values())
    return reps


@pytest.mark.parametrize("n", sorted(TABLE2_LINE15))
def test_table2_line15_isomorphism_classes(n, line15_representatives):
    assert len(line15_representatives[n]) == TABLE2_LINE15[n]


@pytest.mark.parametrize("n", sorted(TABLE2_LINE19))
def test_table2_line19_pl_spheres(n, line15_representatives):
    got = sum(O.pl_sphere(n, n + 4, K) for K in line15_representatives[n])
    assert got == TABLE2_LINE19[n]


def test_pl_sphere_closed_cases():
    import itertools
    octahedron = [_mask((a, b, c)) for a in (0, 1) for b in (2, 3) for c in (4, 5)]
    assert O.pl_sphere(3, 6, octahedron) is True
    for n in range(2, 7):  # the boundary of a simplex
        facets = [_mask(c) for c in itertools.combinations(range(n + 1), n)]
        assert O.pl_sphere(n, n + 1, facets) is True
    # the 6-vertex real projective plane: every edge in two triangles, H_1(RP^2; Z2) = Z2
    rp2 = [_mask(t) for t in ((0, 1, 2), (0, 2, 3), (0, 3, 4), (0, 4, 5), (0, 5, 1),
                              (1, 2, 4), (1, 3, 4), (1, 3, 5), (2, 3, 5), (2, 4, 5))]
    assert O.pl_sphere(3, 6, rp2) is False
    tri = [_mask(e) for e in ((0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5))]
    assert O.pl_sphere(2, 6, tri) is False                     # two circles
    assert O.pl_sphere(3, 8, _suspension(tri, 6)) is False     # suspension of two circles


def _relabel(K, perm):
    return [sum(1 << perm[v] for v in range(16) if (F >> v) & 1) for F in K]


def test_canonical_form_is_invariant_under_relabeling():
    rng = np.random.default_rng(5)
    cx = _line13_complexes(4)
    for K in [cx[i] for i in rng.choice(len(cx), size=40, replace=False)]:
        base = O.canonical_form(8, K)
        for _ in range(3):
            perm = list(rng.permutation(8))
            assert O.canonical_form(8, _relabel(K, perm)) == base


def test_canonical_form_separates_non_isomorphic():
    hexagon = [_mask((i, (i + 1) % 6)) for i in range(6)]
    triangles = [_mask(e) for e in ((0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5))]
    assert O.canonical_form(6, hexagon) != O.canonical_form(6, triangles)
