"""The paper's main theorem (the number of Z2^n-colorable seeds of Picard number p <= 4, up
to isomorphism) assembled from the oracle's results, on the CPU.

  - p = 3 (n = 2, 3, 4: 1, 1, 1): Algorithm 4.4's steps with Picard number 3 over every
    injective dual map [M; I_3] give the pentagon (n = 2) and C^4(7) (n = 4); the octahedron
    (n = 3) supports a dual map but no injective one, and is added as Section 4.3 does;
  - p = 4, n = 4: the extra seed of Section 4.3 ("20 + 1") is the boundary of the
    4-dimensional cross-polytope: a seed and a PL sphere that is isomorphic to none of the
    complexes the IDCM runs find;
  - p = 4: Table 2's line-19 row, plus that seed, plus the n = 11 seeds of the stored run
    (make_n11_seeds.py) give the theorem's row and its total 3153.
"""
import itertools

import oracle as O
from conftest import load_n11_seeds
from paper_2301_00806_gb300 import instances as I

TABLE2_LINE19 = {2: 1, 3: 4, 4: 20, 5: 142, 6: 733, 7: 1190, 8: 776, 9: 243, 10: 39}
THEOREM_P4 = {2: 1, 3: 4, 4: 21, 5: 142, 6: 733, 7: 1190, 8: 776, 9: 243, 10: 39, 11: 4}
THEOREM_P3 = {2: 1, 3: 1, 4: 1}


def _mask(vs):
    return sum(1 << v for v in vs)


def _cross_polytope_boundary(d):
    """Facets of the boundary of the d-dimensional cross-polytope: one vertex of each of the
    d antipodal pairs {2i, 2i + 1}."""
    return [_mask(2 * i + b for i, b in enumerate(bits)) for bits in itertools.product((0, 1),
                                                                                       repeat=d)]


def _idcm_seeds(n, p):
    """Classes of the seeds (Pic(K) = p, seedness, PL sphere) among the WPMs that contain
    the base facet and support some injective dual map [M; I_p] (every such map, no orbit
    reduction), as canonical forms."""
    m = n + p
    units = [1 << k for k in range(p)]
    allowed = [v for v in range(1, 1 << p) if bin(v).count("1") >= 2]
    forms = set()
    for rows in itertools.combinations(allowed, n):
        f = O.candidate_facets("dual", n, m, list(rows) + units)
        c, _, _, masks = O.enumerate_dfs(n, m, f, base_facet=True, list_mode=True,
                                         capacity=1 << 16)
        for i in range(c):
            K = O.masks_to_facets(f, masks[i])
            if O.pic_seed(n, m, K):
                forms.add(O.canonical_form(m, K))
    return {fm for fm in forms if O.pl_sphere(n, m, list(fm))}


def test_picard3_row():
    got = {n: len(_idcm_seeds(n, 3)) for n in (2, 3, 4)}
    assert got == {2: 1, 3: 0, 4: 1}
    pentagon = [_mask((i, (i + 1) % 5)) for i in range(5)]
    assert _idcm_seeds(2, 3) == {O.canonical_form(5, pentagon)}
    # C^4(7): Gale's evenness condition on 7 cyclically ordered vertices
    c47 = [_mask(s) for s in itertools.combinations(range(7), 4)
           if all(sum(1 for v in s if v > a and v < b) % 2 == 0
                  for a, b in itertools.combinations([x for x in range(7) if x not in s], 2))]
    assert len(c47) == 14
    assert _idcm_seeds(4, 3) == {O.canonical_form(7, c47)}
    # the octahedron: a seed and a PL sphere of Picard number 3 with no injective dual map
    octa = _cross_polytope_boundary(3)
    assert O.pic_seed(3, 6, octa) and O.pl_sphere(3, 6, octa)
    got[3] += 1
    assert got == THEOREM_P3 and sum(got.values()) == 3


def test_cross_polytope_is_the_extra_n4_seed():
    K = _cross_polytope_boundary(4)
    assert O.pic_seed(4, 8, K) and O.pl_sphere(4, 8, K)
    form = O.canonical_form(8, K)
    found = set()
    for rows in I.idcm_orbit_reps(4):
        f = O.candidate_facets("dual", 4, 8, rows)
        c, _, _, masks = O.enumerate_dfs(4, 8, f, cap=O.CAP_UBT, base_facet=True,
                                         list_mode=True, capacity=1 << 16)
        for i in range(c):
            X = O.masks_to_facets(f, masks[i])
            if len(X) == len(K) and O.pic_full(8, X):
                found.add(O.canonical_form(8, X))
    assert form not in found


def test_picard4_row_and_total():
    totals, classes, _ = load_n11_seeds()
    row = dict(TABLE2_LINE19)
    row[4] += 1                                   # the cross-polytope of Section 4.3
    row[11] = sum(1 for c in classes if c[1])     # the oracle's n = 11 run
    assert row == THEOREM_P4
    assert sum(row.values()) == 3153
