"""Isomorphism classes (Algorithm 4.4, line 14) computed by the library's host routine
wpm_iso_classes, which needs no GPU: the same partition as the oracle's canonical forms on
the line-13 complexes of n = 2..5 (built by the oracle), hence Table 2's line-15 counts."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2301_00806_gb300 import instances as I, wpm

TABLE2_LINE15 = {2: 2, 3: 5, 4: 49, 5: 256}


def _complexes(n):
    flats, offs = [], [0]
    for rows in I.idcm_orbit_reps(n):
        f = O.candidate_facets("dual", n, n + 4, rows)
        _, _, _, masks = O.enumerate_dfs(n, n + 4, f, cap=-2, base_facet=True,
                                         capacity=1 << 17)
        keep = O.filter_pic_seed(n, n + 4, f, masks).astype(bool)
        fl, of = wpm.complexes_from_masks(f, masks[keep])
        flats.append(fl)
        offs += list(offs[-1] + of[1:].astype(np.int64))
    return np.concatenate(flats), np.asarray(offs, dtype=np.uint64)


@pytest.mark.parametrize("n", sorted(TABLE2_LINE15))
def test_iso_classes_match_the_oracle(n):
    flat, off = _complexes(n)
    cls, count = wpm.iso_classes(n + 4, flat, off)
    assert count == TABLE2_LINE15[n]
    forms, want = {}, []
    for c in range(off.size - 1):
        f = O.canonical_form(n + 4, flat[off[c]:off[c + 1]])
        want.append(forms.setdefault(f, len(forms)))
    assert np.array_equal(cls, np.asarray(want, dtype=np.int32))


def test_iso_classes_of_relabeled_copies():
    flat, off = _complexes(4)
    rng = np.random.default_rng(11)
    pick = rng.choice(off.size - 1, size=30, replace=False)
    fl2, off2 = [], [0]
    for c in pick:  # each picked complex, then a randomly relabeled copy of it
        K = flat[off[c]:off[c + 1]].astype(int)
        perm = rng.permutation(8)
        R = np.array([sum(1 << int(perm[v]) for v in range(8) if (F >> v) & 1) for F in K])
        for X in (K, R):
            fl2.append(X)
            off2.append(off2[-1] + len(X))
    cls, _ = wpm.iso_classes(8, np.concatenate(fl2).astype(np.uint16),
                             np.asarray(off2, dtype=np.uint64))
    assert np.array_equal(cls[0::2], cls[1::2])


def _pic_only_complexes(n, stride):
    """Every stride-th line-7 WPM of n (base facet and cap, all IDCM orbits) that uses all
    n + 4 vertices, without the seedness filter: wedges, suspensions and joins included,
    whose automorphism groups are large."""
    flats, offs = [], [0]
    k = 0
    for rows in I.idcm_orbit_reps(n):
        f = O.candidate_facets("dual", n, n + 4, rows)
        c, _, _, masks = O.enumerate_dfs(n, n + 4, f, cap=-2, base_facet=True,
                                         capacity=1 << 17)
        for i in range(c):
            K = O.masks_to_facets(f, masks[i])
            if not O.pic_full(n + 4, K):
                continue
            if k % stride == 0:
                flats.append(np.asarray(K, dtype=np.uint16))
                offs.append(offs[-1] + len(K))
            k += 1
    return np.concatenate(flats), np.asarray(offs, dtype=np.uint64)


@pytest.mark.parametrize("n,stride", [(3, 1), (4, 3)])
def test_iso_classes_of_symmetric_complexes_match_the_oracle(n, stride):
    flat, off = _pic_only_complexes(n, stride)
    cls, count = wpm.iso_classes(n + 4, flat, off)
    forms, want = {}, []
    for c in range(off.size - 1):
        f = O.canonical_form(n + 4, flat[off[c]:off[c + 1]])
        want.append(forms.setdefault(f, len(forms)))
    assert count == len(forms)
    assert np.array_equal(cls, np.asarray(want, dtype=np.int32))


def _join(*parts):
    """Facets of the join of the boundaries of simplices with the given vertex counts."""
    import itertools
    blocks, v = [], 0
    for size in parts:
        verts = list(range(v, v + size))
        blocks.append([sum(1 << u for u in verts if u != w) for w in verts])
        v += size
    return [sum(c) for c in itertools.product(*blocks)], v


@pytest.mark.parametrize("parts_a,parts_b", [((2, 2, 5, 5), (2, 3, 4, 5)),
                                             ((3, 3, 4, 4), (2, 4, 4, 4)),
                                             ((2, 2, 2, 2, 2, 2, 2), (2, 2, 2, 2, 2, 4))])
def test_iso_classes_of_joins(parts_a, parts_b):
    """Joins of simplex boundaries (automorphism groups up to 2^7 7! = 645,120): seeded
    relabelings of one join share a class, another join on as many vertices does not."""
    A, m = _join(*parts_a)
    B, mb = _join(*parts_b)
    assert m == mb
    rng = np.random.default_rng(m)
    complexes = []
    for X in (A, B):
        for _ in range(4):
            perm = rng.permutation(m)
            complexes.append([sum(1 << int(perm[u]) for u in range(m) if (F >> u) & 1)
                              for F in X])
    cls, count = wpm.iso_classes(m, *_as_flat(complexes))
    assert count == 2
    assert len(set(cls[:4])) == 1 and len(set(cls[4:])) == 1 and cls[0] != cls[4]


def test_iso_classes_input_errors():
    with pytest.raises(wpm.WpmError):
        wpm.iso_classes(6, np.array([1 << 7], dtype=np.uint16), np.array([0, 1], dtype=np.uint64))


# ---------------------------------------------------------------------------------------
# PL sphereness (Algorithm 4.4, line 16) by the library's host routine wpm_pl_spheres
# ---------------------------------------------------------------------------------------

TABLE2_LINE19 = {2: 1, 3: 4, 4: 20, 5: 142}


def _mask(vs):
    return sum(1 << v for v in vs)


def _as_flat(complexes):
    flat = np.concatenate([np.asarray(K, dtype=np.uint16) for K in complexes])
    off = np.concatenate([[0], np.cumsum([len(K) for K in complexes])]).astype(np.uint64)
    return flat, off


@pytest.mark.parametrize("n", sorted(TABLE2_LINE19))
def test_pl_spheres_match_the_oracle(n):
    flat, off = _complexes(n)
    cls, count = wpm.iso_classes(n + 4, flat, off)
    first = [int(np.flatnonzero(cls == c)[0]) for c in range(count)]
    reps = [flat[off[c]:off[c + 1]] for c in first]
    got, k = wpm.pl_spheres(n, n + 4, *_as_flat(reps))
    want = np.array([O.pl_sphere(n, n + 4, K) for K in reps])
    assert np.array_equal(got, want)
    assert k == TABLE2_LINE19[n]


def test_pl_spheres_closed_cases():
    import itertools
    octahedron = [_mask((a, b, c)) for a in (0, 1) for b in (2, 3) for c in (4, 5)]
    rp2 = [_mask(t) for t in ((0, 1, 2), (0, 2, 3), (0, 3, 4), (0, 4, 5), (0, 5, 1),
                              (1, 2, 4), (1, 3, 4), (1, 3, 5), (2, 3, 5), (2, 4, 5))]
    boundary = [_mask(c) for c in itertools.combinations(range(5), 4)]
    got, k = wpm.pl_spheres(3, 6, *_as_flat([octahedron, rp2]))
    assert list(got) == [True, False] and k == 1
    got, _ = wpm.pl_spheres(4, 5, *_as_flat([boundary]))
    assert list(got) == [True]
    with pytest.raises(wpm.WpmError):  # a facet of the wrong size
        wpm.pl_spheres(3, 6, *_as_flat([[_mask((0, 1))]]))


def test_n11_stored_classes_through_the_host_routines():
    """The oracle's n = 11 classes (make_n11_seeds.py): the library's PL-sphere test gives
    the stored flags (4 spheres), and its isomorphism classes put seeded relabelings of each
    class with that class and nowhere else."""
    from conftest import load_n11_seeds
    _, classes, _ = load_n11_seeds()
    reps = [K for _, _, K in classes]
    got, k = wpm.pl_spheres(11, 15, *_as_flat(reps))
    assert list(got) == [s for _, s, _ in classes] and k == 4
    rng = np.random.default_rng(15)
    complexes, want = [], []
    for c, K in enumerate(reps):
        for _ in range(3):
            perm = rng.permutation(15)
            complexes.append([sum(1 << int(perm[u]) for u in range(15) if (F >> u) & 1)
                              for F in K])
            want.append(c)
    order = rng.permutation(len(complexes))
    cls, count = wpm.iso_classes(15, *_as_flat([complexes[i] for i in order]))
    assert count == len(reps)
    labels = {}
    for i, c in zip(order, cls):
        assert labels.setdefault(int(c), want[i]) == want[i]
