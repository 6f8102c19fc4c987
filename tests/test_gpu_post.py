"""GPU post-filters of Algorithm 4.4 (lines 8-12): Pic(K) = 4 (every vertex used) and the
seedness condition of Proposition 3.1, applied to the sorted lists. Against Table 2's
line-13 row for n = 2..10 and against the oracle's filter map by map."""
import numpy as np
import pytest

from paper_2301_00806_gb300 import instances as I
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TABLE2_LINE13 = {2: 22, 3: 578, 4: 13679, 5: 47012, 6: 204714, 7: 310217, 8: 305280,
                 9: 140933, 10: 57956}
BOTH = 3  # WPM_POST_PIC | WPM_POST_SEED


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2301_00806_gb300 import wpm
    wpm.lib()
    return wpm


@pytest.mark.parametrize("n", sorted(TABLE2_LINE13))
def test_table2_line13(W, n):
    reps = I.idcm_orbit_reps(n)
    specs = [W.BatchSpec("dual", n, n + 4, r, cap=-2, base_facet=True) for r in reps]
    counts = [r.count for r in W.enumerate_batch(specs, list_mode=False)]
    fspecs = [W.BatchSpec("dual", n, n + 4, r, cap=-2, base_facet=True, post_filter=BOTH)
              for r in reps]
    res = W.enumerate_batch(fspecs, list_mode=True, capacities=[max(1, c) for c in counts])
    assert all(r.status == 0 for r in res)
    assert sum(r.count for r in res) == TABLE2_LINE13[n]


@pytest.mark.parametrize("seed", range(8))
def test_post_filter_matches_oracle(W, seed):
    n = 4 + seed % 3
    inst = I.single_dual(n, 300 + seed)
    f = O.instance_facets(inst)
    c, _, _, masks = O.enumerate_dfs(n, n + 4, f, cap=-2, capacity=1 << 17)
    keep = O.filter_pic_seed(n, n + 4, f, masks).astype(bool)
    g = W.enumerate("dual", n, n + 4, inst.cols, cap=-2, capacity=max(1, c),
                    post_filter=BOTH)
    assert g.count == int(keep.sum())
    assert np.array_equal(g.masks, masks[keep])


@pytest.mark.parametrize("seed", range(4))
def test_pic_only(W, seed):
    n = 5
    inst = I.single_dual(n, 400 + seed)
    f = O.instance_facets(inst)
    c, _, _, masks = O.enumerate_dfs(n, n + 4, f, cap=-2, capacity=1 << 17)
    allv = (1 << (n + 4)) - 1
    keep = []
    for row in masks:
        used = 0
        for j in range(f.size):
            if (int(row[j // 64]) >> (j % 64)) & 1:
                used |= int(f[j])
        keep.append(used == allv)
    keep = np.array(keep, dtype=bool)
    g = W.enumerate("dual", n, n + 4, inst.cols, cap=-2, capacity=max(1, c), post_filter=1)
    assert g.count == int(keep.sum())
    assert np.array_equal(g.masks, masks[keep])


def test_post_filter_errors(W):
    inst = I.single_dual(5, 0)
    spec = W.BatchSpec("dual", 5, 9, inst.cols, cap=-2, post_filter=BOTH)
    with pytest.raises(W.WpmError) as e:
        W.enumerate_batch([spec], list_mode=False)
    assert e.value.code == W.ERR_INPUT
    bad = W.BatchSpec("dual", 5, 9, inst.cols, cap=-2, post_filter=8)
    with pytest.raises(W.WpmError) as e:
        W.enumerate_batch([bad], list_mode=True, capacities=[1 << 12])
    assert e.value.code == W.ERR_INPUT


TABLE2_LINE15 = {2: 2, 3: 5, 4: 49, 5: 256, 6: 1791, 7: 2194, 8: 1401, 9: 381, 10: 56}


@pytest.mark.parametrize("n", sorted(TABLE2_LINE15))
def test_table2_line15(W, n):
    """Algorithm 4.4 lines 1-15: GPU enumeration and post-filters over one map per IDCM
    orbit, then the library's isomorphism classes (host) across all of them."""
    reps = I.idcm_orbit_reps(n)
    specs = [W.BatchSpec("dual", n, n + 4, r, cap=-2, base_facet=True) for r in reps]
    counts = [r.count for r in W.enumerate_batch(specs, list_mode=False)]
    fspecs = [W.BatchSpec("dual", n, n + 4, r, cap=-2, base_facet=True, post_filter=BOTH)
              for r in reps]
    res = W.enumerate_batch(fspecs, list_mode=True, capacities=[max(1, c) for c in counts])
    flats, offs = [], [0]
    for r, rows in zip(res, reps):
        f = W.candidate_facets("dual", n, n + 4, rows)
        fl, of = W.complexes_from_masks(f, r.masks)
        flats.append(fl)
        offs += list(offs[-1] + of[1:].astype(np.int64))
    _, classes = W.iso_classes(n + 4, np.concatenate(flats), np.asarray(offs, dtype=np.uint64))
    assert classes == TABLE2_LINE15[n]


TABLE2_LINE19 = {2: 1, 3: 4, 4: 20, 5: 142, 6: 733, 7: 1190, 8: 776, 9: 243, 10: 39}


@pytest.mark.parametrize("n", sorted(TABLE2_LINE19))
def test_table2_line19(W, n):
    """All of Algorithm 4.4 for n <= 10: GPU enumeration and post-filters, then (host) one
    representative per isomorphism class and the PL-sphere criterion of Lemma 3.3."""
    reps = I.idcm_orbit_reps(n)
    specs = [W.BatchSpec("dual", n, n + 4, r, cap=-2, base_facet=True) for r in reps]
    counts = [r.count for r in W.enumerate_batch(specs, list_mode=False)]
    fspecs = [W.BatchSpec("dual", n, n + 4, r, cap=-2, base_facet=True, post_filter=BOTH)
              for r in reps]
    res = W.enumerate_batch(fspecs, list_mode=True, capacities=[max(1, c) for c in counts])
    flats, offs = [], [0]
    for r, rows in zip(res, reps):
        fl, of = W.complexes_from_masks(W.candidate_facets("dual", n, n + 4, rows), r.masks)
        flats.append(fl)
        offs += list(offs[-1] + of[1:].astype(np.int64))
    flat, off = np.concatenate(flats), np.asarray(offs, dtype=np.uint64)
    cls, classes = W.iso_classes(n + 4, flat, off)
    first = np.unique(cls, return_index=True)[1]
    rflat = np.concatenate([flat[off[c]:off[c + 1]] for c in first])
    roff = np.concatenate([[0], np.cumsum([int(off[c + 1] - off[c]) for c in first])])
    _, spheres = W.pl_spheres(n, n + 4, rflat, roff.astype(np.uint64))
    assert spheres == TABLE2_LINE19[n]
