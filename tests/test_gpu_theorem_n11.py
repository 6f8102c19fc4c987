"""GPU tests of Section 4.4's n = 11 construction (paper_2301_00806_gb300.seeds) and of
the conditioned searches it runs.

  - the n = 10 run without the seedness discard: 114 PL spheres, 39 of them seeds (the
    numbers the paper gives for the links it starts from);
  - the n = 11 run from those 114 links: exactly 4 seeds (the paper's Theorem), the same
    4 isomorphism classes as the oracle's run over every labelled link (stored);
  - the conditioned searches of the 16 stored sample links, bit-exact against the oracle
    run on the same conditions (sorted masks, counts, nodes, probes);
  - Table 2 through the module for n = 2..6.
"""
import numpy as np
import pytest

import oracle as O
from conftest import load_n11_seeds
from paper_2301_00806_gb300 import instances as I, seeds, wpm

pytestmark = pytest.mark.gpu

TOTALS, CLASSES, SAMPLES = load_n11_seeds()
TABLE2 = {2: (90, 22, 2, 1), 3: (1119, 578, 5, 4), 4: (20383, 13679, 49, 20),
          5: (79877, 47012, 256, 142), 6: (322837, 204714, 1791, 733)}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    wpm.lib()


def _sample_link(orbit, words):
    rep = I.idcm_orbit_reps(10)[orbit]
    f10 = O.candidate_facets("dual", 10, 14, rep)
    return rep, [int(f10[j]) for j in range(len(f10)) if (int(words[j // 64]) >> (j % 64)) & 1]


@pytest.mark.parametrize("n", sorted(TABLE2))
def test_table2_through_the_module(n):
    run = seeds.colorable_seeds(n)
    assert (run.line7, run.line13, run.line15, run.line19) == TABLE2[n]


def test_n11_theorem_four_seeds():
    links, run = seeds.colorable_seeds_n11()
    # the links: n = 10 PL spheres that use all 14 vertices, seeds and non-seeds
    assert links.line7 == 99374 == TOTALS["line7_n10"]
    assert links.line13 == TOTALS["links"]
    assert links.line19 == 114
    assert sum(O.pic_seed(10, 14, K) for _, K in links.spheres) == 39
    assert all(O.pic_full(14, K) for _, K in links.spheres)
    # n = 11: exactly 4 seeds, the classes the oracle found through every labelled link
    assert run.maps == 114
    assert run.line19 == 4
    want = {tuple(c[2]) for c in CLASSES if c[1]}
    got = {O.canonical_form(15, K) for _, K in run.spheres}
    assert got == want
    for rows, K in run.spheres:
        assert sorted(rows) == list(range(1, 16))


@pytest.mark.parametrize("post", [0, wpm.POST_PIC | wpm.POST_SEED], ids=["all", "pic_seed"])
def test_conditioned_searches_match_the_oracle(post):
    specs, want = [], []
    for orbit, words, count, nodes, probes, kept in SAMPLES:
        rep, L = _sample_link(orbit, words)
        lam, M, fin, fout = wpm.link_conditions(11, 15, rep, L)
        specs.append(wpm.BatchSpec("dual", 11, 15, lam, cap=wpm.CAP_UBT, forced_in=fin,
                                   forced_out=fout, n_facets=M, post_filter=post))
        _, f, ofin, ofout = O.link_conditions(11, 15, rep, L)
        c, nd, pr, masks = O.enumerate_dfs(11, 15, f, cap=O.CAP_UBT, forced_in=ofin,
                                           forced_out=ofout, list_mode=True, capacity=64)
        assert (c, nd, pr) == (count, nodes, probes)
        if post and c:
            masks = masks[O.filter_pic_seed(11, 15, f, masks).astype(bool)]
        want.append((c, nd, pr, masks))
    got = wpm.enumerate_batch(specs, list_mode=True, capacities=[64] * len(specs))
    for g, (c, nd, pr, masks) in zip(got, want):
        assert g.status == wpm.OK
        if not post:
            assert (g.nodes, g.probes) == (nd, pr)
        assert g.count == masks.shape[0]
        if g.count:
            assert np.array_equal(g.masks, masks)
