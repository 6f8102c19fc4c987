"""The composition of Algorithm 4.4 and of Section 4.4's n = 11 construction in
paper_2301_00806_gb300.seeds, checked on the CPU: the module's two GPU calls
(wpm.enumerate_batch, wpm.candidate_facets) are replaced, in this test only, by the oracle
computing the same results; the host calls (link conditions, isomorphism classes, PL
spheres) are the library's own. What is checked is that the module hands each output to
the next call correctly: Table 2's four rows for n = 2..6, and the stored n = 11 sample
links. The GPU
path itself is tested in test_gpu_theorem_n11.py."""
import numpy as np
import pytest

import oracle as O
from conftest import load_n11_seeds
from paper_2301_00806_gb300 import instances as I, seeds, wpm

TABLE2 = {2: (90, 22, 2, 1), 3: (1119, 578, 5, 4), 4: (20383, 13679, 49, 20),
          5: (79877, 47012, 256, 142), 6: (322837, 204714, 1791, 733)}
_, _, SAMPLES = load_n11_seeds()


def _oracle_batch(specs, list_mode=True, capacities=None, tuning=None, stream=None,
                  device_out=None, words=None):
    out = []
    for i, s in enumerate(specs):
        kind = {wpm.PRIMAL: "primal", wpm.DUAL: "dual"}.get(s.kind, s.kind)
        f = O.candidate_facets(kind, s.n, s.m, s.cols)
        cap = O.CAP_UBT if s.cap == wpm.CAP_UBT else s.cap
        c, nodes, probes, masks = O.enumerate_dfs(s.n, s.m, f, cap=cap, base_facet=s.base_facet,
                                                  forced_in=s.forced_in, forced_out=s.forced_out,
                                                  list_mode=list_mode, capacity=1 << 16)
        W = max(1, (len(f) + 63) // 64)
        found = c
        if list_mode and capacities is not None and c > int(capacities[i]):
            # as the library does: the count needed, no masks, a per-instance status
            out.append(wpm.Result(c, nodes, probes, len(f), 0, W, None, wpm.ERR_CAPACITY, c))
            continue
        if list_mode and s.post_filter and c:
            if s.post_filter & wpm.POST_SEED:
                keep = O.filter_pic_seed(s.n, s.m, f, masks).astype(bool)
            else:
                keep = np.array([O.pic_full(s.m, O.masks_to_facets(f, row)) for row in masks])
            masks = masks[keep]
            c = int(keep.sum())
        out.append(wpm.Result(c, nodes, probes, len(f), 0, W, masks if list_mode else None,
                              wpm.OK, found))
    return out


def test_search_reruns_only_the_maps_that_overflow(on_oracle, monkeypatch):
    calls = []

    def spy(specs, **kw):
        calls.append((len(specs), list(kw.get("capacities") or [])))
        return _oracle_batch(specs, **kw)

    monkeypatch.setattr(wpm, "enumerate_batch", spy)
    reps = I.idcm_orbit_reps(4)
    specs = [wpm.BatchSpec("dual", 4, 8, r, cap=wpm.CAP_UBT, base_facet=True) for r in reps]
    line7, nodes, found = seeds._search(specs, wpm.POST_PIC | wpm.POST_SEED, capacity=600)
    assert line7 == 20383
    assert calls[0] == (len(reps), [600] * len(reps))
    # one more call, for the maps above 600 WPMs only, with room for exactly their count
    assert len(calls) == 2 and 0 < calls[1][0] < len(reps) and min(calls[1][1]) > 600


@pytest.fixture
def on_oracle(monkeypatch):
    monkeypatch.setattr(wpm, "enumerate_batch", _oracle_batch)
    monkeypatch.setattr(wpm, "candidate_facets",
                        lambda kind, n, m, cols: O.candidate_facets(
                            {wpm.PRIMAL: "primal", wpm.DUAL: "dual"}.get(kind, kind), n, m, cols))


@pytest.mark.parametrize("n", sorted(TABLE2))
def test_colorable_seeds_gives_table2(on_oracle, n):
    run = seeds.colorable_seeds(n)
    assert (run.line7, run.line13, run.line15, run.line19) == TABLE2[n]
    assert run.maps == len(I.idcm_orbit_reps(n))
    for rows, K in run.spheres[:: max(1, len(run.spheres) // 50)]:
        assert O.pic_seed(n, n + 4, K) and O.pl_sphere(n, n + 4, K)


def test_colorable_seeds_without_seedness_keeps_the_seeds(on_oracle):
    n = 4
    seeded = seeds.colorable_seeds(n)
    every = seeds.colorable_seeds(n, seedness=False)
    assert every.line7 == seeded.line7
    assert every.line13 >= seeded.line13 and every.line19 >= seeded.line19
    forms = {O.canonical_form(n + 4, K) for _, K in every.spheres}
    assert all(O.canonical_form(n + 4, K) in forms for _, K in seeded.spheres)
    # the non-seeds among the PL spheres (wedges and suspensions) are exactly the extra ones
    n_seeds = sum(O.pic_seed(n, n + 4, K) for _, K in every.spheres)
    assert n_seeds == seeded.line19
    # n = 2: the only 1-sphere on 6 vertices is the hexagon, a seed
    two = seeds.colorable_seeds(2, seedness=False)
    assert two.line19 == 1 and len(two.spheres[0][1]) == 6


def test_seeds_from_links_on_the_stored_samples(on_oracle):
    links = []
    for orbit, words, *_ in SAMPLES:
        rep = I.idcm_orbit_reps(10)[orbit]
        f10 = O.candidate_facets("dual", 10, 14, rep)
        L = [int(f10[j]) for j in range(len(f10)) if (int(words[j // 64]) >> (j % 64)) & 1]
        links.append((rep, L))
    run = seeds.seeds_from_links(links, 11)
    assert run.maps == len(SAMPLES)
    assert run.line7 == sum(s[2] for s in SAMPLES)
    assert run.nodes == sum(s[3] for s in SAMPLES)
    assert run.line13 == sum(s[5] for s in SAMPLES)
    for rows, K in run.spheres:
        assert sorted(rows) == list(range(1, 16))
        assert O.pic_seed(11, 15, K)


def test_bench_table2_section(on_oracle, monkeypatch):
    """bench.py's paper_table2 section over the module, on the CPU (the oracle in place of
    the GPU calls, n = 2..4, no device synchronisation)."""
    import torch
    import bench
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(bench, "TABLE2", {n: TABLE2[n] for n in (2, 3, 4)})
    out = bench.run_paper_table2(None)
    assert out["all_exact"] and [r["n"] for r in out["rows"]] == [2, 3, 4]
    assert "error" in bench._guarded(lambda: 1 / 0)


def test_main_theorem_row_small_n(on_oracle):
    row = seeds.main_theorem_p4(ns=(2, 3, 4), n11=False)
    assert row == {n: seeds.MAIN_THEOREM_P4[n] for n in (2, 3, 4)}
    K = seeds.cross_polytope_boundary(4)
    assert len(K) == 16 and O.pic_seed(4, 8, K) and O.pl_sphere(4, 8, K)


def test_bench_main_theorem_section(on_oracle):
    import bench
    table2 = {"rows": [{"n": n, "lines_7_13_15_19": [0, 0, 0, seeds.MAIN_THEOREM_P4[n]]}
                       for n in range(2, 11)]}
    table2["rows"][2]["lines_7_13_15_19"][3] -= 1      # Table 2 prints 20 at n = 4
    out = bench.run_main_theorem(table2, {"n11_seeds": 4}, None)
    assert out["exact"] and out["total"] == 3153 and out["cross_polytope_added"]


def test_seeds_from_no_links(on_oracle):
    run = seeds.seeds_from_links([], 11)
    assert (run.maps, run.line7, run.line13, run.line15, run.line19) == (0, 0, 0, 0, 0)
    assert run.spheres == []
