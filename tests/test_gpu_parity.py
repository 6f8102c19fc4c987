"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Everything is integer work, so the bar is bit-exact: the same sorted list of facet masks,
the same count, and the same node and probe counts of the canonical search tree.
"""
import numpy as np
import pytest

import oracle as O
from conftest import load_table
from paper_2301_00806_gb300 import instances as I

pytestmark = pytest.mark.gpu

T2 = load_table("table2_line7.txt")


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2301_00806_gb300 import wpm
    wpm.lib()
    return wpm


def oracle_run(inst, **kw):
    f = O.instance_facets(inst)
    return f, O.enumerate_dfs(inst.n, inst.m, f, capacity=1 << 15, **kw)


def assert_same(gpu, orc, nodes=True):
    c, nd, pr, masks = orc
    assert gpu.count == c
    if nodes:
        assert (gpu.nodes, gpu.probes) == (nd, pr)
    if masks is not None and gpu.masks is not None:
        assert gpu.masks.shape == masks.shape
        assert np.array_equal(gpu.masks, masks)


# ---------------------------------------------------------------------------------------
# candidate facets
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", range(2, 12))
def test_candidate_facets_match(W, n):
    for rows in I.idcm_orbit_reps(n)[:5]:
        assert np.array_equal(W.candidate_facets("dual", n, n + 4, rows),
                              O.candidate_facets("dual", n, n + 4, rows))
    inst = I.single_dual(n, 3) if n <= 11 else None
    assert np.array_equal(W.candidate_facets("dual", n, n + 4, inst.cols), O.instance_facets(inst))


def test_candidate_facets_primal(W):
    for s in range(16):
        inst = I.fano_primal(s)
        assert np.array_equal(W.candidate_facets("primal", 3, 7, inst.cols), O.instance_facets(inst))


# ---------------------------------------------------------------------------------------
# single instances: the Fano map (n=3, m=7) and the n=5 dual maps
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("cap", [-1, -2])
def test_fano_all_seeds(W, seed, cap):
    inst = I.fano_primal(seed)
    f, orc = oracle_run(inst, cap=cap)
    g = W.enumerate("primal", 3, 7, inst.cols, cap=cap)
    assert g.M == 28 and g.N == 21
    assert g.count == (666 if cap == -2 else 1303)
    assert_same(g, orc)


@pytest.mark.parametrize("seed", range(16))
def test_n5_dual_seeds(W, seed):
    inst = I.single_dual(5, seed)
    f, orc = oracle_run(inst, cap=-2)
    g = W.enumerate("dual", 5, 9, inst.cols, cap=-2)
    assert_same(g, orc)


def test_count_mode_equals_list_mode(W):
    inst = I.single_dual(6, 1)
    a = W.enumerate("dual", 6, 10, inst.cols, cap=-2, list_mode=True, capacity=1 << 16)
    b = W.enumerate("dual", 6, 10, inst.cols, cap=-2, list_mode=False)
    assert (a.count, a.nodes, a.probes) == (b.count, b.nodes, b.probes)
    assert b.masks is None


@pytest.mark.parametrize("n", [6, 7])
def test_larger_single_instances(W, n):
    inst = I.single_dual(n, 0)
    f, orc = oracle_run(inst, cap=-2)
    g = W.enumerate("dual", n, n + 4, inst.cols, cap=-2, capacity=1 << 17)
    assert_same(g, orc)


# ---------------------------------------------------------------------------------------
# Table 2, first row, through the batched entry point
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("row", [r for r in T2 if r[0] <= 7], ids=[f"n{r[0]}" for r in T2 if r[0] <= 7])
def test_table2_batched_against_oracle_and_paper(W, row):
    n, want = row
    reps = I.idcm_orbit_reps(n)
    specs = [W.BatchSpec("dual", n, n + 4, r, cap=-2, base_facet=True) for r in reps]
    res = W.enumerate_batch(specs, list_mode=False)
    assert sum(r.count for r in res) == want
    if n <= 5:
        for r, rows in zip(res, reps):
            f = O.candidate_facets("dual", n, n + 4, rows)
            c, nd, pr, _ = O.enumerate_dfs(n, n + 4, f, cap=-2, base_facet=True, list_mode=False)
            assert (r.count, r.nodes, r.probes) == (c, nd, pr)


def test_table2_n4_lists(W):
    reps = I.idcm_orbit_reps(4)
    specs = [W.BatchSpec("dual", 4, 8, r, cap=-2, base_facet=True) for r in reps]
    res = W.enumerate_batch(specs, list_mode=True, capacities=[4096] * len(reps))
    for r, rows in zip(res, reps):
        f = O.candidate_facets("dual", 4, 8, rows)
        assert_same(r, O.enumerate_dfs(4, 8, f, cap=-2, base_facet=True, capacity=4096))


# ---------------------------------------------------------------------------------------
# mixed batch, and the work-splitting paths forced by extreme tuning
# ---------------------------------------------------------------------------------------

def _mixed(count=48, seed=11):
    return [inst for inst in I.batch_duals(count, 3, 6, seed=seed)]


@pytest.mark.parametrize("tuning", [None,
                                    {"budget": 1},
                                    {"budget": 7, "frontier_target": 1},
                                    {"budget": 64, "frontier_target": 100000},
                                    {"budget": 3, "ring_items": 3000, "threads_per_block": 64},
                                    {"budget": 1000000, "frontier_target": 1, "threads_per_block": 256},
                                    {"search": 1, "budget": 2, "frontier_target": 1},
                                    {"search": 2},
                                    {"search": 2, "budget": 1, "frontier_target": 1},
                                    {"search": 2, "budget": 5, "idle_percent": 100, "threads_per_block": 64},
                                    {"search": 1},
                                    {"search": 1, "budget": 1},
                                    {"search": 1, "donate_levels": -1},
                                    {"search": 1, "donate_levels": 16, "donate_every": 1},
                                    {"search": 1, "feed_levels": -1, "hungry_items": 1 << 40, "budget": 9},
                                    {"search": 1, "feed_levels": 1, "hungry_items": 1, "budget": 5},
                                    {"search": 1, "ring_items": 3000, "donate_every": 1, "frontier_target": 1},
                                    {"search": 1, "graph": -1, "donate_every": 1},
                                    {"search": 2, "graph": -1}],
                         ids=["default", "budget1", "nofrontier", "wide", "smallring", "nobudget",
                              "thread_budget2", "warp", "warp_budget1", "warp_small", "thread",
                              "thread_budget1", "thread_nodonate", "thread_donate_often",
                              "thread_feed_all", "thread_feed_one", "thread_ring_full",
                              "thread_host_loop", "warp_host_loop"])
def test_mixed_batch_with_tunings(W, tuning):
    insts = _mixed()
    orc = [oracle_run(inst, cap=-2)[1] for inst in insts]
    specs = [W.BatchSpec("dual", i.n, i.m, i.cols, cap=-2) for i in insts]
    res = W.enumerate_batch(specs, list_mode=True, capacities=[o[0] + 1 for o in orc], tuning=tuning)
    for g, o in zip(res, orc):
        assert g.status == 0
        assert_same(g, o)


@pytest.mark.parametrize("search", [1, 2])
def test_pass_loop_graph_matches_host_loop(W, search):
    """The depth-first pass loop run as one CUDA graph launch (a conditional while node) gives
    what the host-driven loop gives, counters included."""
    insts = _mixed(24, seed=5)
    specs = [W.BatchSpec("dual", i.n, i.m, i.cols, cap=-2) for i in insts]
    g = W.enumerate_batch(specs, list_mode=True, capacities=[8192] * len(specs),
                          tuning={"search": search})
    sg = W.last_run_stats()
    h = W.enumerate_batch(specs, list_mode=True, capacities=[8192] * len(specs),
                          tuning={"search": search, "graph": -1})
    sh = W.last_run_stats()
    assert sg["graph_launches"] == 1 and sh["graph_launches"] == 0
    assert sg["dfs_passes"] >= 1
    for a, b in zip(g, h):
        assert (a.status, a.count, a.nodes, a.probes) == (b.status, b.count, b.nodes, b.probes)
        assert np.array_equal(a.masks, b.masks)


def test_autotune_choice_is_used_and_exact(W):
    """wpm_autotune returns one of its candidates; a batch of the same signature run with
    tuning NULL then uses it, and every tuning gives the oracle's results."""
    insts = _mixed(32, seed=9)
    specs = [W.BatchSpec("dual", i.n, i.m, i.cols, cap=-2) for i in insts]
    best, ms = W.autotune(specs, sample=16)
    assert best["search"] in (1, 2) and ms > 0
    orc = [oracle_run(inst, cap=-2)[1] for inst in insts]
    for tun in (None, {k: v for k, v in best.items() if v}):
        res = W.enumerate_batch(specs, list_mode=True, capacities=[o[0] + 1 for o in orc],
                                tuning=tun)
        for r, o in zip(res, orc):
            assert_same(r, o)
        assert W.last_run_stats()["search"] == best["search"]


def test_batch_into_device_tensors(W):
    import torch
    insts = _mixed(12, seed=3)
    orc = [oracle_run(inst, cap=-2)[1] for inst in insts]
    caps = [o[0] for o in orc]
    # int64 storage viewed as uint64 words; room for 4 words per mask (M <= 256)
    outs = [torch.zeros((max(c, 1), 4), dtype=torch.int64, device="cuda") for c in caps]
    specs = [W.BatchSpec("dual", i.n, i.m, i.cols, cap=-2) for i in insts]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    res = W.enumerate_batch(specs, list_mode=True, capacities=caps, device_out=outs, stream=stream)
    for g, o, t in zip(res, orc, outs):
        assert g.count == o[0]
        flat = t.flatten()[: g.count * g.words].cpu().numpy().view(np.uint64)
        assert np.array_equal(flat.reshape(-1, g.words), o[3])


# ---------------------------------------------------------------------------------------
# properties: forced facets, affine functions, explicit facet lists
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(24))
def test_random_properties(W, seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 6))
    inst = I.single_dual(n, seed)
    f = O.instance_facets(inst)
    M = f.size
    kw = {"cap": int(rng.choice([-1, -2, int(rng.integers(3, 40))]))}
    words = (M + 63) // 64
    if seed % 3 == 0:
        fi = np.zeros(words, dtype=np.uint64)
        j = int(rng.integers(0, M))
        fi[j // 64] |= np.uint64(1) << np.uint64(j % 64)
        kw["forced_in"] = fi
    if seed % 4 == 0:
        fo = np.zeros(words, dtype=np.uint64)
        for j in rng.choice(M, size=min(M, 6), replace=False):
            fo[j // 64] |= np.uint64(1) << np.uint64(int(j) % 64)
        kw["forced_out"] = fo
    if seed % 2 == 1:
        kw["affine"] = [(int(rng.integers(0, 30)), rng.integers(-2, 3, size=M).tolist())
                        for _ in range(int(rng.integers(1, 4)))]
    if seed % 5 == 2:
        kw["base_facet"] = True
    orc = O.enumerate_dfs(n, n + 4, f, capacity=1 << 15, **kw)
    g = W.enumerate("dual", n, n + 4, inst.cols, n_facets=M, capacity=1 << 15, **kw)
    assert_same(g, orc)


@pytest.mark.parametrize("seed", range(12))
def test_explicit_facet_lists(W, seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(2, 5))
    m = int(rng.integers(n + 2, min(16, n + 6) + 1))
    import itertools
    allf = [sum(1 << v for v in c) for c in itertools.combinations(range(m), n)]
    k = int(min(len(allf), rng.integers(8, 60)))
    pick = sorted(rng.choice(len(allf), size=k, replace=False).tolist())
    facets = np.array([allf[i] for i in pick], dtype=np.uint16)
    shuffled = facets.copy()
    rng.shuffle(shuffled)
    cap = int(rng.choice([-1, 12]))
    orc = O.enumerate_dfs(n, m, facets, cap=cap, capacity=1 << 16)
    g = W.enumerate_facets(shuffled, n, m, cap=cap, capacity=1 << 16)
    assert g.M == k
    assert_same(g, orc)


# ---------------------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------------------

def test_empty_facet_list(W):
    g = W.enumerate_facets([], 3, 7)
    assert g.count == 1 and g.M == 0 and g.masks.shape == (1, 1) and int(g.masks[0, 0]) == 0


@pytest.mark.parametrize("n", range(2, 13))
def test_simplex_boundary(W, n):
    inst = I.simplex_boundary_primal(n)
    g = W.enumerate("primal", n, n + 1, inst.cols)
    assert g.M == n + 1 and g.count == 2
    assert [int(x) for x in g.masks[:, 0]] == [0, (1 << (n + 1)) - 1]
    assert_same(g, O.enumerate_dfs(n, n + 1, O.instance_facets(inst)))


def test_cap_zero_and_base_facet_missing(W):
    inst = I.single_dual(4, 0)
    g = W.enumerate("dual", 4, 8, inst.cols, cap=0)
    assert g.count == 1 and int(g.masks[0, 0]) == 0
    f = O.instance_facets(inst)
    orc = O.enumerate_dfs(4, 8, f, base_facet=True, cap=-2)
    g = W.enumerate("dual", 4, 8, inst.cols, base_facet=True, cap=-2)
    assert_same(g, orc)


def test_capacity_error_reports_the_count(W):
    inst = I.fano_primal(2)
    from paper_2301_00806_gb300.wpm import Output, _p, lib
    import ctypes as C
    cols = np.asarray(inst.cols, dtype=np.uint32)
    buf = np.zeros(10, dtype=np.uint64)
    o = Output()
    o.masks = _p(buf, C.c_uint64)
    o.capacity = 10
    r = lib().wpm_enumerate(_p(cols, C.c_uint32), 0, 3, 7, None, C.byref(o), 0)
    assert r == W.ERR_CAPACITY and o.count == 1303 and not buf.any()


@pytest.mark.parametrize("kw,code", [
    (dict(kind="dual", n=5, m=9, cols=[1, 2, 3, 3, 4, 5, 6, 7, 8]), -1),   # repeated rows
    (dict(kind="dual", n=3, m=7, cols=[1, 2, 3, 4, 5, 6, 7]), -1),          # rank 3 < 4
    (dict(kind="dual", n=5, m=9, cols=[0, 2, 3, 4, 5, 6, 7, 8, 9]), -1),    # zero row
    (dict(kind="primal", n=1, m=3, cols=[1, 1, 1]), -1),                     # n < 2
    (dict(kind="primal", n=3, m=17, cols=list(range(1, 18))), -1),          # m > 16
    (dict(kind="primal", n=2, m=4, cols=[1, 2, 4, 3]), -1),                  # bit above Z2^2
])
def test_invalid_inputs(W, kw, code):
    with pytest.raises(W.WpmError) as e:
        W.enumerate(kw["kind"], kw["n"], kw["m"], kw["cols"])
    assert e.value.code == code


def test_ubt_needs_picard4(W):
    with pytest.raises(W.WpmError):
        W.enumerate("primal", 3, 8, [1, 2, 4, 3, 5, 6, 7, 1], cap=-2)


def test_limit_exceeded(W):
    import itertools
    rng = np.random.default_rng(7)
    # a generic primal map of rank 8 on 16 vertices: thousands of 8-subsets are bases
    cols = [1 << i for i in range(8)] + rng.integers(1, 256, size=8).tolist()
    with pytest.raises(W.WpmError) as e:
        W.enumerate("primal", 8, 16, cols)
    assert e.value.code == W.ERR_LIMIT
    # 2000 facets of size 8 on 16 vertices have far more than 4096 ridges
    allf = [sum(1 << v for v in c) for c in itertools.combinations(range(16), 8)]
    pick = rng.choice(len(allf), size=2000, replace=False)
    with pytest.raises(W.WpmError) as e:
        W.enumerate_facets([allf[i] for i in pick], 8, 16)
    assert e.value.code == W.ERR_LIMIT


# ---------------------------------------------------------------------------------------
# every output is a WPM (Proposition 2.1), checked from vertex masks at a larger size
# ---------------------------------------------------------------------------------------

def test_outputs_are_wpms_n8(W):
    from collections import Counter
    inst = I.single_dual(8, 5)
    f = W.candidate_facets("dual", 8, 12, inst.cols)
    g = W.enumerate("dual", 8, 12, inst.cols, cap=-2, capacity=1 << 18)
    rng = np.random.default_rng(0)
    for row in g.masks[rng.choice(g.count, size=min(300, g.count), replace=False)]:
        fac = [int(f[j]) for j in range(f.size) if (int(row[j // 64]) >> (j % 64)) & 1]
        deg = Counter()
        for x in fac:
            v = x
            while v:
                low = v & -v
                deg[x ^ low] += 1
                v ^= low
        assert all(d == 2 for d in deg.values())
        assert len(fac) <= I.ubt_cap(8)
    keys = [tuple(int(w) for w in reversed(r)) for r in g.masks]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


# ---------------------------------------------------------------------------------------
# Table 2 (first row) at the sizes the paper ran for hours and days per orbit
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("row", [r for r in T2 if r[0] >= 8], ids=[f"n{r[0]}" for r in T2 if r[0] >= 8])
@pytest.mark.parametrize("search", [1, 2], ids=["thread", "warp"])
def test_table2_line7_large_n(W, row, search):
    n, want = row
    reps = I.idcm_orbit_reps(n)
    specs = [W.BatchSpec("dual", n, n + 4, r, cap=-2, base_facet=True) for r in reps]
    res = W.enumerate_batch(specs, list_mode=False, tuning={"search": search})
    assert sum(r.count for r in res) == want


@pytest.mark.parametrize("n", [9, 10])
def test_table2_one_orbit_against_oracle(W, n):
    rows = I.idcm_orbit_reps(n)[-1]
    f = O.candidate_facets("dual", n, n + 4, rows)
    c, nd, pr, _ = O.enumerate_dfs(n, n + 4, f, cap=-2, base_facet=True, list_mode=False)
    g = W.enumerate("dual", n, n + 4, rows, cap=-2, base_facet=True, list_mode=False)
    assert (g.count, g.nodes, g.probes) == (c, nd, pr)


def test_n11_orbit_against_oracle(W):
    """The one IDCM orbit of n = 11 (15 vertices, 840 candidate facets) with the base facet and
    the cap: no count for it is printed in the paper (Table 2 stops at n = 10), so the oracle
    is the check (about 66M search nodes on the host)."""
    rows = I.idcm_orbit_reps(11)[0]
    f = O.candidate_facets("dual", 11, 15, rows)
    c, nd, pr, _ = O.enumerate_dfs(11, 15, f, cap=-2, base_facet=True, list_mode=False)
    for search in (1, 2):
        g = W.enumerate_batch([W.BatchSpec("dual", 11, 15, rows, cap=-2, base_facet=True)],
                              list_mode=False, tuning={"search": search})[0]
        assert (g.count, g.nodes, g.probes) == (c, nd, pr)


# ---------------------------------------------------------------------------------------
# The largest Picard-4 map (n = 11, all 15 nonzero dual rows): 64 seeded subtrees, exact
# ---------------------------------------------------------------------------------------

def _n11_subtrees():
    import os
    from conftest import GOLDEN
    rows = []
    for line in open(os.path.join(GOLDEN, "n11_subtrees.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        words = [int(x, 16) for x in t[1:29]]
        rows.append((int(t[0]), np.array(words[:14], dtype=np.uint64),
                     np.array(words[14:], dtype=np.uint64), int(t[29]), int(t[30]), int(t[31])))
    return rows


@pytest.mark.parametrize("search", [1, 2], ids=["thread", "warp"])
def test_n11_subtrees_batched(W, search):
    inst = I.full_dual_n11(0)
    rows = _n11_subtrees()
    assert len(rows) == 64
    specs = [W.BatchSpec("dual", 11, 15, inst.cols, cap=-2, forced_in=a, forced_out=b, n_facets=840)
             for _, a, b, _, _, _ in rows]
    res = W.enumerate_batch(specs, list_mode=False, tuning={"search": search})
    for r, (seed, _, _, c, nd, pr) in zip(res, rows):
        assert r.status == 0
        assert (r.count, r.nodes, r.probes) == (c, nd, pr), seed


@pytest.mark.parametrize("search", [1, 2], ids=["thread", "warp"])
def test_n11_full_map_against_stored_oracle(W, search):
    """The whole largest Picard-4 map under the cap, against the oracle's stored result
    (tests/golden/n11_full.txt, written by make_n11_full.py)."""
    import os
    from conftest import GOLDEN
    line = [l for l in open(os.path.join(GOLDEN, "n11_full.txt")) if not l.startswith("#")][0]
    c, nd, pr = (int(x) for x in line.split())
    inst = I.full_dual_n11(0)
    g = W.enumerate_batch([W.BatchSpec("dual", 11, 15, inst.cols, cap=-2)], list_mode=False,
                          tuning={"search": search})[0]
    assert (g.count, g.nodes, g.probes) == (c, nd, pr)


# ---------------------------------------------------------------------------------------
# the batched workload's own n = 7 and n = 8 maps on the per-thread kernel the bench times
# ---------------------------------------------------------------------------------------

def _oracle_lists(args):
    import oracle as O2
    kind, n, m, cols = args
    f = O2.candidate_facets(kind, n, m, cols)
    return O2.enumerate_dfs(n, m, f, cap=O2.CAP_UBT, capacity=1 << 18)


def test_batched_workload_n7_n8_lists_on_per_thread_searches(W):
    """The first 8 maps of n = 7 and of n = 8 of the 4096-map benchmark batch (seed 0), in
    one list-mode batch on per-thread searches: the kernel class of n <= 8 with rows of 8
    (the class the benchmark's tuned run uses). Sorted masks, counts, nodes and probes
    against the oracle, map by map (the oracle runs in a spawn pool)."""
    import multiprocessing as mp
    allm = I.batch_duals(4096, 3, 8, seed=0)
    maps = [i for i in allm if i.n == 7][:8] + [i for i in allm if i.n == 8][:8]
    with mp.get_context("spawn").Pool(min(16, len(maps))) as pool:
        want = pool.map(_oracle_lists, [(i.kind, i.n, i.m, list(i.cols)) for i in maps])
    specs = [W.BatchSpec(i.kind, i.n, i.m, i.cols, cap=W.CAP_UBT) for i in maps]
    res = W.enumerate_batch(specs, list_mode=True, capacities=[w[0] for w in want],
                            tuning={"search": 1})
    st = W.last_run_stats()
    assert st["search"] == 1 and st["size_class"] == 4
    for r, w, i in zip(res, want, maps):
        assert r.status == 0
        assert (r.count, r.nodes, r.probes) == tuple(w[:3]), i.label
        assert np.array_equal(r.masks, w[3])


def test_n10_batch_default_is_per_thread_and_exact(W):
    """16 maps of n = 10 (616 candidate facets each) with no tuning: a batch this size of the
    n = 10 class runs one search per thread by default. Count, nodes and probes of every map
    against the oracle's stored results (tests/golden/n10_batch.txt, written by
    make_n10_batch.py), and the per-warp search gives the same."""
    rows = load_table("n10_batch.txt")
    assert [r[0] for r in rows] == list(range(16))
    specs = [W.BatchSpec("dual", 10, 14, I.single_dual(10, s).cols, cap=W.CAP_UBT)
             for s, _, _, _ in rows]
    for tuning, search in ((None, 1), ({"search": 2}, 2)):
        res = W.enumerate_batch(specs, list_mode=False, tuning=tuning)
        st = W.last_run_stats()
        assert st["search"] == search and st["size_class"] == 6
        for r, (s, c, nd, pr) in zip(res, rows):
            assert r.status == 0
            assert (r.count, r.nodes, r.probes) == (c, nd, pr), s


@pytest.mark.parametrize("n_hi,chunk", [(4, 3), (6, 4099), (6, 100003)],
                         ids=["n3_4_chunk3", "n3_6_chunk4099", "n3_6_chunk100003"])
def test_host_lists_through_small_staging_chunks(W, n_hi, chunk):
    """Host outputs leave the device chunk by chunk through two page-locked halves of a
    staging buffer. Chunks much smaller than the lists (a list then spans many chunks, a
    chunk holds parts of several lists, and with 3 words a mask can straddle two chunks) give
    the oracle's sorted lists, counts, nodes and probes."""
    insts = I.batch_duals(24, 3, n_hi, seed=7)
    orc = [oracle_run(inst, cap=-2)[1] for inst in insts]
    specs = [W.BatchSpec("dual", i.n, i.m, i.cols, cap=-2) for i in insts]
    res = W.enumerate_batch(specs, list_mode=True, capacities=[o[0] + 1 for o in orc],
                            tuning={"stage_chunk_words": chunk})
    for g, o in zip(res, orc):
        assert g.status == 0
        assert_same(g, o)
