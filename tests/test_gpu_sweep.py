"""GPU parity of the GF(2) cycle-space sweep engines (Section 2.1; Section 4.4's fixed
coordinates). Engine 1 sweeps the convenient basis: forced rows fix coordinates, Z blocks
allow at most two generators each (within Hamming distance 2 of the fixed part), the other
generators are free; `nodes` counts the combinations visited, |X|, which must equal the
oracle's route over the same basis (orc_enumerate_sweep_blocks; |X| depends only on the
block sizes, which the kernel's span fixes). Engine 2 sweeps all 2^s elements of ker_Z2 A.
Both give the same counts and sorted lists as the oracle's search."""
import numpy as np
import pytest

from conftest import load_n11_seeds
from oracle import oracle as O
from paper_2301_00806_gb300 import instances as I

pytestmark = pytest.mark.gpu

BLOCKS = {"engine": 1}
PLAIN = {"engine": 2}


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2301_00806_gb300 import wpm
    wpm.lib()
    return wpm


def sweep_one(W, kind, n, m, cols, tuning, capacity=1 << 15, **kw):
    spec = W.BatchSpec(kind, n, m, cols, **kw)
    return W.enumerate_batch([spec], list_mode=True, capacities=[capacity], tuning=tuning)[0]


def _okw(kw):
    """The batch spec's properties in the oracle's argument names."""
    return {k: v for k, v in kw.items() if k != "n_facets"}


def check(g, n, m, f, tuning, **kw):
    orc = O.enumerate_dfs(n, m, f, capacity=1 << 15, **_okw(kw))
    assert g.status == 0
    assert g.count == orc[0]
    assert np.array_equal(g.masks, orc[3])
    if tuning is PLAIN:
        assert g.nodes == 1 << O.kernel_dim(n, f)
    else:
        blk = O.enumerate_sweep_blocks(n, m, f, capacity=1 << 15, max_log2_x=48, **_okw(kw))
        assert g.nodes == blk[1]
        assert g.nodes <= 1 << O.kernel_dim(n, f)
    assert g.probes == 0


@pytest.mark.parametrize("tuning", [BLOCKS, PLAIN], ids=["blocks", "plain"])
@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("cap", [-1, -2])
def test_fano_sweep(W, tuning, seed, cap):
    inst = I.fano_primal(seed)
    f = O.instance_facets(inst)
    g = sweep_one(W, "primal", 3, 7, inst.cols, tuning, cap=cap)
    assert g.count == (1303 if cap == -1 else 666)
    check(g, 3, 7, f, tuning, cap=cap)


@pytest.mark.parametrize("tuning", [BLOCKS, PLAIN], ids=["blocks", "plain"])
@pytest.mark.parametrize("seed", range(6))
def test_n5_sweep(W, tuning, seed):
    inst = I.single_dual(5, seed)
    f = O.instance_facets(inst)
    check(sweep_one(W, "dual", 5, 9, inst.cols, tuning, cap=-2), 5, 9, f, tuning, cap=-2)


@pytest.mark.parametrize("tuning", [BLOCKS, PLAIN], ids=["blocks", "plain"])
def test_mixed_batch_sweep_equals_search(W, tuning):
    insts = I.batch_duals(40, 2, 5, seed=21)
    specs = [W.BatchSpec("dual", i.n, i.m, i.cols, cap=-2) for i in insts]
    caps = [1 << 14] * len(specs)
    sw = W.enumerate_batch(specs, list_mode=True, capacities=caps, tuning=tuning)
    se = W.enumerate_batch(specs, list_mode=True, capacities=caps)
    for a, b, inst in zip(sw, se, insts):
        assert a.status == 0 and b.status == 0
        assert a.count == b.count
        assert np.array_equal(a.masks, b.masks)
        f = O.instance_facets(inst)
        if tuning is PLAIN:
            assert a.nodes == 1 << O.kernel_dim(inst.n, f)
        else:
            assert a.nodes == O.enumerate_sweep_blocks(inst.n, inst.m, f, cap=-2,
                                                       capacity=1 << 14)[1]


@pytest.mark.parametrize("tuning", [BLOCKS, PLAIN], ids=["blocks", "plain"])
@pytest.mark.parametrize("seed", range(12))
def test_sweep_properties(W, tuning, seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(3, 6))
    inst = I.single_dual(n, 40 + seed)
    f = O.instance_facets(inst)
    M = f.size
    words = (M + 63) // 64
    kw = {"cap": int(rng.choice([-1, -2, int(rng.integers(3, 40))]))}
    if seed % 3 == 0:
        fi = np.zeros(words, dtype=np.uint64)
        j = int(rng.integers(0, M))
        fi[j // 64] |= np.uint64(1) << np.uint64(j % 64)
        kw["forced_in"] = fi
    if seed % 4 == 1:
        fo = np.zeros(words, dtype=np.uint64)
        for j in rng.choice(M, size=min(M, 6), replace=False):
            fo[j // 64] |= np.uint64(1) << np.uint64(int(j) % 64)
        kw["forced_out"] = fo
    if seed % 2 == 1:
        kw["affine"] = [(int(rng.integers(0, 30)), rng.integers(-2, 3, size=M).tolist())
                        for _ in range(int(rng.integers(1, 4)))]
    if seed % 5 == 2:
        kw["base_facet"] = True
    g = sweep_one(W, "dual", n, n + 4, inst.cols, tuning, n_facets=M, **kw)
    check(g, n, n + 4, f, tuning, **kw)


def test_table2_n4_sweep(W):
    """Table 2's first row at n = 4 (20383) by the convenient-basis sweep, one map per IDCM
    orbit, the base facet fixing one coordinate."""
    reps = I.idcm_orbit_reps(4)
    specs = [W.BatchSpec("dual", 4, 8, r, cap=-2, base_facet=True) for r in reps]
    res = W.enumerate_batch(specs, list_mode=False, tuning=BLOCKS)
    assert sum(r.count for r in res) == 20383


def _mask_bits(words, count):
    return [j for j in range(count) if (int(words[j // 64]) >> (j % 64)) & 1]


def test_section_4_4_links_through_the_sweep(W):
    """Section 4.4's route on the GPU: the 16 stored n = 11 sample links, conditions (1) and
    (2) as forced sets, fix 56 of the 64 kernel coordinates; the sweep over the rest gives the
    stored counts and, mask for mask, the oracle's lists."""
    _, _, samples = load_n11_seeds()
    specs, want = [], []
    for orbit, words, count, nodes, probes, kept in samples:
        rep = I.idcm_orbit_reps(10)[orbit]
        f10 = O.candidate_facets("dual", 10, 14, rep)
        L = [int(f10[j]) for j in _mask_bits(words, len(f10))]
        lam, f, fin, fout = O.link_conditions(11, 15, rep, L)
        specs.append(W.BatchSpec("dual", 11, 15, lam, cap=-2, forced_in=fin, forced_out=fout,
                                 n_facets=f.size))
        blk = O.enumerate_sweep_blocks(11, 15, f, cap=O.CAP_UBT, forced_in=fin, forced_out=fout,
                                       capacity=64)
        assert blk[0] == count
        want.append(blk)
    assert len(specs) == 16
    res = W.enumerate_batch(specs, list_mode=True, capacities=[64] * len(specs), tuning=BLOCKS)
    for r, w in zip(res, want):
        assert r.status == 0
        assert (r.count, r.nodes) == (w[0], w[1])
        assert np.array_equal(r.masks, w[3])


def test_sweep_limits(W):
    inst = I.single_dual(5, 0)
    f = O.instance_facets(inst)
    s = O.kernel_dim(5, f)
    spec = W.BatchSpec("dual", 5, 9, inst.cols, cap=-2)
    with pytest.raises(W.WpmError) as e:
        W.enumerate_batch([spec], list_mode=False, tuning={"engine": 2, "sweep_max_s": s - 1})
    assert e.value.code == W.ERR_LIMIT
    lx = O.convenient_basis(5, 9, f)["log2_x"]
    with pytest.raises(W.WpmError) as e:
        W.enumerate_batch([spec], list_mode=False,
                          tuning={"engine": 1, "sweep_max_s": int(lx) - 1})
    assert e.value.code == W.ERR_LIMIT
    big = I.full_dual_n11(0)   # s = 64, |X| about 2^55 even with blocks
    with pytest.raises(W.WpmError) as e:
        W.enumerate_batch([W.BatchSpec("dual", 11, 15, big.cols, cap=-2)], list_mode=False,
                          tuning=BLOCKS)
    assert e.value.code == W.ERR_LIMIT
