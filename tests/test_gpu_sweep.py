"""GPU parity of the GF(2) cycle-space sweep engine (Section 2.1): every element of ker_Z2 A
in Gray-code order, kept when every ridge has degree 0 or 2 (Proposition 2.1) and the
properties hold. Same counts and sorted lists as the oracle; `nodes` counts the 2^s kernel
elements visited (s = dim ker_Z2 A, from the oracle's elimination)."""
import numpy as np
import pytest

from paper_2301_00806_gb300 import instances as I
from oracle import oracle as O

pytestmark = pytest.mark.gpu

SWEEP = {"engine": 1}


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2301_00806_gb300 import wpm
    wpm.lib()
    return wpm


def sweep_one(W, kind, n, m, cols, capacity=1 << 15, **kw):
    spec = W.BatchSpec(kind, n, m, cols, **kw)
    return W.enumerate_batch([spec], list_mode=True, capacities=[capacity], tuning=SWEEP)[0]


def check(g, orc, f, n):
    c, _, _, masks = orc
    assert g.status == 0
    assert g.count == c
    assert np.array_equal(g.masks, masks)
    assert g.nodes == 1 << O.kernel_dim(n, f)
    assert g.probes == 0


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("cap", [-1, -2])
def test_fano_sweep(W, seed, cap):
    inst = I.fano_primal(seed)
    f = O.instance_facets(inst)
    orc = O.enumerate_dfs(3, 7, f, cap=cap, capacity=1 << 12)
    assert orc[0] == (1303 if cap == -1 else 666)
    check(sweep_one(W, "primal", 3, 7, inst.cols, cap=cap), orc, f, 3)


@pytest.mark.parametrize("seed", range(6))
def test_n5_sweep(W, seed):
    inst = I.single_dual(5, seed)
    f = O.instance_facets(inst)
    orc = O.enumerate_dfs(5, 9, f, cap=-2, capacity=1 << 15)
    check(sweep_one(W, "dual", 5, 9, inst.cols, cap=-2), orc, f, 5)


def test_mixed_batch_sweep_equals_search(W):
    insts = I.batch_duals(40, 2, 5, seed=21)
    specs = [W.BatchSpec("dual", i.n, i.m, i.cols, cap=-2) for i in insts]
    caps = [1 << 14] * len(specs)
    sw = W.enumerate_batch(specs, list_mode=True, capacities=caps, tuning=SWEEP)
    se = W.enumerate_batch(specs, list_mode=True, capacities=caps)
    for a, b, inst in zip(sw, se, insts):
        assert a.status == 0 and b.status == 0
        assert a.count == b.count
        assert np.array_equal(a.masks, b.masks)
        f = O.instance_facets(inst)
        assert a.nodes == 1 << O.kernel_dim(inst.n, f)


@pytest.mark.parametrize("seed", range(12))
def test_sweep_properties(W, seed):
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
    orc = O.enumerate_dfs(n, n + 4, f, capacity=1 << 15, **kw)
    g = sweep_one(W, "dual", n, n + 4, inst.cols, n_facets=M, **kw)
    check(g, orc, f, n)


def test_table2_n4_sweep(W):
    """Table 2's first row at n = 4 (20383) by the sweep, one map per IDCM orbit."""
    reps = I.idcm_orbit_reps(4)
    specs = [W.BatchSpec("dual", 4, 8, r, cap=-2, base_facet=True) for r in reps]
    res = W.enumerate_batch(specs, list_mode=False, tuning=SWEEP)
    assert sum(r.count for r in res) == 20383


def test_sweep_limits(W):
    big = I.single_dual(8, 3)  # M > 256 candidate facets
    f = O.instance_facets(big)
    assert f.size > 256
    with pytest.raises(W.WpmError) as e:
        sweep_one(W, "dual", 8, 12, big.cols, cap=-2)
    assert e.value.code == W.ERR_LIMIT
    inst = I.single_dual(5, 0)
    s = O.kernel_dim(5, O.instance_facets(inst))
    spec = W.BatchSpec("dual", 5, 9, inst.cols, cap=-2)
    with pytest.raises(W.WpmError) as e:
        W.enumerate_batch([spec], list_mode=False, tuning={"engine": 1, "sweep_max_s": s - 1})
    assert e.value.code == W.ERR_LIMIT
