"""GPU: the serving engine (continuous batching). A job's result is the same whether it runs
alone (wpm_enumerate) or among other jobs submitted while it is on the device."""
import numpy as np
import pytest

import oracle as O
from paper_2301_00806_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2301_00806_gb300 import wpm
    wpm.lib()
    return wpm


def _drain(E, want):
    got = {}
    for _ in range(100000):
        E.step()
        for j in E.poll():
            got[j] = E.result(j)
        if len(got) >= want:
            break
    return got


@pytest.mark.parametrize("max_n,budget", [(6, 512), (9, 512), (9, 0)],
                         ids=["n6", "n9", "n9_default_budget"])
def test_jobs_alone_and_in_the_mix_agree(W, max_n, budget):
    jobs = I.poisson_jobs(rate=200.0, duration=0.2, n_lo=5, n_hi=max_n, seed=3)
    assert len(jobs) >= 20
    alone = [W.enumerate("dual", j.n, j.m, j.cols, cap=-2, capacity=1 << 17) for j in jobs]
    E = W.Engine(max_n=max_n, max_jobs=16, budget=budget, memory_bytes=1 << 30)
    ids = []
    got = {}
    # submit in arrival order, stepping between arrivals so that jobs join a running mix
    for k, j in enumerate(jobs):
        ids.append(E.submit("dual", j.n, j.m, j.cols, cap=-2, list_mode=True,
                            capacity=alone[k].count + 1))
        if k % 3 == 2:
            E.step()
            for jid in E.poll():
                got[jid] = E.result(jid)
    got.update(_drain(E, len(jobs) - len(got)))
    assert set(got) == set(ids)
    for jid, a in zip(ids, alone):
        g = got[jid]
        assert g.status == 0
        assert (g.count, g.nodes, g.probes) == (a.count, a.nodes, a.probes)
        assert np.array_equal(g.masks, a.masks)
    E.close()
    if max_n == 9 and budget:
        # and against the oracle: the first n = 7 and n = 8 jobs and the smallest n = 9 job of
        # the mix (the oracle in a spawn pool)
        import multiprocessing as mp
        pick = [next(k for k, j in enumerate(jobs) if j.n == 7),
                next(k for k, j in enumerate(jobs) if j.n == 8),
                min((k for k, j in enumerate(jobs) if j.n == 9), key=lambda k: alone[k].nodes)]
        with mp.get_context("spawn").Pool(len(pick)) as pool:
            want = pool.map(_oracle_job, [(jobs[k].n, list(jobs[k].cols)) for k in pick])
        for k, w in zip(pick, want):
            g = got[ids[k]]
            assert (g.count, g.nodes, g.probes) == tuple(w[:3]), jobs[k].n
            assert np.array_equal(g.masks, w[3])


def _oracle_job(args):
    import oracle as O2
    n, cols = args
    f = O2.candidate_facets("dual", n, n + 4, cols)
    return O2.enumerate_dfs(n, n + 4, f, cap=O2.CAP_UBT, capacity=1 << 18)


def test_engine_matches_oracle_with_properties(W):
    E = W.Engine(max_n=6, max_jobs=4, budget=64, memory_bytes=1 << 28)
    cases = []
    for s in range(6):
        inst = I.single_dual(5, 40 + s)
        f = O.instance_facets(inst)
        fo = np.zeros((f.size + 63) // 64, dtype=np.uint64)
        fo[0] = np.uint64(1 << s)
        kw = dict(cap=-2, base_facet=(s % 2 == 0), forced_out=fo)
        jid = E.submit("dual", 5, 9, inst.cols, list_mode=True, capacity=1 << 14,
                       n_facets=f.size, **kw)
        cases.append((jid, O.enumerate_dfs(5, 9, f, capacity=1 << 14, **kw)))
    got = _drain(E, len(cases))
    for jid, (c, nd, pr, masks) in cases:
        g = got[jid]
        assert (g.count, g.nodes, g.probes) == (c, nd, pr)
        assert np.array_equal(g.masks, masks)
    E.close()


def test_engine_capacity_and_limits(W):
    E = W.Engine(max_n=5, max_jobs=2, budget=256, memory_bytes=1 << 26)
    inst = I.single_dual(5, 1)
    small = E.submit("dual", 5, 9, inst.cols, cap=-2, list_mode=True, capacity=10)
    big = E.submit("dual", 8, 12, I.single_dual(8, 0).cols, cap=-2)
    got = _drain(E, 2)
    assert got[small].status == W.ERR_CAPACITY and got[small].count > 10
    assert got[big].status == W.ERR_LIMIT
    E.close()


def test_engine_refuses_post_filters(W):
    E = W.Engine(max_n=5, max_jobs=2, budget=256, memory_bytes=1 << 26)
    inst = I.single_dual(5, 2)
    with pytest.raises(W.WpmError) as e:
        E.submit("dual", 5, 9, inst.cols, cap=-2, list_mode=True, capacity=1 << 12,
                 post_filter=W.POST_SEED)
    assert e.value.code == W.ERR_INPUT
    E.close()
