"""Failure paths that can be made to happen without faulting a GPU.

Every device wait of the search passes is bounded: a wait that runs out sets an error bit
and the kernel returns, so the host reads a status and the context stays usable. The tests
make each bound run out on purpose through the C ABI's tuning fields (a wall-time limit, a
ready flag that no writer raises, a one-step idle bound) and check the reported status, the
partial counts against the oracle's, and that the next call still gives exact results. The
serving engine's admission check is tested by a job that could never fit in its memory.
"""
import os

import numpy as np
import pytest

import oracle as O
from conftest import GOLDEN
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


def _fano_still_exact(W):
    inst = I.fano_primal(2)
    g = W.enumerate("primal", 3, 7, inst.cols, cap=W.CAP_UBT)
    c, nodes, probes, masks = O.enumerate_dfs(3, 7, O.instance_facets(inst), cap=O.CAP_UBT)
    assert (g.count, g.nodes, g.probes) == (c, nodes, probes)
    assert np.array_equal(g.masks, masks)


def _n11_full():
    line = [ln for ln in open(os.path.join(GOLDEN, "n11_full.txt")) if not ln.startswith("#")][0]
    return tuple(int(x) for x in line.split())


@pytest.mark.parametrize("search", [1, 2], ids=["thread", "warp"])
def test_time_limit_reports_timeout_with_partial_counts(W, search):
    """The whole n = 11 map takes far longer than 5 ms: the run stops at the limit and the
    map reports WPM_ERR_TIMEOUT with counts that are a part of the oracle's stored totals."""
    c, nd, pr = _n11_full()
    inst = I.full_dual_n11(0)
    g = W.enumerate_batch([W.BatchSpec("dual", 11, 15, inst.cols, cap=W.CAP_UBT)],
                          list_mode=False, tuning={"search": search, "time_limit_ms": 5})[0]
    assert g.status == W.ERR_TIMEOUT
    assert g.count <= c and 0 < g.nodes < nd and g.probes <= pr
    _fano_still_exact(W)


def test_ready_flag_wait_runs_out_and_the_kernel_returns(W):
    """Items handed over inside a per-thread pass are read only once their ready flag is
    raised. With the test hook, readers wait for a stamp that no writer raises: each such
    wait gives up after ready_polls polls, the pass returns, and the run reports
    WPM_ERR_TIMEOUT. Two n = 6 maps on some 100,000 per-thread searches leave most searches
    waiting (a frontier of 16 items), so busy ones hand work over at every chance
    (donate_every = 1)."""
    maps = [I.single_dual(6, 20), I.single_dual(6, 21)]
    specs = [W.BatchSpec("dual", 6, 10, i.cols, cap=W.CAP_UBT) for i in maps]
    tuning = {"search": 1, "frontier_target": 16, "donate_every": 1, "donate_levels": 4,
              "ready_polls": 64, "test_unpublished": 1, "graph": -1}
    res = W.enumerate_batch(specs, list_mode=False, tuning=tuning)
    # the run as a whole failed: every map carries the status, the message says why
    assert all(r.status == W.ERR_TIMEOUT for r in res)
    assert b"bounded wait" in W.lib().wpm_last_error()
    # the same run without the hook, with the default bound (64 polls can also run out in a
    # correct run, before a writer publishes), is exact, and so is an unrelated call after it
    res = W.enumerate_batch(specs, list_mode=False,
                            tuning=dict(tuning, test_unpublished=0, ready_polls=0))
    for r, i in zip(res, maps):
        want = O.enumerate_dfs(i.n, i.m, O.instance_facets(i), cap=O.CAP_UBT, list_mode=False)
        assert (r.count, r.nodes, r.probes) == tuple(want[:3])
    _fano_still_exact(W)


@pytest.mark.parametrize("idle_polls", [1, 7])
def test_waiting_searches_that_leave_early_change_no_count(W, idle_polls):
    """A waiting search leaves its pass after idle_polls fruitless steps; the work it would
    have taken stays in the ring for the next pass, so counts are unchanged."""
    maps = I.batch_duals(24, 4, 6, seed=5)
    specs = [W.BatchSpec("dual", i.n, i.m, i.cols, cap=W.CAP_UBT) for i in maps]
    res = W.enumerate_batch(specs, list_mode=True, capacities=[1 << 16] * len(specs),
                            tuning={"search": 1, "idle_polls": idle_polls})
    for r, i in zip(res, maps):
        c, nodes, probes, masks = O.enumerate_dfs(i.n, i.m, O.instance_facets(i),
                                                  cap=O.CAP_UBT, capacity=1 << 16)
        assert r.status == 0
        assert (r.count, r.nodes, r.probes) == (c, nodes, probes)
        assert np.array_equal(r.masks, masks)


def test_engine_refuses_a_job_larger_than_its_memory(W):
    """A list-mode job whose output region exceeds the engine's whole output memory could
    never be admitted; submit refuses it with WPM_ERR_NOMEM and later jobs are served."""
    eng = W.Engine(memory_bytes=1 << 20, max_jobs=8, max_n=6)
    try:
        big = I.single_dual(5, 3)
        with pytest.raises(W.WpmError) as e:
            eng.submit("dual", 5, 9, big.cols, cap=W.CAP_UBT, list_mode=True,
                       capacity=1 << 20)
        assert e.value.code == W.ERR_NOMEM
        small = I.single_dual(5, 4)
        jid = eng.submit("dual", 5, 9, small.cols, cap=W.CAP_UBT, list_mode=True,
                         capacity=1 << 14)
        done = []
        for _ in range(10000):
            eng.step()
            done += eng.poll()
            if jid in done:
                break
        assert jid in done
        r = eng.result(jid)
        c, nodes, probes, masks = O.enumerate_dfs(5, 9, O.instance_facets(small),
                                                  cap=O.CAP_UBT, capacity=1 << 14)
        assert r.status == W.OK and (r.count, r.nodes, r.probes) == (c, nodes, probes)
        assert np.array_equal(r.masks, masks)
    finally:
        eng.close()
