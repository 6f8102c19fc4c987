"""Host logic of the serving loop and of the serving workload, on CPU: the Poisson stream,
the latency statistics, and the request loop against a stand-in engine (resubmission on a
capacity error, completion, latency bookkeeping)."""
import math

import numpy as np

from paper_2301_00806_gb300 import instances as I, serving


def _rank2(rows):
    """GF(2) rank of 4-bit row vectors."""
    rows = list(rows)
    r = 0
    for bit in range(4):
        piv = next((i for i in range(r, len(rows)) if (rows[i] >> bit) & 1), None)
        if piv is None:
            continue
        rows[r], rows[piv] = rows[piv], rows[r]
        for i in range(len(rows)):
            if i != r and (rows[i] >> bit) & 1:
                rows[i] ^= rows[r]
        r += 1
    return r


def test_poisson_stream():
    jobs = I.poisson_jobs(rate=200, duration=60, n_lo=5, n_hi=9, seed=0)
    t = [j.extra["t_arrival"] for j in jobs]
    assert all(0 < a < b for a, b in zip(t, t[1:])) and t[-1] < 60
    assert abs(len(jobs) - 12000) < 5 * math.sqrt(12000)     # Poisson count
    gaps = np.diff([0.0] + t)
    assert abs(gaps.mean() - 1 / 200) < 0.1 / 200             # exponential gaps, mean 1/rate
    assert {j.n for j in jobs} == {5, 6, 7, 8, 9}
    for j in jobs[:500]:
        assert j.m == j.n + 4 and len(set(j.cols)) == j.m and 0 not in j.cols
        assert _rank2(j.cols) == 4
    again = I.poisson_jobs(rate=200, duration=60, n_lo=5, n_hi=9, seed=0)
    assert [j.cols for j in again] == [j.cols for j in jobs]  # seeded


def test_latency_statistics():
    st = serving.ServeStats(jobs=5, completed=5, wall_s=2.0, nodes=100,
                            latencies_ms=[5.0, 1.0, 3.0, 2.0, 4.0])
    assert st.percentile(50) == 3.0 and st.percentile(0) == 1.0 and st.percentile(100) == 5.0
    s = st.summary()
    assert s["p50_ms"] == 3.0 and s["mean_ms"] == 3.0
    assert s["jobs_per_s"] == 2.5 and s["nodes_per_s"] == 50.0
    assert serving.ServeStats().percentile(99) is None


class _FakeResult:
    def __init__(self, status, count, nodes):
        self.status, self.count, self.nodes = status, count, nodes


class _FakeEngine:
    """Finishes every job at the next step; a job's first result is a capacity error when
    it asked for fewer masks than it has."""

    def __init__(self, **kw):
        self.next = 1
        self.running, self.done, self.cap = [], [], {}
        self.steps = 0
        self.closed = False

    def submit(self, kind, n, m, cols, cap=None, list_mode=True, capacity=0):
        jid = self.next
        self.next += 1
        self.cap[jid] = capacity
        self.running.append(jid)
        return jid

    def step(self):
        self.steps += 1
        self.done += self.running
        n = len(self.running)
        self.running = []
        return n

    def poll(self):
        d, self.done = self.done, []
        return d

    def result(self, jid, capacity=0):
        need = 7
        if self.cap[jid] < need:
            return _FakeResult(serving.wpm.ERR_CAPACITY, need, 0)
        return _FakeResult(serving.wpm.OK, need, 1000)

    def close(self):
        self.closed = True


def test_request_loop_against_a_stand_in_engine(monkeypatch):
    made = []

    def factory(**kw):
        e = _FakeEngine(**kw)
        made.append(e)
        return e

    monkeypatch.setattr(serving.wpm, "Engine", factory)
    jobs = I.poisson_jobs(rate=2000, duration=0.02, n_lo=5, n_hi=6, seed=1)
    assert len(jobs) >= 10
    st = serving.serve(jobs, capacity={5: 3, 6: 100})   # n = 5 jobs are resubmitted
    n5 = sum(j.n == 5 for j in jobs)
    assert st.completed == len(jobs) and st.failed == 0
    assert st.resubmitted == n5
    assert st.nodes == 1000 * len(jobs)
    assert len(st.latencies_ms) == len(jobs) and min(st.latencies_ms) >= 0.0
    assert made and made[0].closed
