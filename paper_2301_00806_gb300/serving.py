"""A request loop over the serving engine: jobs arrive on their own clock, are submitted when
they arrive, and are admitted by the engine as device memory and slots free up; the loop keeps
stepping the engine (one search pass over everything resident per step) and collects finished
jobs. Latency = completion time - arrival time.

Used by bench.py for the serving workload; usable on its own:

    from paper_2301_00806_gb300 import instances as I, serving
    stats = serving.serve(I.poisson_jobs(rate=200, duration=60, n_lo=5, n_hi=9))
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

from . import wpm

# Output capacity requested per job (masks), by n: about twice the largest count seen on the
# seeded maps of that size; a job that needs more is resubmitted with its exact count.
DEFAULT_CAPACITY = {2: 64, 3: 2048, 4: 8192, 5: 32768, 6: 131072, 7: 262144, 8: 393216,
                    9: 524288, 10: 524288, 11: 524288}


@dataclass
class ServeStats:
    jobs: int = 0
    completed: int = 0
    resubmitted: int = 0
    failed: int = 0
    wall_s: float = 0.0
    nodes: int = 0
    latencies_ms: List[float] = field(default_factory=list)
    steps: int = 0
    max_active: int = 0

    def percentile(self, q: float) -> Optional[float]:
        if not self.latencies_ms:
            return None
        xs = sorted(self.latencies_ms)
        k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
        return xs[k]

    def summary(self) -> dict:
        return {"jobs": self.jobs, "completed": self.completed, "failed": self.failed,
                "resubmitted": self.resubmitted, "wall_s": self.wall_s,
                "p50_ms": self.percentile(50), "p99_ms": self.percentile(99),
                "mean_ms": (sum(self.latencies_ms) / len(self.latencies_ms)
                            if self.latencies_ms else None),
                "jobs_per_s": self.completed / self.wall_s if self.wall_s else None,
                "nodes_per_s": self.nodes / self.wall_s if self.wall_s else None,
                "engine_steps": self.steps, "max_active_jobs": self.max_active}


def serve(jobs, list_mode: bool = True, max_n: int = 9, max_jobs: int = 1024,
          budget: int = 1 << 20, memory_bytes: int = 64 << 30, capacity: Dict[int, int] = None,
          stream=None, deadline_s: float = 0.0, log=None, slice_ms: int = 0) -> ServeStats:
    """Serve `jobs` (instances with extra['t_arrival'] in seconds) in real time. With
    deadline_s > 0 the loop gives up after that many seconds (unfinished jobs are left out of
    the statistics); `log` (a callable) receives a progress line about every second."""
    capacity = capacity or DEFAULT_CAPACITY
    E = wpm.Engine(memory_bytes=memory_bytes, max_jobs=max_jobs, budget=budget, max_n=max_n,
                   stream=stream, slice_ms=slice_ms)
    st = ServeStats(jobs=len(jobs))
    arrival = {}
    meta = {}
    order = sorted(range(len(jobs)), key=lambda k: jobs[k].extra["t_arrival"])
    nxt = 0
    t0 = time.perf_counter()
    last_log = 0.0
    try:
        while st.completed + st.failed < len(jobs):
            now = time.perf_counter() - t0
            if deadline_s and now > deadline_s:
                break
            if log and now - last_log >= 1.0:
                last_log = now
                log(f"t={now:.1f}s submitted={nxt} completed={st.completed} "
                    f"steps={st.steps} active={st.max_active}")
            while nxt < len(order) and jobs[order[nxt]].extra["t_arrival"] <= now:
                j = jobs[order[nxt]]
                jid = E.submit(j.kind, j.n, j.m, j.cols, cap=wpm.CAP_UBT, list_mode=list_mode,
                               capacity=capacity.get(j.n, 1 << 16) if list_mode else 0)
                arrival[jid] = j.extra["t_arrival"]
                meta[jid] = j
                nxt += 1
            active = E.step()
            st.steps += 1
            st.max_active = max(st.max_active, active)
            for jid in E.poll():
                r = E.result(jid)
                if r.status == wpm.ERR_CAPACITY:  # resubmit with the exact size, same arrival
                    j = meta[jid]
                    nj = E.submit(j.kind, j.n, j.m, j.cols, cap=wpm.CAP_UBT, list_mode=True,
                                  capacity=r.count)
                    arrival[nj] = arrival[jid]
                    meta[nj] = j
                    st.resubmitted += 1
                    continue
                done_t = time.perf_counter() - t0
                if r.status == wpm.OK:
                    st.completed += 1
                    st.nodes += r.nodes
                    st.latencies_ms.append(1000.0 * (done_t - arrival[jid]))
                else:
                    st.failed += 1
            if active == 0 and nxt < len(order):
                wait = jobs[order[nxt]].extra["t_arrival"] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        st.wall_s = time.perf_counter() - t0
    finally:
        E.close()
    return st
