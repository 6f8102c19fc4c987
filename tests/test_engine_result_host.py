"""The Python binding of wpm_engine_result (wpm.Engine.result), checked on the CPU against a
stand-in for the C call that follows its documented contract: a finished list-mode job whose
buffer is too small (or absent) reports WPM_ERR_CAPACITY with its count and stays available;
a large enough buffer receives the masks and the job is released; a job that failed reports
its own status. The binding must ask for the count first and then fill an array of exactly
that size, return an empty (0, W) array for an empty list, and pass a job's failure through.
The engine itself is tested on the GPU in test_gpu_serving.py."""
import ctypes as C

import numpy as np
import pytest

from paper_2301_00806_gb300 import wpm


class _Job:
    def __init__(self, masks, status=wpm.OK, list_mode=True):
        self.masks = np.ascontiguousarray(masks, dtype=np.uint64)
        self.status = status
        self.list_mode = list_mode


class _FakeLib:
    """wpm_engine_result and wpm_engine_destroy as wpm_engine.cpp implements them."""

    def __init__(self, jobs):
        self.jobs = jobs
        self.calls = []  # (job id, capacity offered, buffer given)

    def wpm_engine_result(self, h, job_id, out_ref):
        o = out_ref._obj
        job = self.jobs.get(int(job_id))
        self.calls.append((int(job_id), int(o.capacity), bool(o.masks)))
        if job is None:
            return wpm.ERR_INPUT
        count, w = job.masks.shape
        o.count = count
        o.found = count
        o.nodes = 10 * count + 1
        o.probes = 3
        o.words_per_mask = w
        o.M = 64 * w
        o.N = 7
        o.status = job.status
        rc = job.status
        if rc == wpm.OK and job.list_mode:
            if o.capacity < count or (count and not o.masks):
                return wpm.ERR_CAPACITY  # the result stays available
            if count:
                C.memmove(o.masks, job.masks.ctypes.data, job.masks.nbytes)
        del self.jobs[int(job_id)]
        return rc

    def wpm_engine_destroy(self, h):
        pass


@pytest.fixture
def engine(monkeypatch):
    def make(jobs):
        fake = _FakeLib(jobs)
        monkeypatch.setattr(wpm, "lib", lambda: fake)
        E = wpm.Engine.__new__(wpm.Engine)
        E._h = C.c_void_p(1)
        E._modes = {jid: job.list_mode for jid, job in jobs.items()}
        return E, fake
    return make


def test_list_is_fetched_into_an_array_of_exactly_its_size(engine):
    masks = np.arange(3 * 5, dtype=np.uint64).reshape(5, 3) * 0x100000001
    E, fake = engine({7: _Job(masks)})
    r = E.result(7)
    assert r.status == wpm.OK and r.count == 5 and r.words == 3 and r.nodes == 51
    assert r.masks.shape == (5, 3) and np.array_equal(r.masks, masks)
    # first the count (no buffer), then exactly that many masks
    assert fake.calls == [(7, 0, False), (7, 5, True)]
    assert 7 not in fake.jobs and 7 not in E._modes


def test_empty_list_gives_an_empty_array(engine):
    E, fake = engine({3: _Job(np.zeros((0, 2), dtype=np.uint64))})
    r = E.result(3)
    assert r.status == wpm.OK and r.count == 0
    assert r.masks.shape == (0, 2)
    assert fake.calls == [(3, 0, False)]


def test_failed_job_passes_its_status_through(engine):
    E, fake = engine({9: _Job(np.zeros((4, 1), dtype=np.uint64), status=wpm.ERR_CAPACITY)})
    r = E.result(9)
    assert r.status == wpm.ERR_CAPACITY and r.masks is None and r.count == 4
    assert 9 not in fake.jobs


def test_count_mode_job_has_no_masks(engine):
    E, fake = engine({5: _Job(np.zeros((6, 1), dtype=np.uint64), list_mode=False)})
    r = E.result(5)
    assert r.status == wpm.OK and r.count == 6 and r.masks is None
    assert fake.calls == [(5, 0, False)]


def test_unknown_job_is_an_input_error(engine):
    E, _ = engine({})
    r = E.result(42)
    assert r.status == wpm.ERR_INPUT and r.masks is None
