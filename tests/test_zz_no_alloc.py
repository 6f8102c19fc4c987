"""wpm_candidate_facets_static: the allocation-free entry point (device scratch in one fixed
__device__ array of the library) must give exactly what wpm_candidate_facets gives.

Callers that cannot allocate (a service whose device memory is reserved once at start-up, a
framework that owns the allocator, code inside stream capture) use it; this file is named to
run last, and it passes alone in a fresh process as well as after the other tests."""
import ctypes as C

import numpy as np
import pytest

from paper_2301_00806_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2301_00806_gb300 import wpm
    L = wpm.lib()
    L.wpm_candidate_facets_static.argtypes = [C.POINTER(C.c_uint32), C.c_int, C.c_int, C.c_int,
                                              C.POINTER(C.c_uint16), C.c_int, C.c_void_p]
    return L


def _call(fn, inst, extra=()):
    cols = np.asarray(inst.cols, dtype=np.uint32)
    out = np.zeros(4096, dtype=np.uint16)
    kind = 0 if inst.kind == "primal" else 1
    r = fn(cols.ctypes.data_as(C.POINTER(C.c_uint32)), kind, inst.n, inst.m,
           out.ctypes.data_as(C.POINTER(C.c_uint16)), out.size, *extra)
    return r, out[:max(r, 0)].copy()


def test_static_matches_allocating_entry_point_twice_in_a_row(lib):
    # largest map first, then smaller ones: leftover scratch contents must not matter
    for inst in [I.full_dual_n11(3), I.single_dual(5, 2), I.fano_primal(4), I.single_dual(8, 1)]:
        want_r, want = _call(lib.wpm_candidate_facets, inst)
        assert want_r > 0
        for _ in range(2):
            got_r, got = _call(lib.wpm_candidate_facets_static, inst, (None,))
            assert got_r == want_r
            assert np.array_equal(got, want)


def test_static_rejects_maps_beyond_its_scratch(lib):
    inst = I.Instance(n=8, m=16, kind="primal", cols=[1 << (i % 8) for i in range(16)])
    r, _ = _call(lib.wpm_candidate_facets_static, inst, (None,))
    assert r == -6  # WPM_ERR_LIMIT
    assert b"static" in lib.wpm_last_error()
