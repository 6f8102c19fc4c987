"""wpm_candidate_facets_static: the allocation-free entry point (device scratch in one fixed
__device__ array of the library) must give exactly what wpm_candidate_facets gives.

Callers that cannot allocate (a service whose device memory is reserved once at start-up, a
framework that owns the allocator) use it. Each case calls it twice in a row, on the default
stream and on a caller's stream, with the largest maps first so that leftover contents of the
shared array cannot matter, and checks that device memory in use does not change across the
calls. This file is named to run last, and it passes alone in a fresh process as well as after
the other tests."""
import ctypes as C

import numpy as np
import pytest

from paper_2301_00806_gb300 import instances as I

pytestmark = pytest.mark.gpu

# n = 6 on 16 vertices: 8008 facet ranks and 4368 ridge ranks, about 463 KB of the 512 KiB
# array (M = 1280 candidates, N = 1728 ridges)
NEAR_BOUND = I.Instance(n=6, m=16, kind="primal",
                        cols=[1, 2, 4, 8, 16, 32, 1, 2, 4, 8, 16, 32, 3, 12, 48, 63])


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


def _maps():
    return [NEAR_BOUND, I.full_dual_n11(3), I.single_dual(5, 2), I.fano_primal(4),
            I.single_dual(8, 1)]


def test_static_matches_allocating_entry_point_twice_in_a_row(lib):
    import torch
    maps = _maps()
    want = []
    for inst in maps:
        r, f = _call(lib.wpm_candidate_facets, inst)
        assert r > 0, lib.wpm_last_error()
        want.append((r, f))
    side = torch.cuda.Stream()
    # one warm call (module loading on first use may take device memory), then measure
    _call(lib.wpm_candidate_facets_static, I.fano_primal(0), (None,))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    for stream in (None, side.cuda_stream):
        for inst, (want_r, want_f) in zip(maps, want):
            for _ in range(2):
                got_r, got = _call(lib.wpm_candidate_facets_static, inst, (stream,))
                assert got_r == want_r, lib.wpm_last_error()
                assert np.array_equal(got, want_f)
                assert lib.wpm_last_error() == b""
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_static_rejects_maps_beyond_its_scratch(lib):
    # n = 7 on 16 vertices: about 725 KB of scratch
    inst = I.Instance(n=7, m=16, kind="primal", cols=[1 << (i % 7) for i in range(16)])
    r, _ = _call(lib.wpm_candidate_facets_static, inst, (None,))
    assert r == -6  # WPM_ERR_LIMIT
    assert b"static" in lib.wpm_last_error()
    # the next successful call starts with a clear error string
    r, _ = _call(lib.wpm_candidate_facets_static, I.fano_primal(1), (None,))
    assert r == 28 and lib.wpm_last_error() == b""
