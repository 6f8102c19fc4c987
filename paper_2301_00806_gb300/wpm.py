"""Python binding of libwpm (include/wpm.h): argument marshalling only.

Every function calls the C ABI of the in-tree libwpm.so; all enumeration work runs in its
CUDA kernels. There is no CPU fallback: without the built library or a CUDA device the
calls raise.

Masks are returned as numpy uint64 arrays of shape (count, W) with facet j at bit j%64 of
word j/64, rows sorted ascending as multiword integers (word W-1 most significant), or
written into a caller's torch CUDA tensor.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

OK = 0
ERR_INPUT = -1
ERR_CAPACITY = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
ERR_NOMEM = -5
ERR_LIMIT = -6

PRIMAL = 0
DUAL = 1
MODE_LIST = 0
MODE_COUNT = 1
CAP_NONE = -1
CAP_UBT = -2
MAX_FACETS = 2048  # WPM_MAX_FACETS

_KIND = {"primal": PRIMAL, "dual": DUAL, PRIMAL: PRIMAL, DUAL: DUAL}


class WpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libwpm error {code}: {msg}")
        self.code = code


class Conditions(C.Structure):
    _fields_ = [("ubt_cap", C.c_int32), ("require_base_facet", C.c_int32),
                ("n_facets", C.c_int32), ("forced_in", C.POINTER(C.c_uint64)),
                ("forced_out", C.POINTER(C.c_uint64)), ("n_affine", C.c_int32),
                ("affine_c0", C.POINTER(C.c_int32)), ("affine_coef", C.POINTER(C.c_int32)),
                ("post_filter", C.c_int32), ("reserved", C.c_int32)]

POST_PIC = 1   # keep WPMs that use all m vertices (Pic(K) = m - n)
POST_SEED = 2  # keep WPMs that satisfy the seedness condition


class Output(C.Structure):
    _fields_ = [("count", C.c_uint64), ("nodes", C.c_uint64), ("probes", C.c_uint64),
                ("masks", C.POINTER(C.c_uint64)), ("capacity", C.c_uint64),
                ("masks_on_device", C.c_int32), ("words_per_mask", C.c_int32),
                ("M", C.c_int32), ("N", C.c_int32), ("status", C.c_int32),
                ("reserved", C.c_int32), ("found", C.c_uint64)]


class Instance(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("m", C.c_int32),
                ("reserved", C.c_int32), ("lambda_cols", C.POINTER(C.c_uint32)),
                ("cond", C.POINTER(Conditions))]


class Tuning(C.Structure):
    _fields_ = [("frontier_target", C.c_int32), ("budget", C.c_int32),
                ("threads_per_block", C.c_int32), ("idle_percent", C.c_int32),
                ("ring_items", C.c_int64), ("search", C.c_int32), ("profile", C.c_int32),
                ("time_limit_ms", C.c_int32), ("feed_levels", C.c_int32),
                ("hungry_items", C.c_int64), ("donate_levels", C.c_int32),
                ("donate_every", C.c_int32), ("graph", C.c_int32), ("engine", C.c_int32),
                ("sweep_max_s", C.c_int32), ("ready_polls", C.c_int32),
                ("idle_polls", C.c_int32), ("test_unpublished", C.c_int32),
                ("stage_chunk_words", C.c_int32)]


class RunStats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("expand_passes", C.c_uint64),
                ("dfs_passes", C.c_uint64), ("sort_passes", C.c_uint64), ("items", C.c_uint64),
                ("dfs_ms", C.c_double), ("expand_ms", C.c_double), ("search", C.c_int32),
                ("size_class", C.c_int32), ("searches", C.c_int32), ("reserved", C.c_int32),
                ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
                ("graph_launches", C.c_uint64), ("run_ms", C.c_double),
                ("copy_out_ms", C.c_double), ("host_copy_ms", C.c_double)]


class EngineConfig(C.Structure):
    _fields_ = [("memory_bytes", C.c_int64), ("max_jobs", C.c_int32), ("budget", C.c_int32),
                ("max_n", C.c_int32), ("slice_ms", C.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libwpm.so (building it if the sources are newer). Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            u16p, u32p, u64p = C.POINTER(C.c_uint16), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
            L.wpm_candidate_facets.argtypes = [u32p, C.c_int, C.c_int, C.c_int, u16p, C.c_int]
            L.wpm_enumerate.argtypes = [u32p, C.c_int, C.c_int, C.c_int, C.POINTER(Conditions),
                                        C.POINTER(Output), C.c_int]
            L.wpm_enumerate_facets.argtypes = [u16p, C.c_int, C.c_int, C.c_int,
                                               C.POINTER(Conditions), C.POINTER(Output), C.c_int]
            L.wpm_enumerate_batch.argtypes = [C.POINTER(Instance), C.c_int, C.POINTER(Output),
                                              C.c_int, C.POINTER(Tuning), C.c_void_p]
            L.wpm_last_error.restype = C.c_char_p
            L.wpm_autotune.argtypes = [C.POINTER(Instance), C.c_int, C.c_int, C.POINTER(Tuning),
                                       C.POINTER(C.c_double), C.c_void_p]
            L.wpm_iso_classes.argtypes = [C.c_int, C.c_int, u64p, u16p, C.POINTER(C.c_int32)]
            L.wpm_iso_classes.restype = C.c_long
            L.wpm_pl_spheres.argtypes = [C.c_int, C.c_int, C.c_int, u64p, u16p,
                                         C.POINTER(C.c_uint8)]
            L.wpm_pl_spheres.restype = C.c_long
            L.wpm_link_conditions.argtypes = [C.c_int, C.c_int, u32p, C.c_uint32, u16p, C.c_int,
                                              u32p, u64p, u64p, C.c_int]
            L.wpm_last_run_stats.argtypes = [C.POINTER(RunStats)]
            L.wpm_release_workspace.argtypes = []
            L.wpm_engine_create.argtypes = [C.POINTER(EngineConfig), C.c_void_p, C.POINTER(C.c_void_p)]
            L.wpm_engine_submit.argtypes = [C.c_void_p, C.POINTER(Instance), C.c_int, C.c_uint64,
                                            C.POINTER(C.c_uint64)]
            L.wpm_engine_step.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
            L.wpm_engine_poll.argtypes = [C.c_void_p, u64p, C.c_int]
            L.wpm_engine_result.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(Output)]
            L.wpm_int_peak.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
            L.wpm_engine_destroy.argtypes = [C.c_void_p]
            L.wpm_engine_destroy.restype = None
            _lib = L
    return _lib


def _err(code: int) -> WpmError:
    return WpmError(code, lib().wpm_last_error().decode(errors="replace"))


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(C.POINTER(t))


class _Keep:
    """Holds numpy buffers alive while a ctypes struct points into them."""

    def __init__(self):
        self.items = []

    def add(self, a):
        self.items.append(a)
        return a


def _conditions(cap=CAP_NONE, base_facet=False, n_facets=0, forced_in=None, forced_out=None,
                affine=None, keep: Optional[_Keep] = None, post_filter=0) -> Conditions:
    keep = keep or _Keep()
    c = Conditions()
    c.ubt_cap = cap
    c.post_filter = post_filter
    c.require_base_facet = 1 if base_facet else 0
    c.n_facets = n_facets
    W = max(1, (n_facets + 63) // 64)
    for name, val in (("forced_in", forced_in), ("forced_out", forced_out)):
        if val is None:
            setattr(c, name, None)
        else:
            a = np.zeros(W, dtype=np.uint64)
            v = np.asarray(val, dtype=np.uint64).ravel()
            a[:v.size] = v
            setattr(c, name, _p(keep.add(a), C.c_uint64))
    if affine:
        c0 = keep.add(np.asarray([g[0] for g in affine], dtype=np.int32))
        coef = keep.add(np.ascontiguousarray(np.stack([np.asarray(g[1], dtype=np.int32)
                                                       for g in affine])))
        c.n_affine = len(affine)
        c.affine_c0 = _p(c0, C.c_int32)
        c.affine_coef = _p(coef, C.c_int32)
    return c


@dataclass
class Result:
    count: int
    nodes: int
    probes: int
    M: int
    N: int
    words: int
    masks: Optional[np.ndarray]
    status: int = OK
    found: int = 0  # WPMs found before the post-filters (= count without them)


def _result(o: Output, masks) -> Result:
    return Result(int(o.count), int(o.nodes), int(o.probes), int(o.M), int(o.N),
                  int(o.words_per_mask), masks, int(o.status), int(o.found))


def candidate_facets(kind, n: int, m: int, cols: Sequence[int]) -> np.ndarray:
    """Candidate facets (uint16 vertex masks, lexicographic order), computed on the GPU."""
    cc = np.asarray(cols, dtype=np.uint32)
    out = np.zeros(1 << 14, dtype=np.uint16)
    r = lib().wpm_candidate_facets(_p(cc, C.c_uint32), _KIND[kind], n, m, _p(out, C.c_uint16),
                                   out.size)
    if r < 0:
        raise _err(r)
    return out[:r].copy()


def _run_single(call, list_mode: bool, capacity: int) -> Result:
    while True:
        o = Output()
        if list_mode:
            buf = np.zeros((max(capacity, 1), 16), dtype=np.uint64)  # widest mask: 16 words
            o.masks = _p(buf, C.c_uint64)
            o.capacity = capacity
        r = call(o)
        if r == ERR_CAPACITY and list_mode:
            capacity = int(o.count)
            continue
        if r != OK:
            raise _err(r)
        masks = None
        if list_mode:
            w = int(o.words_per_mask)
            masks = buf.reshape(-1)[: int(o.count) * w].reshape(int(o.count), w).copy()
        return _result(o, masks)


def enumerate(kind, n: int, m: int, cols: Sequence[int], cap=CAP_NONE, base_facet=False,
              forced_in=None, forced_out=None, affine=None, n_facets=0, list_mode=True,
              capacity: int = 1 << 14, post_filter: int = 0) -> Result:
    """wpm_enumerate: all WPMs of one map. forced masks / affine rows need n_facets = M;
    post_filter: POST_PIC | POST_SEED (list mode)."""
    keep = _Keep()
    cc = keep.add(np.asarray(cols, dtype=np.uint32))
    cond = _conditions(cap, base_facet, n_facets, forced_in, forced_out, affine, keep,
                       post_filter)
    mode = MODE_LIST if list_mode else MODE_COUNT
    return _run_single(lambda o: lib().wpm_enumerate(_p(cc, C.c_uint32), _KIND[kind], n, m,
                                                     C.byref(cond), C.byref(o), mode),
                       list_mode, capacity)


def enumerate_facets(facets: Sequence[int], n: int, m: int, cap=CAP_NONE, base_facet=False,
                     forced_in=None, forced_out=None, affine=None, list_mode=True,
                     capacity: int = 1 << 14) -> Result:
    """wpm_enumerate_facets: WPMs over an explicit facet list (renumbered lexicographically)."""
    keep = _Keep()
    f = keep.add(np.asarray(facets, dtype=np.uint16))
    cond = _conditions(cap, base_facet, f.size if (forced_in is not None or forced_out is not None
                                                   or affine) else 0,
                       forced_in, forced_out, affine, keep)
    mode = MODE_LIST if list_mode else MODE_COUNT
    return _run_single(lambda o: lib().wpm_enumerate_facets(_p(f, C.c_uint16), f.size, n, m,
                                                            C.byref(cond), C.byref(o), mode),
                       list_mode, capacity)


@dataclass
class BatchSpec:
    kind: object
    n: int
    m: int
    cols: Sequence[int]
    cap: int = CAP_NONE
    base_facet: bool = False
    forced_in: object = None
    forced_out: object = None
    affine: object = None
    n_facets: int = 0
    post_filter: int = 0


def enumerate_batch(specs: List[BatchSpec], list_mode=True, capacities=None, tuning=None,
                    stream=None, device_out=None, words=None, host_out=None) -> List[Result]:
    """wpm_enumerate_batch over many maps in one batched GPU run.

    capacities: per-instance mask capacity (list mode). device_out: optional list of torch
    CUDA uint64 tensors (one per instance, capacity x W) to receive the masks on the device;
    then Result.masks is None and the tensors hold the sorted masks. stream: a torch CUDA
    stream (or raw cudaStream_t int). words: per-instance words per mask (ceil(M/64), e.g.
    from a counting run) to size host buffers exactly; default 16 (the widest). host_out:
    optional list of contiguous numpy uint64 arrays (one per instance, at least
    capacity x words elements) to receive the masks, reusable from call to call; Result.masks
    is then a view of it."""
    n = len(specs)
    keep = _Keep()
    insts = (Instance * max(n, 1))()
    outs = (Output * max(n, 1))()
    conds = []
    bufs = []
    for i in range(n):
        s = specs[i]
        cc = keep.add(np.asarray(s.cols, dtype=np.uint32))
        cond = _conditions(s.cap, s.base_facet, s.n_facets, s.forced_in, s.forced_out, s.affine,
                           keep, s.post_filter)
        conds.append(cond)
        insts[i].kind = _KIND[s.kind]
        insts[i].n = s.n
        insts[i].m = s.m
        insts[i].lambda_cols = _p(cc, C.c_uint32)
        insts[i].cond = C.pointer(cond)
        if list_mode:
            cap = int(capacities[i]) if capacities is not None else (1 << 12)
            if device_out is not None:
                t = device_out[i]
                outs[i].masks = C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_uint64))
                outs[i].masks_on_device = 1
                outs[i].capacity = cap
                bufs.append(None)
            else:
                w = int(words[i]) if words is not None else 16
                if host_out is not None:
                    buf = host_out[i]
                    if (buf.dtype != np.uint64 or not buf.flags.c_contiguous
                            or buf.size < max(cap, 1) * w):
                        raise ValueError(f"host_out[{i}]: need a contiguous uint64 array of "
                                         f"{max(cap, 1) * w} elements")
                    buf = buf.reshape(-1)
                else:
                    buf = np.empty(max(cap, 1) * w, dtype=np.uint64)
                bufs.append(buf)
                outs[i].masks = _p(buf, C.c_uint64)
                outs[i].capacity = cap
        else:
            bufs.append(None)
    tun = None
    if tuning:
        tun = Tuning()
        for k, v in tuning.items():
            setattr(tun, k, v)
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    r = lib().wpm_enumerate_batch(insts, n, outs, MODE_LIST if list_mode else MODE_COUNT,
                                  C.byref(tun) if tun is not None else None,
                                  C.c_void_p(st) if st else None)
    if r not in (OK, ERR_CAPACITY, ERR_TIMEOUT):
        raise _err(r)
    res = []
    for i in range(n):
        o = outs[i]
        masks = None
        if list_mode and bufs[i] is not None and o.status == OK:
            w = int(o.words_per_mask)
            # a view of the buffer the library filled (no second copy of the list)
            masks = bufs[i][: int(o.count) * w].reshape(int(o.count), w)
        res.append(_result(o, masks))
    return res


class Engine:
    """A serving engine (continuous batching, wpm_engine_* of the C ABI).

    submit() queues a job and returns its id; step() admits what fits in device memory and
    runs one search pass over every resident job; poll() lists finished job ids; result()
    fetches one (a Result; masks in list mode)."""

    def __init__(self, memory_bytes=0, max_jobs=0, budget=0, max_n=0, stream=None, slice_ms=0):
        cfg = EngineConfig()
        cfg.memory_bytes = memory_bytes
        cfg.max_jobs = max_jobs
        cfg.budget = budget
        cfg.max_n = max_n
        cfg.slice_ms = slice_ms
        st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        h = C.c_void_p()
        r = lib().wpm_engine_create(C.byref(cfg), C.c_void_p(st) if st else None, C.byref(h))
        if r != OK:
            raise _err(r)
        self._h = h
        self._modes = {}

    def submit(self, kind, n, m, cols, cap=CAP_NONE, base_facet=False, forced_in=None,
               forced_out=None, affine=None, n_facets=0, list_mode=False, capacity=0,
               post_filter=0) -> int:
        keep = _Keep()
        cc = keep.add(np.asarray(cols, dtype=np.uint32))
        cond = _conditions(cap, base_facet, n_facets, forced_in, forced_out, affine, keep,
                           post_filter)
        inst = Instance()
        inst.kind = _KIND[kind]
        inst.n = n
        inst.m = m
        inst.lambda_cols = _p(cc, C.c_uint32)
        inst.cond = C.pointer(cond)
        jid = C.c_uint64()
        r = lib().wpm_engine_submit(self._h, C.byref(inst), MODE_LIST if list_mode else MODE_COUNT,
                                    capacity, C.byref(jid))
        if r != OK:
            raise _err(r)
        self._modes[int(jid.value)] = list_mode
        return int(jid.value)

    def step(self) -> int:
        n = C.c_int()
        r = lib().wpm_engine_step(self._h, C.byref(n))
        if r != OK:
            raise _err(r)
        return int(n.value)

    def poll(self, cap: int = 4096) -> List[int]:
        ids = np.zeros(cap, dtype=np.uint64)
        k = lib().wpm_engine_poll(self._h, _p(ids, C.c_uint64), cap)
        if k < 0:
            raise _err(k)
        return [int(x) for x in ids[:k]]

    def result(self, job_id: int, capacity: int = 0) -> Result:
        """The finished job's Result. A list-mode job's masks are fetched in two calls: the
        first (no buffer) reports the count, the second fills an array of exactly that size
        (`capacity` is accepted for compatibility and not needed)."""
        list_mode = self._modes.get(job_id, False)
        o = Output()
        r = lib().wpm_engine_result(self._h, job_id, C.byref(o))
        masks = None
        if r == ERR_CAPACITY and list_mode and o.status == OK:
            count, w = int(o.count), int(o.words_per_mask)
            masks = np.empty((count, w), dtype=np.uint64)
            o = Output()
            o.masks = _p(masks, C.c_uint64)
            o.capacity = count
            r = lib().wpm_engine_result(self._h, job_id, C.byref(o))
        elif list_mode and r == OK and o.status == OK:
            masks = np.zeros((0, int(o.words_per_mask)), dtype=np.uint64)
        self._modes.pop(job_id, None)
        if r != OK and r != o.status:
            masks = None
        res = _result(o, masks)
        res.status = int(o.status) if r == OK or r == o.status else r
        return res

    def close(self):
        if getattr(self, "_h", None):
            lib().wpm_engine_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(specs: List[BatchSpec], sample: int = 0, stream=None):
    """wpm_autotune: time the library's candidate tunings on a sample of the batch and keep
    the fastest for batches of the same signature. Returns (tuning dict, ms on the sample)."""
    n = len(specs)
    keep = _Keep()
    insts = (Instance * max(n, 1))()
    for i in range(n):
        s = specs[i]
        cc = keep.add(np.asarray(s.cols, dtype=np.uint32))
        cond = _conditions(s.cap, s.base_facet, s.n_facets, s.forced_in, s.forced_out, s.affine,
                           keep)
        keep.add(cond)
        insts[i].kind = _KIND[s.kind]
        insts[i].n = s.n
        insts[i].m = s.m
        insts[i].lambda_cols = _p(cc, C.c_uint32)
        insts[i].cond = C.pointer(cond)
    st = None
    if stream is not None:
        st = stream if isinstance(stream, int) else stream.cuda_stream
    best = Tuning()
    ms = C.c_double()
    r = lib().wpm_autotune(insts, n, sample, C.byref(best), C.byref(ms), st)
    if r != OK:
        raise _err(r)
    return {f: getattr(best, f) for f, _ in Tuning._fields_ if f != "reserved"}, ms.value


def int_peak(op: int = 0, iters: int = 1 << 15):
    """wpm_int_peak: measured integer instructions per second of the GPU (op 0: lop3 + add
    chains, op 1: popc + xor chains). Returns (ops/s, ms of the timed launch)."""
    ops, ms = C.c_double(), C.c_double()
    r = lib().wpm_int_peak(op, iters, C.byref(ops), C.byref(ms))
    if r != OK:
        raise _err(r)
    return float(ops.value), float(ms.value)


def last_run_stats() -> dict:
    """Statistics of this thread's last run (kernel launches, passes, pass durations)."""
    st = RunStats()
    r = lib().wpm_last_run_stats(C.byref(st))
    if r != OK:
        raise _err(r)
    return {f: getattr(st, f) for f, _ in RunStats._fields_ if f != "reserved"}


def release_workspace() -> None:
    lib().wpm_release_workspace()


def complexes_from_masks(facets, masks):
    """(vertex masks of the selected facets, concatenated; offsets) of output masks (count,
    W) of a map whose candidate facets (vertex masks, lexicographic order) are `facets`."""
    f = np.asarray(facets, dtype=np.uint16)
    mk = np.ascontiguousarray(masks, dtype=np.uint64)
    if mk.size == 0:
        return np.zeros(0, dtype=np.uint16), np.zeros(1, dtype=np.uint64)
    bits = np.unpackbits(mk.view(np.uint8).reshape(mk.shape[0], -1), axis=1,
                         bitorder="little")[:, : f.size].astype(bool)
    flat = np.broadcast_to(f, bits.shape)[bits]
    offsets = np.concatenate([[0], np.cumsum(bits.sum(axis=1))]).astype(np.uint64)
    return np.ascontiguousarray(flat, dtype=np.uint16), offsets


def iso_classes(m: int, flat, offsets):
    """wpm_iso_classes: (class of each complex, number of classes) for complexes given as
    concatenated facet vertex masks with offsets (see complexes_from_masks)."""
    fl = np.ascontiguousarray(flat, dtype=np.uint16)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    count = off.size - 1
    cls = np.zeros(max(count, 1), dtype=np.int32)
    n = lib().wpm_iso_classes(m, count, _p(off, C.c_uint64), _p(fl, C.c_uint16),
                              _p(cls, C.c_int32))
    if n < 0:
        raise _err(int(n))
    return cls[:count], int(n)


def pl_spheres(n: int, m: int, flat, offsets):
    """wpm_pl_spheres: (1/0 per complex, number of PL spheres) for complexes given as
    concatenated facet vertex masks with offsets."""
    fl = np.ascontiguousarray(flat, dtype=np.uint16)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    count = off.size - 1
    out = np.zeros(max(count, 1), dtype=np.uint8)
    k = lib().wpm_pl_spheres(n, m, count, _p(off, C.c_uint64), _p(fl, C.c_uint16),
                             _p(out, C.c_uint8))
    if k < 0:
        raise _err(int(k))
    return out[:count].astype(bool), int(k)


def link_conditions(n: int, m: int, mu_rows: Sequence[int], link_facets, apex_row: int = 0):
    """wpm_link_conditions (Section 4.4, conditions (1) and (2)): for the link L (facet
    vertex masks on [m-1]) of the apex m - 1 under the dual map mu_rows (m - 1 rows), returns
    (K's m dual rows, M, forced_in, forced_out) with the masks as ceil(M/64) uint64 words over
    K's candidate facets. apex_row 0: the one nonzero vector mu misses."""
    mu = np.ascontiguousarray(mu_rows, dtype=np.uint32)
    if mu.size != m - 1:
        raise WpmError(ERR_INPUT, f"mu has {mu.size} rows, m - 1 = {m - 1} needed")
    lf = np.ascontiguousarray(link_facets, dtype=np.uint16)
    lam = np.zeros(m, dtype=np.uint32)
    words = MAX_FACETS // 64
    fin = np.zeros(words, dtype=np.uint64)
    fout = np.zeros(words, dtype=np.uint64)
    M = lib().wpm_link_conditions(n, m, _p(mu, C.c_uint32), apex_row, _p(lf, C.c_uint16),
                                  lf.size, _p(lam, C.c_uint32), _p(fin, C.c_uint64),
                                  _p(fout, C.c_uint64), words)
    if M < 0:
        raise _err(M)
    W = max(1, (M + 63) // 64)
    return [int(x) for x in lam], int(M), fin[:W].copy(), fout[:W].copy()
