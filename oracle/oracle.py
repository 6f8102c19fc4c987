"""ctypes binding for the C oracle (`oracle.c`). Test infrastructure only.

Every function here takes and returns plain Python / numpy values; the enumeration
functions return (count, nodes, probes, masks) with masks a (count, W) uint64 array sorted
ascending as multiword integers (word W-1 most significant), or None in counting mode.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CAP_NONE = -1
CAP_UBT = -2


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cond(C.Structure):
    _fields_ = [("cap", C.c_int32), ("base_facet", C.c_int32),
                ("forced_in", C.POINTER(C.c_uint64)), ("forced_out", C.POINTER(C.c_uint64)),
                ("n_affine", C.c_int32), ("c0", C.POINTER(C.c_int32)),
                ("coef", C.POINTER(C.c_int32))]


class _Stats(C.Structure):
    _fields_ = [("count", C.c_uint64), ("nodes", C.c_uint64), ("probes", C.c_uint64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u16p, u32p, u64p = C.POINTER(C.c_uint16), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
            L.orc_candidate_facets.argtypes = [C.c_int, C.c_int, C.c_int, u32p, u16p, C.c_int]
            L.orc_ridges.argtypes = [C.c_int, C.c_int, u16p, u16p, C.POINTER(C.c_int32), C.c_int]
            L.orc_kernel_dim.argtypes = [C.c_int, C.c_int, u16p]
            L.orc_ubt_cap.argtypes = [C.c_int]
            for name in ("orc_enumerate_brute", "orc_enumerate_dfs"):
                getattr(L, name).argtypes = [C.c_int, C.c_int, C.c_int, u16p, C.POINTER(_Cond),
                                             u64p, C.c_uint64, C.POINTER(_Stats)]
            L.orc_enumerate_sweep.argtypes = [C.c_int, C.c_int, C.c_int, u16p, C.POINTER(_Cond),
                                              u64p, C.c_uint64, C.POINTER(_Stats), C.c_int]
            L.orc_enumerate_sweep_fixed.argtypes = [C.c_int, C.c_int, C.c_int, u16p,
                                                    C.POINTER(_Cond), u64p, C.c_uint64,
                                                    C.POINTER(_Stats), C.c_int]
            L.orc_enumerate_sweep_blocks.argtypes = [C.c_int, C.c_int, C.c_int, u16p,
                                                     C.POINTER(_Cond), u64p, C.c_uint64,
                                                     C.POINTER(_Stats), C.c_double]
            L.orc_convenient_basis.argtypes = [C.c_int, C.c_int, C.c_int, u16p, C.POINTER(_Cond),
                                               C.POINTER(C.c_int32), C.c_int,
                                               C.POINTER(C.c_double)]
            L.orc_enumerate_dfs_budget.argtypes = [C.c_int, C.c_int, C.c_int, u16p,
                                                   C.POINTER(_Cond), C.POINTER(_Stats),
                                                   C.c_uint64]
            L.orc_walk.argtypes = [C.c_int, C.c_int, C.c_int, u16p, C.POINTER(_Cond), C.c_uint64,
                                   C.c_int, u64p, u64p]
            L.orc_pic_seed.argtypes = [C.c_int, C.c_int, C.c_int, u16p]
            L.orc_filter_pic_seed.argtypes = [C.c_int, C.c_int, C.c_int, u16p, u64p, C.c_long,
                                              C.c_int, C.POINTER(C.c_uint8)]
            L.orc_filter_pic_seed.restype = C.c_long
            L.orc_canonical_form.argtypes = [C.c_int, C.c_int, u16p, u16p]
            L.orc_pl_sphere.argtypes = [C.c_int, C.c_int, C.c_int, u16p]
            L.orc_n2_cycle_sets.argtypes = [C.c_int, u16p, C.c_int]
            L.orc_n2_cycle_sets.restype = C.c_long
            L.orc_n2_cycle_count.argtypes = [C.c_int, u16p]
            L.orc_n2_cycle_count.restype = C.c_long
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise OracleError(f"{what} failed with code {rc}")
    return rc


def _p(arr: np.ndarray, ctype):
    return arr.ctypes.data_as(C.POINTER(ctype))


def candidate_facets(kind: str, n: int, m: int, cols: Sequence[int]) -> np.ndarray:
    """Candidate facets (uint16 vertex masks) in lexicographic order."""
    k = {"primal": 0, "dual": 1}[kind]
    c = np.asarray(cols, dtype=np.uint32)
    out = np.zeros(1 << 16, dtype=np.uint16)
    M = _check(lib().orc_candidate_facets(k, n, m, _p(c, C.c_uint32), _p(out, C.c_uint16),
                                          out.size), "candidate_facets")
    return out[:M].copy()


def ridges(n: int, facets: np.ndarray):
    """(ridge vertex masks in lexicographic order, number of parents of each)."""
    f = np.ascontiguousarray(facets, dtype=np.uint16)
    out = np.zeros(1 << 16, dtype=np.uint16)
    npar = np.zeros(1 << 16, dtype=np.int32)
    N = _check(lib().orc_ridges(n, f.size, _p(f, C.c_uint16), _p(out, C.c_uint16),
                                _p(npar, C.c_int32), out.size), "ridges")
    return out[:N].copy(), npar[:N].copy()


def kernel_dim(n: int, facets: np.ndarray) -> int:
    """dim ker_Z2 A for the ridge-facet incidence matrix of the given facets."""
    f = np.ascontiguousarray(facets, dtype=np.uint16)
    return _check(lib().orc_kernel_dim(n, f.size, _p(f, C.c_uint16)), "kernel_dim")


def ubt_cap(n: int) -> int:
    return lib().orc_ubt_cap(n)


def _cond(M: int, cap: int, base_facet: bool, forced_in, forced_out, affine):
    W = (M + 63) // 64
    keep = []
    cond = _Cond()
    cond.cap = cap
    cond.base_facet = 1 if base_facet else 0
    for name, val in (("forced_in", forced_in), ("forced_out", forced_out)):
        if val is None:
            setattr(cond, name, None)
        else:
            a = np.zeros(W, dtype=np.uint64)
            v = np.asarray(val, dtype=np.uint64).ravel()
            a[:v.size] = v
            keep.append(a)
            setattr(cond, name, _p(a, C.c_uint64))
    if affine:
        c0 = np.asarray([g[0] for g in affine], dtype=np.int32)
        coef = np.ascontiguousarray(np.stack([np.asarray(g[1], dtype=np.int32) for g in affine]))
        assert coef.shape == (len(affine), M)
        keep += [c0, coef]
        cond.n_affine = len(affine)
        cond.c0 = _p(c0, C.c_int32)
        cond.coef = _p(coef, C.c_int32)
    else:
        cond.n_affine = 0
    return cond, keep


def _enumerate(fn, n, m, facets, cap, base_facet, forced_in, forced_out, affine, list_mode,
               capacity, extra=()):
    f = np.ascontiguousarray(facets, dtype=np.uint16)
    M = f.size
    W = max(1, (M + 63) // 64)
    cond, keep = _cond(M, cap, base_facet, forced_in, forced_out, affine)
    st = _Stats()
    if list_mode:
        buf = np.zeros((capacity, W), dtype=np.uint64)
        rc = fn(n, m, M, _p(f, C.c_uint16), C.byref(cond), _p(buf, C.c_uint64), capacity,
                C.byref(st), *extra)
    else:
        buf = None
        rc = fn(n, m, M, _p(f, C.c_uint16), C.byref(cond), None, 0, C.byref(st), *extra)
    if rc == -2 and list_mode:
        return _enumerate(fn, n, m, facets, cap, base_facet, forced_in, forced_out, affine,
                          list_mode, int(st.count) + 1, extra)
    _check(rc, fn.__name__)
    del keep
    masks = buf[:st.count].copy() if list_mode else None
    return int(st.count), int(st.nodes), int(st.probes), masks


def enumerate_dfs(n, m, facets, cap=CAP_NONE, base_facet=False, forced_in=None,
                  forced_out=None, affine=None, list_mode=True, capacity=1 << 12):
    """O1: ridge-driven canonical search. Returns (count, nodes, probes, masks)."""
    return _enumerate(lib().orc_enumerate_dfs, n, m, facets, cap, base_facet, forced_in,
                      forced_out, affine, list_mode, capacity)


def enumerate_brute(n, m, facets, cap=CAP_NONE, base_facet=False, forced_in=None,
                    forced_out=None, affine=None, list_mode=True, capacity=1 << 12):
    """O3: all 2^M subsets checked by Proposition 2.1."""
    return _enumerate(lib().orc_enumerate_brute, n, m, facets, cap, base_facet, forced_in,
                      forced_out, affine, list_mode, capacity)


def enumerate_sweep(n, m, facets, cap=CAP_NONE, base_facet=False, forced_in=None,
                    forced_out=None, affine=None, list_mode=True, capacity=1 << 12, max_s=30):
    """O2: sweep of ker_Z2 A (Section 2.1)."""
    return _enumerate(lib().orc_enumerate_sweep, n, m, facets, cap, base_facet, forced_in,
                      forced_out, affine, list_mode, capacity, extra=(max_s,))


def enumerate_sweep_fixed(n, m, facets, cap=CAP_NONE, base_facet=False, forced_in=None,
                          forced_out=None, affine=None, list_mode=True, capacity=1 << 12,
                          max_free=30):
    """O2 with Section 4.4's initialization: forced-in / forced-out facets fix part of the
    kernel coordinates X (column echelon form of the kernel basis, rows in the order I, J,
    rest); only the free coordinates are swept. Returns (count, combinations swept, number
    of free coordinates, masks)."""
    return _enumerate(lib().orc_enumerate_sweep_fixed, n, m, facets, cap, base_facet,
                      forced_in, forced_out, affine, list_mode, capacity, extra=(max_free,))


def enumerate_sweep_blocks(n, m, facets, cap=CAP_NONE, base_facet=False, forced_in=None,
                           forced_out=None, affine=None, list_mode=True, capacity=1 << 12,
                           max_log2_x=30.0):
    """O2 with Section 2.1's convenient basis: forced rows fix part of X (Section 4.4), Z
    blocks over ridges with disjoint parents allow at most two generators each, the other
    free generators are swept. Returns (count, combinations visited = |X|, 0, masks)."""
    return _enumerate(lib().orc_enumerate_sweep_blocks, n, m, facets, cap, base_facet,
                      forced_in, forced_out, affine, list_mode, capacity,
                      extra=(C.c_double(max_log2_x),))


def convenient_basis(n, m, facets, base_facet=False, forced_in=None, forced_out=None):
    """The convenient basis's shape: dict with s, fixed1, fixed0, feasible, the block sizes,
    the single free generators, and log2 |X| (Section 2.1; Table 1's |X| rows)."""
    f = np.ascontiguousarray(facets, dtype=np.uint16)
    cond, keep = _cond(f.size, CAP_NONE, base_facet, forced_in, forced_out, None)
    info = np.zeros(512, dtype=np.int32)
    lx = C.c_double()
    k = _check(lib().orc_convenient_basis(n, m, f.size, _p(f, C.c_uint16), C.byref(cond),
                                          _p(info, C.c_int32), info.size, C.byref(lx)),
               "convenient_basis")
    del keep
    return {"s": int(info[0]), "fixed1": int(info[1]), "fixed0": int(info[2]),
            "feasible": bool(info[3]), "blocks": [int(x) for x in info[6:k]],
            "singles": int(info[5]), "log2_x": float(lx.value)}


def n2_cycle_sets(edges: np.ndarray, max_edges: int = -1) -> int:
    """O4 (n = 2): families of vertex-disjoint cycles with at most max_edges edges."""
    e = np.ascontiguousarray(edges, dtype=np.uint16)
    return _check(lib().orc_n2_cycle_sets(e.size, _p(e, C.c_uint16), max_edges), "n2_cycle_sets")


def n2_cycle_count(edges: np.ndarray) -> int:
    e = np.ascontiguousarray(edges, dtype=np.uint16)
    return _check(lib().orc_n2_cycle_count(e.size, _p(e, C.c_uint16)), "n2_cycle_count")


def instance_facets(inst) -> np.ndarray:
    return candidate_facets(inst.kind, inst.n, inst.m, inst.cols)


def enumerate_dfs_budget(n, m, facets, max_nodes, cap=CAP_NONE, base_facet=False,
                         forced_in=None, forced_out=None, affine=None):
    """O1 in counting mode with a node budget: (count, nodes, probes), or None when the
    search would exceed max_nodes nodes."""
    f = np.ascontiguousarray(facets, dtype=np.uint16)
    cond, keep = _cond(f.size, cap, base_facet, forced_in, forced_out, affine)
    st = _Stats()
    rc = lib().orc_enumerate_dfs_budget(n, m, f.size, _p(f, C.c_uint16), C.byref(cond),
                                        C.byref(st), max_nodes)
    del keep
    if rc == -7:
        return None
    _check(rc, "enumerate_dfs_budget")
    return int(st.count), int(st.nodes), int(st.probes)


def walk(n, m, facets, seed, depth, cap=CAP_NONE):
    """Seeded random walk of `depth` steps down the canonical tree; returns the (In, Out)
    masks of the node reached (uint64 arrays of ceil(M/64) words)."""
    f = np.ascontiguousarray(facets, dtype=np.uint16)
    W = max(1, (f.size + 63) // 64)
    cond, keep = _cond(f.size, cap, False, None, None, None)
    a = np.zeros(W, dtype=np.uint64)
    b = np.zeros(W, dtype=np.uint64)
    _check(lib().orc_walk(n, m, f.size, _p(f, C.c_uint16), C.byref(cond), seed, depth,
                          _p(a, C.c_uint64), _p(b, C.c_uint64)), "walk")
    del keep
    return a, b


def pic_seed(n, m, facet_masks) -> bool:
    """Algorithm 4.4 lines 8-12 on one complex K (its facets as vertex masks): True when K
    uses all m vertices (Pic(K) = 4) and satisfies the seedness condition (Prop. 3.1)."""
    kf = np.ascontiguousarray(facet_masks, dtype=np.uint16)
    return bool(_check(lib().orc_pic_seed(n, m, kf.size, _p(kf, C.c_uint16)), "pic_seed"))


def filter_pic_seed(n, m, facets, masks):
    """Keep flags (uint8 array) of orc_pic_seed over output masks (count, W) of a map whose
    candidate facets are `facets`."""
    f = np.ascontiguousarray(facets, dtype=np.uint16)
    mk = np.ascontiguousarray(masks, dtype=np.uint64)
    count = mk.shape[0]
    W = mk.shape[1] if mk.ndim == 2 else 1
    keep = np.zeros(max(count, 1), dtype=np.uint8)
    _check(lib().orc_filter_pic_seed(n, m, f.size, _p(f, C.c_uint16), _p(mk, C.c_uint64),
                                     count, W, _p(keep, C.c_uint8)), "filter_pic_seed")
    return keep[:count]


def canonical_form(m, facet_masks) -> tuple:
    """Algorithm 4.4 line 14: a canonical form of K (facets as vertex masks on [m]) under
    vertex relabeling; isomorphic complexes, and only they, have equal forms."""
    kf = np.ascontiguousarray(facet_masks, dtype=np.uint16)
    out = np.zeros(max(kf.size, 1), dtype=np.uint16)
    _check(lib().orc_canonical_form(m, kf.size, _p(kf, C.c_uint16), _p(out, C.c_uint16)),
           "canonical_form")
    return tuple(int(x) for x in out[:kf.size])


def masks_to_facets(facets, mask_row):
    """Vertex masks of the facets selected by one output mask row."""
    M = len(facets)
    return [int(facets[j]) for j in range(M) if (int(mask_row[j // 64]) >> (j % 64)) & 1]


def pl_sphere(n, m, facet_masks) -> bool:
    """Algorithm 4.4 line 16 by Lemma 3.3: the link of every face of K (the empty face
    included) is a Z2-homology sphere."""
    kf = np.ascontiguousarray(facet_masks, dtype=np.uint16)
    return bool(_check(lib().orc_pl_sphere(n, m, kf.size, _p(kf, C.c_uint16)), "pl_sphere"))


def pic_full(m, facet_masks) -> bool:
    """Algorithm 4.4 line 9 on its own: K keeps Pic(K) = m - n exactly when its facets use
    every vertex of [m] (the seedness test of line 10 is not applied)."""
    used = 0
    for s in facet_masks:
        used |= int(s)
    return used == (1 << m) - 1


def link_conditions(n, m, mu, link_facets, apex_row=None):
    """Section 4.4 (Enumeration for n = 11): the search for the complexes K on [m] whose
    last vertex a = m - 1 has the link L.

    mu: the dual rows of L's map on the vertices 0..m-2 (distinct nonzero vectors of
    Z2^(m-n)); apex_row: the dual row of a, by default the one nonzero vector that mu does
    not take (the paper's case: m = 15 = 2^4 - 1, so the map of K is fixed by mu).
    Every K with Lk_K(a) = L contains the cone {sigma + a : sigma in L}, so
      condition (1): each facet sigma + a (sigma a facet of L) is in K;
      condition (2): each other candidate facet through a is not in K.
    Returns (the m dual rows of K's map, its candidate facets, forced-in mask, forced-out
    mask), the masks as ceil(M/64) uint64 words over the candidate facets."""
    p = m - n
    mu = [int(v) for v in mu]
    assert len(mu) == m - 1
    if apex_row is None:
        missing = [v for v in range(1, 1 << p) if v not in mu]
        assert len(missing) == 1, "the apex row is fixed by mu only when mu misses one vector"
        apex_row = missing[0]
    lam = mu + [int(apex_row)]
    facets = candidate_facets("dual", n, m, lam)
    a = 1 << (m - 1)
    cone = set()
    for s in link_facets:
        s = int(s)
        assert bin(s).count("1") == n - 1 and s < a, "a facet of L is an (n-1)-subset of [m-1]"
        cone.add(s | a)
    W = max(1, (len(facets) + 63) // 64)
    fin = np.zeros(W, dtype=np.uint64)
    fout = np.zeros(W, dtype=np.uint64)
    seen = 0
    for j, s in enumerate(facets):
        s = int(s)
        if not s & a:
            continue
        bit = np.uint64(1 << (j % 64))
        if s in cone:
            fin[j // 64] |= bit
            seen += 1
        else:
            fout[j // 64] |= bit
    assert seen == len(cone), "every cone facet sigma + a must be a candidate facet of K's map"
    return lam, facets, fin, fout
