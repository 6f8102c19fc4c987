"""The library's wpm_link_conditions (Section 4.4, conditions (1) and (2)), a host routine
that needs no GPU, against the oracle's own construction of the same masks: on the stored
n = 11 sample links, on every apex link of small maps, and its error statuses."""
import numpy as np
import pytest

import oracle as O
from conftest import load_n11_seeds
from paper_2301_00806_gb300 import instances as I, wpm

_, _, SAMPLES = load_n11_seeds()


def _bits(words, count):
    return [j for j in range(count) if (int(words[j // 64]) >> (j % 64)) & 1]


@pytest.mark.parametrize("idx", range(len(SAMPLES)))
def test_n11_sample_links_match_the_oracle(idx):
    orbit, words = SAMPLES[idx][:2]
    rep = I.idcm_orbit_reps(10)[orbit]
    f10 = O.candidate_facets("dual", 10, 14, rep)
    L = [int(f10[j]) for j in _bits(words, len(f10))]
    lam_o, f_o, fin_o, fout_o = O.link_conditions(11, 15, rep, L)
    lam, M, fin, fout = wpm.link_conditions(11, 15, rep, L)
    assert lam == lam_o and M == len(f_o) == 840
    assert np.array_equal(fin, fin_o) and np.array_equal(fout, fout_o)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_every_apex_link_of_small_maps(seed):
    """Picard 3, n = 4, m = 7: every apex link of every WPM of a seeded map, in a seeded
    vertex order, given in a shuffled facet order."""
    n, m = 4, 7
    rng = I.SplitMix64(100 + seed)
    rows = rng.shuffle(list(range(1, 8)))
    f = O.candidate_facets("dual", n, m, rows)
    c, _, _, masks = O.enumerate_dfs(n, m, f, list_mode=True, capacity=1 << 16)
    apex = 1 << (m - 1)
    links = {tuple(sorted(int(s) ^ apex for s in O.masks_to_facets(f, masks[i]) if int(s) & apex))
             for i in range(c)}
    links.discard(())
    assert links
    for L in sorted(links):
        Ls = rng.shuffle(list(L))
        lam_o, f_o, fin_o, fout_o = O.link_conditions(n, m, rows[:-1], Ls)
        lam, M, fin, fout = wpm.link_conditions(n, m, rows[:-1], Ls)
        assert lam == lam_o and M == len(f_o)
        assert np.array_equal(fin, fin_o) and np.array_equal(fout, fout_o)


def test_explicit_apex_row():
    n, m, mu, apex_row = 2, 6, [1, 2, 4, 8, 3], 12
    L = [0b00011, 0b00110, 0b01100, 0b11000, 0b10001]   # a 5-cycle on vertices 0..4
    f = O.candidate_facets("dual", n, m, mu + [apex_row])
    apex = 1 << (m - 1)
    supported = [s for s in L if (s | apex) in {int(x) for x in f}]
    lam_o, _, fin_o, fout_o = O.link_conditions(n, m, mu, supported, apex_row=apex_row)
    lam, _, fin, fout = wpm.link_conditions(n, m, mu, supported, apex_row=apex_row)
    assert lam == lam_o == mu + [apex_row]
    assert np.array_equal(fin, fin_o) and np.array_equal(fout, fout_o)


def _status(*args, **kw):
    with pytest.raises(wpm.WpmError) as e:
        wpm.link_conditions(*args, **kw)
    return e.value.code


def test_errors():
    rep = I.idcm_orbit_reps(10)[0]
    f10 = O.candidate_facets("dual", 10, 14, rep)
    L = [int(x) for x in f10[:3]]
    assert _status(11, 15, rep[:-1] + [rep[0]], L) == wpm.ERR_INPUT       # repeated row
    assert _status(11, 15, rep[:-1] + [0], L) == wpm.ERR_INPUT            # zero row
    assert _status(11, 15, rep, L + [L[0]]) == wpm.ERR_INPUT              # repeated facet
    assert _status(11, 15, rep, [L[0] | (1 << 14)]) == wpm.ERR_INPUT     # facet through a
    assert _status(11, 15, rep, [0b111]) == wpm.ERR_INPUT                 # wrong size
    assert _status(11, 15, rep, L, apex_row=rep[0]) == wpm.ERR_INPUT      # apex row taken
    assert _status(10, 15, rep, L) == wpm.ERR_INPUT                       # rows not in Z2^4
    # a 10-subset of [14] whose 4 complementary rows are dependent: its cone is no candidate
    cand = {int(x) for x in f10}
    bad = next(s for s in range(1 << 14) if bin(s).count("1") == 10 and s not in cand)
    assert _status(11, 15, rep, [bad]) == wpm.ERR_INPUT
    # apex_row 0 with two vectors missing (m = 6 < 2^4 - 1)
    assert _status(2, 6, [1, 2, 4, 8, 3], [0b11]) == wpm.ERR_INPUT


def test_capacity_status():
    import ctypes as C
    rep = np.asarray(I.idcm_orbit_reps(10)[0], dtype=np.uint32)
    lam = np.zeros(15, dtype=np.uint32)
    fin = np.zeros(13, dtype=np.uint64)
    fout = np.zeros(13, dtype=np.uint64)
    u32p, u64p = C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
    r = wpm.lib().wpm_link_conditions(11, 15, rep.ctypes.data_as(u32p), 0, None, 0,
                                      lam.ctypes.data_as(u32p), fin.ctypes.data_as(u64p),
                                      fout.ctypes.data_as(u64p), 13)
    assert r == wpm.ERR_CAPACITY                                          # 840 needs 14 words
    assert not lam.any() and not fin.any() and not fout.any()
