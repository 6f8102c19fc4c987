"""Pins for the oracle's sweep over Section 2.1's convenient basis (orc_enumerate_sweep_blocks,
orc_convenient_basis): the Z blocks, the partition I_1..I_l and the sets X_l.

What pins it, besides its own arithmetic:
  * Table 1's |X| row for the set of all n-subsets of [n + 4]: 352 for n = 2 exactly (one
    block of m - n = 4 generators, 1 + 4 + C(4, 2) = 11 choices, five single generators,
    and the base facet {1..n} fixing one coordinate), and the printed orders of magnitude
    for n = 3 and 4;
  * Table 1's max |X(F(lambda))| row over the IDCM orbits, n = 2..11, within the factor that
    an unspecified choice of ridges allows (the paper leaves the choice open), and far below
    the plain 2^s sweep;
  * the set of WPMs: equal, mask for mask, to the definition (brute force over all subsets)
    and to the canonical search, with and without the cap, the base facet, forced facets
    (Section 4.4's fixed coordinates) and general affine properties;
  * the number of combinations visited: the product of the block choices and 2^singles.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from conftest import load_n11_seeds
from paper_2301_00806_gb300 import instances as I


def all_nsubsets(n, m):
    return np.array([sum(1 << v for v in c) for c in itertools.combinations(range(m), n)],
                    dtype=np.uint16)


def one_digit(x):
    """x rounded to one significant digit, as Table 1 prints its large counts."""
    e = math.floor(math.log10(x))
    return round(x / 10 ** e) * 10 ** e


# --------------------------------------------------------------------------------------
# Table 1, |X| for all n-subsets of [n + 4] (the complete case of Section 2.1)
# --------------------------------------------------------------------------------------

def test_complete_case_n2_gives_tables_352():
    f = all_nsubsets(2, 6)
    info = O.convenient_basis(2, 6, f, base_facet=True)
    assert info["s"] == 10 and info["fixed1"] == 1
    # K_6: every vertex (ridge) has five parents, so the one block is Z_4; any two vertices
    # share an edge, so no second ridge has disjoint parents
    assert info["blocks"] == [4] and info["singles"] == 5
    assert round(2 ** info["log2_x"]) == 352 == 11 * 2 ** 5


@pytest.mark.parametrize("n,printed", [(3, 2e5), (4, 1e9)])
def test_complete_case_orders_of_magnitude(n, printed):
    info = O.convenient_basis(n, n + 4, all_nsubsets(n, n + 4), base_facet=True)
    # in the complete case every ridge has m - n + 1 parents: full blocks Z_{m - n}
    assert info["blocks"] and all(k == 4 for k in info["blocks"])
    assert one_digit(2 ** info["log2_x"]) == printed


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_blocks_never_exceed_m_minus_n(n):
    info = O.convenient_basis(n, n + 4, all_nsubsets(n, n + 4), base_facet=True)
    assert max(info["blocks"]) <= 4
    assert info["fixed1"] + info["fixed0"] + sum(info["blocks"]) + info["singles"] == info["s"]


# --------------------------------------------------------------------------------------
# Table 1, max |X(F(lambda))| over the IDCM orbits
# --------------------------------------------------------------------------------------

TABLE1_MAX_X = {2: 56, 3: 3e3, 4: 5e5, 5: 1e6, 6: 2e7, 7: 9e8, 8: 1e11, 9: 3e12, 10: 4e14,
                11: 4e16}


@pytest.mark.parametrize("n", sorted(TABLE1_MAX_X))
def test_per_map_x_tracks_table1(n):
    best, plain = 0.0, 0.0
    for rows in I.idcm_orbit_reps(n):
        f = O.candidate_facets("dual", n, n + 4, rows)
        info = O.convenient_basis(n, n + 4, f, base_facet=True)
        best = max(best, 2 ** info["log2_x"])
        plain = max(plain, 2.0 ** (info["s"] - 1))
    # the paper leaves the choice of ridges open; any reasonable choice lands within a
    # small factor of its printed maximum
    assert TABLE1_MAX_X[n] / 2 <= best <= TABLE1_MAX_X[n] * 2, best
    # and the blocks matter, more as n grows: the plain sweep is larger (2x from n = 4 on,
    # 10x from n = 7 on, about 170x at n = 11)
    assert plain > best
    assert n < 4 or plain >= 2 * best
    assert n < 7 or plain >= 10 * best


# --------------------------------------------------------------------------------------
# The set of WPMs
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("cap", [O.CAP_NONE, O.CAP_UBT])
@pytest.mark.parametrize("seed", [0, 5, 11])
def test_fano_blocks_equal_brute_force(cap, seed):
    f = O.instance_facets(I.fano_primal(seed))
    b = O.enumerate_brute(3, 7, f, cap=cap)
    x = O.enumerate_sweep_blocks(3, 7, f, cap=cap)
    assert x[0] == b[0] == (666 if cap == O.CAP_UBT else 1303)
    assert np.array_equal(x[3], b[3])
    info = O.convenient_basis(3, 7, f)
    assert x[1] == round(2 ** info["log2_x"])  # combinations visited = |X|
    assert x[1] < 2 ** info["s"]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("base", [False, True])
def test_n5_blocks_equal_search(seed, base):
    inst = I.single_dual(5, seed)
    f = O.instance_facets(inst)
    d = O.enumerate_dfs(5, 9, f, cap=O.CAP_UBT, base_facet=base, capacity=1 << 14)
    x = O.enumerate_sweep_blocks(5, 9, f, cap=O.CAP_UBT, base_facet=base, capacity=1 << 14)
    assert x[0] == d[0] and np.array_equal(x[3], d[3])


def _random_case(rng, n):
    m = int(rng.integers(n + 1, min(16, n + 5) + 1))
    allf = all_nsubsets(n, m)
    M = int(min(allf.size, rng.integers(6, 19)))
    pick = np.sort(rng.choice(allf.size, size=M, replace=False))
    return m, allf[pick]


@pytest.mark.parametrize("seed", range(40))
def test_random_properties_blocks_equal_brute_force(seed):
    """Random facet sets with forced-in / forced-out facets, caps and affine properties:
    forced rows fix coordinates and move the blocks' centres c_l, which the brute force
    knows nothing about."""
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.integers(2, 5))
    m, facets = _random_case(rng, n)
    M = facets.size
    kw = {}
    if seed % 2:
        kw["cap"] = int(rng.integers(0, M + 1))
    if seed % 3 == 0:
        kw["forced_in"] = [int(rng.integers(0, 1 << M)) & int(rng.integers(0, 1 << M))]
    if seed % 5 == 0:
        kw["forced_out"] = [int(rng.integers(0, 1 << M)) & int(rng.integers(0, 1 << M))]
    if seed % 4 in (1, 2):
        kw["affine"] = [(int(rng.integers(-3, 6)), rng.integers(-2, 3, size=M).tolist())
                        for _ in range(int(rng.integers(1, 3)))]
    if seed % 7 == 0:
        kw["base_facet"] = True
    b = O.enumerate_brute(n, m, facets, **kw)
    x = O.enumerate_sweep_blocks(n, m, facets, **kw)
    assert x[0] == b[0]
    assert np.array_equal(x[3], b[3])


def _mask_bits(words, count):
    return [j for j in range(count) if (int(words[j // 64]) >> (j % 64)) & 1]


@pytest.mark.parametrize("idx", range(6))
def test_section_4_4_links_blocks_equal_fixed_sweep_and_search(idx):
    """The stored n = 11 sample links (Section 4.4's conditions (1), (2) as forced sets): the
    convenient basis fixes the same number of coordinates as the paper's x_t rule and may
    add blocks over the rest; the outputs equal the conditioned search's and the stored
    count."""
    _, _, samples = load_n11_seeds()
    orbit, words, count = samples[idx][:3]
    rep = I.idcm_orbit_reps(10)[orbit]
    f10 = O.candidate_facets("dual", 10, 14, rep)
    L = [int(f10[j]) for j in _mask_bits(words, len(f10))]
    _, f, fin, fout = O.link_conditions(11, 15, rep, L)
    d = O.enumerate_dfs(11, 15, f, cap=O.CAP_UBT, forced_in=fin, forced_out=fout, capacity=64)
    x = O.enumerate_sweep_blocks(11, 15, f, cap=O.CAP_UBT, forced_in=fin, forced_out=fout,
                                 capacity=64)
    fx = O.enumerate_sweep_fixed(11, 15, f, cap=O.CAP_UBT, forced_in=fin, forced_out=fout,
                                 capacity=64)
    assert x[0] == d[0] == fx[0] == count and np.array_equal(x[3], d[3])
    info = O.convenient_basis(11, 15, f, forced_in=fin, forced_out=fout)
    assert info["s"] == 64
    assert info["s"] - info["fixed1"] - info["fixed0"] == fx[2]   # the free coordinates
    assert x[1] <= fx[1] == 2 ** fx[2]                            # blocks only remove cases
