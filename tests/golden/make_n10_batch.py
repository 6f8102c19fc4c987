"""Write n10_batch.txt: the oracle's exact results on a batch of 16 maps of n = 10.

The maps are instances.single_dual(10, s) for s = 0..15 (m = 14, 616 candidate facets each),
with the upper-bound-theorem cap and no other property: the smallest batch of n = 10 maps
on which the library picks one search per thread by default. Each line holds: seed, count,
nodes, probes of the canonical search. Calls only the oracle (about two minutes of one CPU
core per map; the maps run in parallel, one process each).

    python tests/golden/make_n10_batch.py
"""
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2301_00806_gb300 import instances as I  # noqa: E402

SEEDS = range(16)


def one(seed):
    inst = I.single_dual(10, seed)
    f = O.instance_facets(inst)
    c, nodes, probes, _ = O.enumerate_dfs(inst.n, inst.m, f, cap=O.CAP_UBT, list_mode=False)
    return seed, c, nodes, probes


def main():
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(len(SEEDS), os.cpu_count() or 1)) as pool:
        rows = pool.map(one, SEEDS)
    print(f"{time.time() - t0:.1f} s")
    with open(os.path.join(HERE, "n10_batch.txt"), "w") as fh:
        fh.write("# instances.single_dual(10, seed), UBT cap: seed count nodes probes (oracle)\n")
        for r in rows:
            fh.write(" ".join(str(x) for x in r) + "\n")


if __name__ == "__main__":
    main()
