"""Write n11_full.txt: the oracle's exact result on the whole largest Picard-4 map.

The map is instances.full_dual_n11(0) (n = 11, m = 15, the 15 nonzero vectors of Z2^4 as
dual rows in the order drawn by seed 0), with the upper-bound-theorem cap and no other
property. The line holds: count, nodes, probes of the canonical search. Calls only the
oracle (a few minutes of one CPU core).

    python tests/golden/make_n11_full.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2301_00806_gb300 import instances as I  # noqa: E402


def main():
    inst = I.full_dual_n11(0)
    f = O.instance_facets(inst)
    t0 = time.time()
    c, nodes, probes, _ = O.enumerate_dfs(11, 15, f, cap=O.CAP_UBT, list_mode=False)
    print(c, nodes, probes, f"{time.time() - t0:.1f} s")
    with open(os.path.join(HERE, "n11_full.txt"), "w") as fh:
        fh.write("# instances.full_dual_n11(0), UBT cap: count nodes probes (oracle)\n")
        fh.write(f"{c} {nodes} {probes}\n")


if __name__ == "__main__":
    main()
