"""Write n11_subtrees.txt: exact oracle results on 64 subtrees of the largest Picard-4 map.

The map is the n = 11, m = 15 dual map whose rows are all 15 nonzero vectors of Z2^4 in the
order drawn by seed 0 (instances.full_dual_n11(0)); the property is the upper-bound-theorem
cap. Subtree s is the node reached by the oracle's seeded random walk of 6 steps down the
canonical tree (seed = s), given as forced-in = its In, forced-out = its Out. Each line:
seed, In and Out as 14 hexadecimal uint64 words each (word 0 first), and the oracle's count,
node and probe counts of the subtree. Calls only the oracle.

    python tests/golden/make_n11_subtrees.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2301_00806_gb300 import instances as I  # noqa: E402

N_SUBTREES = 64
DEPTH = 6


def main():
    inst = I.full_dual_n11(0)
    f = O.instance_facets(inst)
    lines = ["# seed in[14 hex words] out[14 hex words] count nodes probes"]
    for seed in range(N_SUBTREES):
        a, b = O.walk(11, 15, f, seed, DEPTH, cap=O.CAP_UBT)
        c, nodes, probes, _ = O.enumerate_dfs(11, 15, f, cap=O.CAP_UBT, forced_in=a, forced_out=b,
                                              list_mode=False)
        words = [f"{int(x):016x}" for x in a] + [f"{int(x):016x}" for x in b]
        lines.append(" ".join([str(seed)] + words + [str(c), str(nodes), str(probes)]))
        print(lines[-1][:40], c, nodes, probes, flush=True)
    with open(os.path.join(HERE, "n11_subtrees.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
