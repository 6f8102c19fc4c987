"""bench.py's full-size parity check on CPU: the oracle's results for the sampled maps against
the timed step's per-map results and the sorted mask lists read back from the output buffers
(here CPU tensors standing in for the device buffers). A wrong count, node or probe count, or
a single differing mask word must make the check fail and name the map."""
from dataclasses import dataclass

import numpy as np
import torch

import bench
import oracle as O
from paper_2301_00806_gb300 import instances as I


@dataclass
class R:
    status: int
    count: int
    nodes: int
    probes: int


def _sample():
    maps = I.batch_duals(8, 3, 5, seed=2)
    out, oracle_res, dev, words = [], {}, [], []
    for k, inst in enumerate(maps):
        f = O.instance_facets(inst)
        c, nodes, probes, masks = O.enumerate_dfs(inst.n, inst.m, f, cap=O.CAP_UBT,
                                                  capacity=1 << 14)
        out.append(R(0, c, nodes, probes))
        dev.append(torch.from_numpy(masks.reshape(-1).view(np.int64).copy()))
        words.append(masks.shape[1])
        if k % 2 == 0:  # the sample: every second map
            oracle_res[k] = (c, nodes, probes, masks)
    return out, oracle_res, dev, words


def test_exact_sample_passes():
    out, oracle_res, dev, words = _sample()
    p = bench.parity_sample(oracle_res, out, dev, words)
    assert p["exact"] and p["maps"] == len(oracle_res) and p["mismatches"] == []


def test_a_wrong_node_count_is_reported():
    out, oracle_res, dev, words = _sample()
    out[2] = R(0, out[2].count, out[2].nodes + 1, out[2].probes)
    p = bench.parity_sample(oracle_res, out, dev, words)
    assert not p["exact"] and p["mismatches"][0]["map"] == 2


def test_a_wrong_mask_word_is_reported():
    out, oracle_res, dev, words = _sample()
    k = max(oracle_res, key=lambda j: out[j].count)
    assert out[k].count > 1
    dev[k][words[k]] ^= 1  # the second mask's lowest word
    p = bench.parity_sample(oracle_res, out, dev, words)
    assert not p["exact"] and p["mismatches"] == [{"map": k, "masks_differ": True}]
