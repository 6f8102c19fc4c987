import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


def load_table(name):
    """Rows of a whitespace table under tests/golden, '#' lines skipped, ints parsed."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(x) for x in line.split()])
    return rows


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def load_n11_seeds():
    """tests/golden/n11_seeds.txt (written by make_n11_seeds.py from the oracle alone):
    (totals dict, classes [(members, is_sphere, facets)], samples [(orbit, link mask words,
    count, nodes, probes, kept)])."""
    totals, classes, samples = {}, [], []
    with open(os.path.join(GOLDEN, "n11_seeds.txt")) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "class":
                classes.append((int(t[1]), bool(int(t[2])), [int(x, 16) for x in t[3:]]))
            elif t[0] == "sample":
                samples.append((int(t[1]), [int(x, 16) for x in t[2:-4]],
                                *[int(x) for x in t[-4:]]))
            else:
                totals[t[0]] = int(t[1])
    return totals, classes, samples
