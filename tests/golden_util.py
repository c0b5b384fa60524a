"""Load the hand-computed circuits under tests/golden/ as netlists."""
import json
import os

import netgen

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GOLDEN_NAMES = ["chain3", "reconverge_tie", "three_paths_prune"]


def load(name):
    with open(os.path.join(GOLDEN_DIR, name + ".json")) as f:
        g = json.load(f)
    nl = netgen.from_lists(g["cells"], [[tuple(p) for p in net] for net in g["nets"]])
    return g, nl
