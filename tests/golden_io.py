"""Reader for the hand-worked fixtures under tests/golden/."""
import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(path):
    u, v, w = [], [], []
    ep = vp = None
    mode = None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0] == "edges":
                mode = "edges"
            elif parts[0] == "edge_parent":
                ep = [int(x) for x in parts[1:]]
                mode = None
            elif parts[0] == "vertex_parent":
                vp = [int(x) for x in parts[1:]]
                mode = None
            elif mode == "edges":
                u.append(int(parts[0]))
                v.append(int(parts[1]))
                w.append(float(parts[2]))
    return (np.array(u, np.int32), np.array(v, np.int32), np.array(w, np.float32),
            np.array(ep, np.int32), np.array(vp, np.int32))


def all_cases():
    return sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))
