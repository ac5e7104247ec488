"""Text fixtures with hand-computed maximum-flow values (see each file's header)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    """Parse one fixture: returns dict(n, s, t, value, source_side, src, dst, cap)."""
    out = {"arcs": []}
    in_arcs = False
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if in_arcs:
                out["arcs"].append([int(x) for x in line.split()])
                continue
            key, *vals = line.split()
            if key == "arcs":
                in_arcs = True
            elif key == "source_side":
                out[key] = [int(v) for v in vals]
            else:
                out[key] = int(vals[0])
    a = np.array(out.pop("arcs"), dtype=np.int32).reshape(-1, 3)
    out["src"], out["dst"], out["cap"] = a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy()
    side = np.zeros(out["n"], np.uint8)
    side[out["source_side"]] = 1
    out["source_side"] = side
    return out


FIXTURES = ["diamond.txt", "antiparallel.txt", "disconnected.txt", "matching.txt"]
