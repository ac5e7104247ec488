"""Writes tests/golden/oracle_values.json from the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    out = {}
    g = W.grid(64, 64, 1)
    src, dst, cap = g.numpy()
    out["grid64x64_seed1"] = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"]
    g = W.rmat(14, 16, 2)
    src, dst, cap = g.numpy()
    out["rmat14_seed2"] = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"]
    g = W.bipartite_zipf(1 << 12, 1 << 12, 3)
    src, dst, cap = g.numpy()
    out["bipartite4096_seed3"] = oracle.maxflow_pr(g.n, src, dst, cap, g.s, g.t)["value"]
    with open(os.path.join(HERE, "oracle_values.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(out)


if __name__ == "__main__":
    main()
