"""Writes the golden fixtures of this directory (run from the repository root:
``python tests/golden/make_golden.py``).

The paper prints no worked example, so every stored value here comes from the
oracle: x = (1 - d)(I - dP)^-1 Z (Section 2.1, Eq. pagerank-pf) by the
oracle's dense LAPACK solve (``oracle.dense_solution``) on small seeded graphs,
after the oracle's canonical link merge (``oracle.canonical_csr``).  Nothing
else is called to produce a value.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1501_06350_gb300 import synth  # noqa: E402

D = 0.85
CASES = [
    # name, n, links, seed, dangling share, self-links, weighted, teleport vector
    ("pa_n60", 60, 300, 1, 0.1, False, False, "uniform"),
    ("loops_n200", 200, 1500, 2, 0.2, True, False, "uniform"),
    ("weighted_n200", 200, 1600, 3, 0.1, True, True, "uniform"),
    ("signed_z_n300", 300, 2400, 4, 0.15, False, False, "signed"),
]


def case_inputs(n, m, seed, dang, loops, weighted, zkind):
    g = synth.small_graph(n, m, 500 + seed, dangling_frac=dang, self_loops=loops, weighted=weighted)
    Z = synth.uniform_z(n) if zkind == "uniform" else synth.random_z(n, 600 + seed, signed=True)
    return g, Z


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    for name, n, m, seed, dang, loops, weighted, zkind in CASES:
        g, Z = case_inputs(n, m, seed, dang, loops, weighted, zkind)
        cp, ci, cw = oracle.canonical_csr(g.n, g.ptr, g.idx, g.w)
        x = oracle.dense_solution(g.n, cp, ci, cw if weighted else None, D, Z)
        rec = {
            "what": "x = (1-d)(I - dP)^-1 Z, Section 2.1 Eq. pagerank-pf, by oracle.dense_solution "
                    "on the oracle's canonical CSR; written by tests/golden/make_golden.py",
            "d": D, "n": g.n, "ptr": [int(v) for v in g.ptr], "idx": [int(v) for v in g.idx],
            "w": None if g.w is None else [float(v).hex() for v in g.w],
            "z": [float(v).hex() for v in Z],
            "x": [float(v).hex() for v in x],
        }
        with open(os.path.join(here, name + ".json"), "w") as f:
            json.dump(rec, f, indent=0)
        print(name, g.n, len(g.idx), float(np.abs(x).sum()))


if __name__ == "__main__":
    main()
