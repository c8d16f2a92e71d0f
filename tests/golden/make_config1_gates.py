"""Writes config1_seed1_gates.json: the 209 gates of config 1 (seed 1) after
the nnz <= 4096 cap has been enforced by rejection sampling on the CPU oracle
(tests/helpers.build_config1).  The file is a workload input, not an expected
value: the batched benchmark workload reads it so that nothing outside the
tests runs the oracle to build it.

    python tests/golden/make_config1_gates.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from tests.helpers import build_config1  # noqa: E402


def encode(g):
    out = []
    for x in g:
        if isinstance(x, tuple):
            out.append([list(c) if isinstance(c, tuple) else c for c in x])
        elif isinstance(x, (np.floating, float)):
            out.append(float(x))
        elif isinstance(x, np.ndarray):
            out.append({"re": x.real.tolist(), "im": x.imag.tolist()})
        elif isinstance(x, (np.integer,)):
            out.append(int(x))
        else:
            out.append(x)
    return out


def main():
    circ = build_config1(seed=1)
    data = {"widths": circ["widths"], "eps": circ["eps"], "seed": 1, "cap": 4096,
            "gates": [encode(g) for g in circ["gates"]]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_seed1_gates.json")
    with open(path, "w") as f:
        head = {k: v for k, v in data.items() if k != "gates"}
        f.write(json.dumps(head)[:-1] + ', "gates": [\n')
        f.write(",\n".join(json.dumps(g) for g in data["gates"]))
        f.write("\n]}\n")
    print(path, len(data["gates"]))


if __name__ == "__main__":
    main()
