"""Writes the stored expected values under tests/golden/ by calling only the oracle.

two_moons_64.json: degrees, samples and the SET edge list of Algorithm 2 on a
64-point two-moons set (the shape of the paper's Sec. 5.1 data), sigma = 0.1
with gamma = 1/(2 sigma^2), L = 8, seed 0, self term excluded.  It pins the
oracle against accidental change (regression); its values come from
oracle/fsg_oracle.c, never from the CUDA path.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as ora  # noqa: E402
from paper_2310_13870_gb300 import inputs  # noqa: E402


def main():
    X = inputs.two_moons(n=64, seed=0)
    gam = ora.gamma(0.1)
    g = ora.build_graph(X, gam, L=8, seed=0)
    out = {
        "source": "oracle/fsg_oracle.c via tests/golden/make_golden.py",
        "workload": "two_moons(n=64, seed=0), sigma=0.1 (gamma=1/(2 sigma^2)), L=8, seed=0, EXCLUDE, SET",
        "points": X.tolist(),
        "deg": [float(v) for v in g["deg"]],
        "samples": g["samples"].tolist(),
        "src": g["src"].tolist(),
        "dst": g["dst"].tolist(),
        "w": [float(v) for v in g["w"]],
    }
    with open(os.path.join(HERE, "two_moons_64.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
