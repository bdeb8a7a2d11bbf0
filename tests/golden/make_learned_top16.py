"""Writes learned_top16.json: the 16 outputs of largest |psi_alpha| of the
learned workload's circuit (n=16, d=24) and of its one-gate-per-layer
variant, with their exact amplitudes from the FP64 state vector (oracle),
for the benchmark's error-versus-time measurement (error = the largest
|psi_hat - psi| over these 16 outputs).

    python tests/golden/make_learned_top16.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2007_07379_gb300 import workloads as W  # noqa: E402


def top16(wl):
    psi = oracle.statevector(wl.n, wl.d, wl.gates)
    idx = np.argsort(-np.abs(psi), kind="stable")[:16]
    return {"n": wl.n, "d": wl.d, "alphas": [int(a) for a in idx],
            "re": [float(psi[a].real) for a in idx], "im": [float(psi[a].imag) for a in idx]}


def build() -> dict:
    return {"source": "oracle.statevector (FP64), 16 largest |psi_alpha|",
            "learned": top16(W.learned()), "learned_sparse": top16(W.learned_sparse())}


if __name__ == "__main__":
    with open(os.path.join(HERE, "learned_top16.json"), "w") as f:
        json.dump(build(), f, indent=1)
        f.write("\n")
