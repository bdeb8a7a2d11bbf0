"""The stored top-16 amplitudes of the learned workloads
(tests/golden/learned_top16.json, read by the benchmark's error-versus-time
measurement) are the oracle's: regenerating them gives the same file."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_learned_top16_matches_the_oracle():
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "golden", "make_learned_top16.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    want = mk.build()
    with open(os.path.join(HERE, "golden", "learned_top16.json")) as f:
        got = json.load(f)
    for name in ("learned", "learned_sparse"):
        assert got[name]["alphas"] == want[name]["alphas"]
        assert np.array_equal(got[name]["re"], want[name]["re"])
        assert np.array_equal(got[name]["im"], want[name]["im"])
        mags = np.hypot(got[name]["re"], got[name]["im"])
        assert np.all(np.diff(mags) <= 1e-15)  # largest first
