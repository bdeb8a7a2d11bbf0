"""Pins of the oracle's reference Gibbs sampler (Fig. 2 flowchart, J-penalty
form of the Appendix) against closed forms and brute force."""
import numpy as np
import pytest

import oracle
from paper_2007_07379_gb300 import workloads as W


def _h(g):
    return int(np.sum(np.asarray(g)[:, 0] == W.H))


def test_valid_fraction_closed_form():
    """Stationary law: with error bits e = s XOR (deterministic value), the
    energy is J * sum(e), so each of the M linked bits is wrong independently
    with probability 1/(1+e^J): P(valid) = (1 + e^{-J})^{-M}."""
    n, d = 3, 4
    g = W.random_circuit(n, d, seed=0)
    J = 2.0
    M = n * d - _h(g)
    chains, sweeps = 8192, 40
    r = oracle.gibbs(n, d, g, J=J, seed=11, chains=chains, sweeps=sweeps, burn_in=sweeps - 1)
    assert r["samples"] == chains
    p = (1 + np.exp(-J)) ** (-M)
    se = np.sqrt(p * (1 - p) / chains)
    assert abs(r["valid"] / chains - p) < 5 * se


def test_valid_paths_uniform():
    """Valid paths are equally likely (all have Re E = 0): chi-square over the
    2^h valid paths of the final states."""
    n, d = 3, 5
    g = W.random_circuit(n, d, seed=7)
    h = _h(g)
    assert h >= 3
    chains = 8192
    r = oracle.gibbs(n, d, g, J=2.5, seed=5, chains=chains, sweeps=30)
    st = r["state"]
    ok = oracle.violations(n, d, g, st) == 0
    # a valid path is identified by its H outputs
    hmask = np.zeros(d, dtype=np.uint32)
    for op, L, q0, _ in g:
        if op == W.H:
            hmask[L] |= np.uint32(1 << q0)
    keys = [tuple(row & hmask) for row in st[ok]]
    uniq, counts = np.unique(np.array(keys), axis=0, return_counts=True)
    assert len(uniq) == 2 ** h
    from scipy.stats import chisquare
    assert chisquare(counts).pvalue > 1e-4


def test_amplitudes_within_5_se_tiny():
    """Eq. U23 with p_C uniform over valid paths converges to the exact U."""
    wl = W.tiny()
    n, d, g = wl.n, wl.d, wl.gates
    exact = oracle.statevector(n, d, g)
    h, rank = oracle.gf2_rank(n, d, g)
    r = oracle.gibbs(n, d, g, J=wl.J, seed=wl.seed, chains=256, sweeps=2000)
    est = oracle.estimate_amplitudes(r["cnt"], r["valid"], h)
    Na = 2.0 ** (h - rank)
    se = np.sqrt(np.maximum(Na - np.abs(exact) ** 2, 1e-12) / r["valid"])
    # autocorrelation inflates the i.i.d. SE; allow a factor 3 for it
    assert np.all(np.abs(est - exact) < 5 * 3 * se + 1e-12)


def test_hadamard_chain_se_eq_stdT():
    """Eq. stdT: for d Hadamards (all p-bits free, i.i.d. sweeps) the estimate
    of the |1> amplitude has std 2^{d/2} / sqrt(2T)."""
    d = 6
    g = W.hadamard_chain(d)
    chains, sweeps = 512, 200
    per = []
    for c0 in range(0, chains, 64):
        r = oracle.gibbs(1, d, g, J=3.0, seed=3, chains=64, chain0=c0, sweeps=sweeps)
        per.append(oracle.estimate_amplitudes(r["cnt"], r["valid"], d)[1])
    per = np.array(per)
    T = 64 * sweeps
    want = 2 ** (d / 2) / np.sqrt(2 * T)
    got = np.sqrt(np.mean(np.abs(per) ** 2))  # true value is 0
    # 8 batches: the chi distribution of the spread allows about 40 %
    assert 0.55 * want < got < 1.6 * want


def test_resume_is_bit_identical():
    n, d = 4, 6
    g = W.random_circuit(n, d, seed=3)
    a = oracle.gibbs(n, d, g, J=3.0, seed=9, chains=64, sweeps=30)
    b1 = oracle.gibbs(n, d, g, J=3.0, seed=9, chains=64, sweeps=12)
    b2 = oracle.gibbs(n, d, g, J=3.0, seed=9, chains=64, sweeps=18, sweep0=12, state=b1["state"])
    assert np.array_equal(a["state"], b2["state"])
    assert np.array_equal(a["cnt"], b1["cnt"] + b2["cnt"])
    assert a["valid"] == b1["valid"] + b2["valid"]


def test_chain_ranges_compose():
    """Chains are independent streams keyed by their global id, so a split
    over chain ranges (the multi-rank sharding) reproduces the whole run."""
    n, d = 3, 5
    g = W.random_circuit(n, d, seed=2)
    a = oracle.gibbs(n, d, g, J=3.0, seed=4, chains=96, sweeps=20)
    parts = [oracle.gibbs(n, d, g, J=3.0, seed=4, chains=c, chain0=c0, sweeps=20)
             for c0, c in ((0, 40), (40, 56))]
    assert np.array_equal(a["state"], np.concatenate([p["state"] for p in parts]))
    assert np.array_equal(a["cnt"], parts[0]["cnt"] + parts[1]["cnt"])


def test_alpha_subset_matches_full_histogram():
    n, d = 4, 5
    g = W.random_circuit(n, d, seed=8)
    full = oracle.gibbs(n, d, g, J=3.0, seed=1, chains=64, sweeps=25)
    al = np.array([0, 3, 9, 15], dtype=np.uint32)
    sub = oracle.gibbs(n, d, g, J=3.0, seed=1, chains=64, sweeps=25, alphas=al)
    assert np.array_equal(sub["cnt"], full["cnt"][al])
    assert sub["valid"] == full["valid"]
