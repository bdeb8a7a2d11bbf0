"""Pins of the oracle's exact path sampler on the eliminated network (R2:
non-H bits as functions of the previous layer, H outputs fair coins; the
Appendix's elimination of the J-penalty links) against closed forms and
brute force."""
import numpy as np
import pytest

import oracle
from paper_2007_07379_gb300 import workloads as W


def _hmask(g, d):
    m = np.zeros(d, dtype=np.uint32)
    for op, L, q0, _ in g:
        if op == W.H:
            m[L] |= np.uint32(1 << q0)
    return m


def test_every_sample_is_a_valid_path():
    n, d = 5, 8
    g = W.random_circuit(n, d, seed=21)
    r = oracle.elim(n, d, g, seed=3, chains=200, sweeps=7)
    assert r["samples"] == 200 * 7 and r["valid"] == r["samples"]
    assert int(r["cnt"].sum()) == r["samples"]
    assert np.all(oracle.violations(n, d, g, r["state"]) == 0)


def test_paths_uniform_over_the_valid_paths():
    """Each H output is a fair coin and every other bit is determined, so the
    2^h valid paths are equally likely: chi-square over the H outputs of
    independent draws (one per chain)."""
    n, d = 3, 6
    g = W.random_circuit(n, d, seed=8)
    h = int(np.sum(np.asarray(g)[:, 0] == W.H))
    assert 3 <= h <= 8
    chains = 16384
    r = oracle.elim(n, d, g, seed=5, chains=chains, sweeps=1)
    keys = r["state"] & _hmask(g, d)
    uniq, counts = np.unique(keys, axis=0, return_counts=True)
    assert len(uniq) == 2 ** h
    from scipy.stats import chisquare
    assert chisquare(counts).pvalue > 1e-4


def test_amplitudes_within_5_se_of_the_state_vector():
    """i.i.d. uniform valid paths: the estimator of Eq. U23 has the closed-form
    standard error sqrt((N_alpha - |psi|^2) / T), N_alpha = 2^{h - rank}."""
    for n, d, seed in ((3, 4, 0), (4, 6, 11), (5, 5, 4)):
        g = W.random_circuit(n, d, seed)
        exact = oracle.statevector(n, d, g)
        h, rank = oracle.gf2_rank(n, d, g)
        r = oracle.elim(n, d, g, seed=seed + 1, chains=2048, sweeps=100)
        est = oracle.estimate_amplitudes(r["cnt"], r["valid"], h)
        Na = 2.0 ** (h - rank)
        se = np.sqrt(np.maximum(Na - np.abs(exact) ** 2, 0.0) / r["valid"])
        assert np.all(np.abs(est - exact) <= 5 * se + 1e-12), (n, d, seed)


def test_hadamard_chain_se_eq_stdT():
    """Eq. stdT for d Hadamards: std of the |1> amplitude estimate 2^{d/2} /
    sqrt(2T), and no autocorrelation at all (i.i.d. draws)."""
    d = 6
    g = W.hadamard_chain(d)
    per = []
    for c0 in range(0, 1024, 64):
        r = oracle.elim(1, d, g, seed=3, chains=64, chain0=c0, sweeps=100)
        per.append(oracle.estimate_amplitudes(r["cnt"], r["valid"], d)[1])
    per = np.array(per)
    want = 2 ** (d / 2) / np.sqrt(2 * 64 * 100)
    got = np.sqrt(np.mean(np.abs(per) ** 2))  # true value is 0
    # 16 batches: the spread of the chi distribution allows about 30 %
    assert 0.65 * want < got < 1.4 * want


def test_chain_and_sample_ranges_compose():
    """Draws are keyed by the global chain id and the absolute sample index:
    splitting chains or samples reproduces the whole run exactly."""
    n, d = 4, 6
    g = W.random_circuit(n, d, seed=2)
    a = oracle.elim(n, d, g, seed=4, chains=96, sweeps=20)
    parts = [oracle.elim(n, d, g, seed=4, chains=c, chain0=c0, sweeps=20)
             for c0, c in ((0, 40), (40, 56))]
    assert np.array_equal(a["state"], np.concatenate([p["state"] for p in parts]))
    assert np.array_equal(a["cnt"], parts[0]["cnt"] + parts[1]["cnt"])
    b1 = oracle.elim(n, d, g, seed=4, chains=96, sweeps=8)
    b2 = oracle.elim(n, d, g, seed=4, chains=96, sweeps=12, sweep0=8)
    assert np.array_equal(a["cnt"], b1["cnt"] + b2["cnt"])
    assert np.array_equal(a["state"], b2["state"])


def test_record_rule_and_alpha_subset():
    n, d = 4, 5
    g = W.random_circuit(n, d, seed=8)
    r = oracle.elim(n, d, g, seed=1, chains=32, sweeps=20, burn_in=5, record_every=3)
    assert r["samples"] == 32 * len([t for t in range(20) if t >= 5 and (t - 5) % 3 == 0])
    full = oracle.elim(n, d, g, seed=1, chains=64, sweeps=25)
    al = np.array([0, 3, 9, 15], dtype=np.uint32)
    sub = oracle.elim(n, d, g, seed=1, chains=64, sweeps=25, alphas=al)
    assert np.array_equal(sub["cnt"], full["cnt"][al]) and sub["valid"] == full["valid"]


def test_differs_from_the_gibbs_init_stream():
    """The sample stream (tag 4) is not the Gibbs initial-path stream (tag 1)."""
    n, d = 4, 6
    g = W.random_circuit(n, d, seed=5)
    e = oracle.elim(n, d, g, seed=9, chains=64, sweeps=1)
    gi = oracle.gibbs(n, d, g, J=3.0, seed=9, chains=64, sweeps=0)
    assert not np.array_equal(e["state"], gi["state"])


# ---- the output-clamped sampler (end state fixed to alpha, GF(2) elimination)

def _hkeys(g, d, state):
    return state & _hmask(g, d)


def test_clamped_paths_end_at_alpha_and_are_uniform():
    """The paths to alpha form an affine space of dimension h - r: every draw
    is a valid path ending at alpha, the draws are uniform over the 2^{h-r}
    paths (chi-square), and nfree + rank = h with the rank of orc_gf2_rank."""
    n, d = 4, 8
    g = W.random_circuit(n, d, seed=17)
    h, rank = oracle.gf2_rank(n, d, g)
    assert 3 <= h - rank <= 8
    exact = oracle.statevector(n, d, g)
    a = int(np.argmax(np.abs(exact)))
    r = oracle.elim_clamped(n, d, g, alpha=a, seed=2, chains=8192, sweeps=1)
    assert r["consistent"] and r["nfree"] == h - rank and r["rank"] == rank
    assert r["samples"] == 8192
    st = r["state"]
    assert np.all(st[:, d - 1] == a)
    assert np.all(oracle.violations(n, d, g, st) == 0)
    uniq, counts = np.unique(_hkeys(g, d, st), axis=0, return_counts=True)
    assert len(uniq) == 2 ** (h - rank)
    from scipy.stats import chisquare
    assert chisquare(counts).pvalue > 1e-4


def test_clamped_amplitudes_within_5_se():
    """Per sample X = 2^{h/2-r} w^phase with E X = psi_alpha, so
    SE = sqrt((2^{h-2r} - |psi_alpha|^2) / T); an unreachable alpha draws
    nothing and has psi_alpha = 0 exactly."""
    for n, d, seed in ((4, 8, 17), (5, 6, 3), (3, 9, 12)):
        g = W.random_circuit(n, d, seed)
        exact = oracle.statevector(n, d, g)
        h, rank = oracle.gf2_rank(n, d, g)
        for a in range(1 << n):
            r = oracle.elim_clamped(n, d, g, alpha=a, seed=a + 5, chains=256, sweeps=40)
            if not r["consistent"]:
                assert r["samples"] == 0 and abs(exact[a]) < 1e-12
                continue
            est = oracle.clamped_amplitude(r["cnt"], r["samples"], h, rank)
            se = np.sqrt(max(2.0 ** (h - 2 * rank) - abs(exact[a]) ** 2, 0.0) / r["samples"])
            assert abs(est - exact[a]) <= 5 * se + 1e-12, (n, d, seed, a, est, exact[a], se)


def test_clamped_ranges_compose():
    n, d = 4, 8
    g = W.random_circuit(n, d, seed=17)
    a = oracle.elim_clamped(n, d, g, alpha=3, seed=8, chains=80, sweeps=12)
    p1 = oracle.elim_clamped(n, d, g, alpha=3, seed=8, chains=30, sweeps=12)
    p2 = oracle.elim_clamped(n, d, g, alpha=3, seed=8, chains=50, chain0=30, sweeps=12)
    q1 = oracle.elim_clamped(n, d, g, alpha=3, seed=8, chains=80, sweeps=5)
    q2 = oracle.elim_clamped(n, d, g, alpha=3, seed=8, chains=80, sweeps=7, sweep0=5)
    assert np.array_equal(a["cnt"], p1["cnt"] + p2["cnt"])
    assert np.array_equal(a["state"], np.concatenate([p1["state"], p2["state"]]))
    assert np.array_equal(a["cnt"], q1["cnt"] + q2["cnt"])
    assert np.array_equal(a["state"], q2["state"])
