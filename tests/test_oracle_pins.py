"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it pins.  None of them re-types an oracle formula:
they use hand-worked values of the paper, textbook gate identities, a dense
numpy Kronecker-product simulation, closed forms and brute force.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2007_07379_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SQ2 = np.sqrt(2.0)
W8 = np.exp(1j * np.pi / 4)


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11): published known answers.
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# --------------------------------------------------------------------------
# Sec. 4, Eqs. Had / eq2E: the Hadamard pair.
def _gold_hh():
    paths, sums = [], {}
    for l in open(os.path.join(GOLD, "hadamard_pair.txt")):
        if not l.strip() or l.startswith("#"):
            continue
        t = l.split()
        if t[0] == "sum":
            sums[int(t[1])] = int(t[2])
        else:
            paths.append(tuple(int(x) for x in t))
    return paths, sums


def test_hadamard_pair_path_phases():
    g = W.hadamard_chain(2)
    paths, _ = _gold_hh()
    for s1, s2, s3, ph in paths:
        assert oracle.path_phase(1, 2, g, [s2, s3], beta=s1) == ph


def test_hadamard_pair_path_sums():
    g = W.hadamard_chain(2)
    _, sums = _gold_hh()
    cnt, h = oracle.pathsum_exact(1, 2, g)
    assert h == 2
    raw = cnt.astype(float) @ np.exp(1j * np.pi * np.arange(8) / 4)
    for state, val in sums.items():
        assert abs(raw[state] - val) < 1e-12
    # four samples for a net signal of 2 (Sec. 4): four nonzero paths in all
    assert cnt.sum() == 4


def test_eq2E_all_inputs():
    """E = i pi (s1 s2 + s2 s3) holds for both clamped inputs s1 (Eq. eq2E)."""
    g = W.hadamard_chain(2)
    for s1 in (0, 1):
        for s2 in (0, 1):
            for s3 in (0, 1):
                want = (4 * (s1 * s2 + s2 * s3)) % 8
                assert oracle.path_phase(1, 2, g, [s2, s3], beta=s1) == want


# --------------------------------------------------------------------------
# Textbook state vectors.
def _sv(n, rows, beta=0):
    rows = np.asarray(rows, dtype=np.int32).reshape(-1, 4)
    d = int(rows[:, 1].max()) + 1 if len(rows) else 1
    return oracle.statevector(n, d, rows, beta)


def test_single_gates():
    assert np.allclose(_sv(1, [(W.H, 0, 0, -1)]), [1 / SQ2, 1 / SQ2])
    assert np.allclose(_sv(1, [(W.H, 0, 0, -1)], beta=1), [1 / SQ2, -1 / SQ2])
    assert np.allclose(_sv(1, [(W.T, 0, 0, -1)], beta=1), [0, W8])
    assert np.allclose(_sv(1, [(W.S, 0, 0, -1)], beta=1), [0, 1j])
    # T^2 = S, S^2 = Z, H Z H = X
    plus = [(W.H, 0, 0, -1)]
    tt = plus + [(W.T, 1, 0, -1), (W.T, 2, 0, -1)]
    s = plus + [(W.S, 1, 0, -1)]
    assert np.allclose(_sv(1, tt), _sv(1, s))
    ss = plus + [(W.S, 1, 0, -1), (W.S, 2, 0, -1)]
    assert np.allclose(_sv(1, ss), [1 / SQ2, -1 / SQ2])
    hzh = [(W.H, 0, 0, -1), (W.S, 1, 0, -1), (W.S, 2, 0, -1), (W.H, 3, 0, -1)]
    assert np.allclose(_sv(1, hzh), [0, 1])


def test_bell_ghz_and_cnot_convention():
    bell = _sv(2, [(W.H, 0, 0, -1), (W.CNOT, 1, 0, 1)])
    assert np.allclose(bell, [1 / SQ2, 0, 0, 1 / SQ2])
    # control is q0: with q0 = 1 (basis index 1) the target q1 flips -> index 3
    assert np.allclose(_sv(2, [(W.CNOT, 0, 0, 1)], beta=1), [0, 0, 0, 1])
    assert np.allclose(_sv(2, [(W.CNOT, 0, 0, 1)], beta=2), [0, 0, 1, 0])
    ghz = oracle.statevector(3, 3, W.ghz(3))
    want = np.zeros(8, complex)
    want[0] = want[7] = 1 / SQ2
    assert np.allclose(ghz, want)


def test_cz_symmetric():
    pre = [(W.H, 0, 0, -1), (W.H, 0, 1, -1)]
    a = _sv(2, pre + [(W.CZ, 1, 0, 1)])
    b = _sv(2, pre + [(W.CZ, 1, 1, 0)])
    assert np.allclose(a, b)
    assert np.allclose(a, [0.5, 0.5, 0.5, -0.5])


def _dense(n, d, gates, beta=0):
    """Independent simulation with numpy Kronecker products of the textbook
    matrices (qubit q is bit q of the basis index)."""
    Hm = np.array([[1, 1], [1, -1]]) / SQ2
    Sm = np.diag([1, 1j])
    Tm = np.diag([1, W8])
    I2 = np.eye(2)
    N = 1 << n

    def one(q, m):
        out = np.array([[1.0 + 0j]])
        for qq in range(n - 1, -1, -1):  # kron order: highest qubit first
            out = np.kron(out, m if qq == q else I2)
        return out

    psi = np.zeros(N, complex)
    psi[beta] = 1
    for L in range(d):
        U = np.eye(N, dtype=complex)
        for op, layer, q0, q1 in np.asarray(gates):
            if layer != L:
                continue
            if op in (W.H, W.S, W.T):
                G = one(q0, {W.H: Hm, W.S: Sm, W.T: Tm}[op])
            else:
                G = np.zeros((N, N), complex)
                for x in range(N):
                    if op == W.CNOT:
                        y = x ^ (((x >> q0) & 1) << q1)
                        G[y, x] = 1
                    else:
                        G[x, x] = -1 if ((x >> q0) & 1) and ((x >> q1) & 1) else 1
            U = G @ U
        psi = U @ psi
    return psi


@pytest.mark.parametrize("seed", range(6))
def test_statevector_vs_dense_numpy(seed):
    n, d = 4, 6
    g = W.random_circuit(n, d, seed=100 + seed)
    for beta in (0, 5):
        assert np.allclose(oracle.statevector(n, d, g, beta), _dense(n, d, g, beta), atol=1e-12)


@pytest.mark.parametrize("n,d,seed", [(2, 3, 1), (3, 4, 0), (3, 5, 7), (4, 4, 3), (2, 8, 11), (5, 3, 5)])
def test_pathsum_equals_statevector(n, d, seed):
    """Eq. U: the brute-force path sum is the matrix product exactly."""
    g = W.random_circuit(n, d, seed=seed)
    cnt, h = oracle.pathsum_exact(n, d, g)
    psi = oracle.phase_counts_to_complex(cnt, h)
    assert np.abs(psi - oracle.statevector(n, d, g)).max() < 1e-13
    assert abs(np.sum(np.abs(psi) ** 2) - 1) < 1e-12  # norm 1


@pytest.mark.parametrize("n,d,seed", [(8, 10, 1), (12, 20, 1000), (16, 24, 3000)])
def test_statevector_norm(n, d, seed):
    g = W.random_circuit(n, d, seed=seed)
    psi = oracle.statevector(n, d, g)
    assert abs(np.sum(np.abs(psi) ** 2) - 1) < 1e-10


# --------------------------------------------------------------------------
# Closed forms: Eq. stdT and the GF(2) count of valid paths.
@pytest.mark.parametrize("d", [2, 4, 6, 8])
def test_hadamard_chain_structure(d):
    """Sec. 4.1: 2^d paths, half to each output; |0> total 2^{d/2}, |1> total 0
    (peak 1/2^{d/2} of the per-path magnitude 1/2^{d/2} times 2^{d/2})."""
    g = W.hadamard_chain(d)
    cnt, h = oracle.pathsum_exact(1, d, g)
    assert h == d and cnt.sum() == 2 ** d
    assert cnt[0].sum() == cnt[1].sum() == 2 ** (d - 1)
    raw = cnt.astype(float) @ np.exp(1j * np.pi * np.arange(8) / 4)
    assert abs(raw[0] - 2 ** (d / 2)) < 1e-9 and abs(raw[1]) < 1e-9
    assert oracle.gf2_rank(1, d, g) == (d, 1)


@pytest.mark.parametrize("n,d,seed", [(3, 4, 0), (3, 5, 7), (4, 4, 3), (2, 8, 11), (5, 3, 5), (4, 5, 21)])
def test_gf2_count_of_valid_paths(n, d, seed):
    """N_alpha = 2^{h - rank} or 0, against the brute-force count."""
    g = W.random_circuit(n, d, seed=seed)
    cnt, h = oracle.pathsum_exact(n, d, g)
    h2, r = oracle.gf2_rank(n, d, g)
    assert h2 == h
    Na = cnt.sum(axis=1)
    assert set(np.unique(Na)) <= {0, 2 ** (h - r)}
    assert (Na > 0).sum() == 2 ** r


@pytest.mark.parametrize("n,d,seed,beta", [(3, 4, 0, 0), (3, 5, 7, 5), (4, 4, 3, 0), (2, 8, 11, 2),
                                            (5, 3, 5, 0b10110), (4, 5, 21, 9), (5, 4, 7, 0)])
def test_reached_outputs_match_brute_force(n, d, seed, beta):
    """N_alpha of every output (which outputs the valid paths reach, and how
    many paths each) equals the brute-force count of paths per output, with
    and without input bits; the counts add up to the 2^h valid paths."""
    g = W.random_circuit(n, d, seed=seed)
    cnt, h = oracle.pathsum_exact(n, d, g, beta=beta)
    N = oracle.valid_paths_per_output(n, d, g, beta=beta)
    assert np.array_equal(N, cnt.sum(axis=1).astype(float))
    assert N.sum() == 2.0 ** h
    sub = np.array([3, 0, (1 << n) - 1], dtype=np.uint32) % (1 << n)
    assert np.array_equal(oracle.valid_paths_per_output(n, d, g, alphas=sub, beta=beta), N[sub])
    # E|X|^2 >= |E X|^2 for the per-sample estimator 2^{h/2} [end = a] w^phi
    psi = oracle.statevector(n, d, g, beta=beta)
    assert np.all(N + 1e-12 >= np.abs(psi) ** 2)


def test_reached_outputs_of_ghz_and_hadamard_chain():
    """GHZ-6 reaches |000000> and |111111> through one path each; the n = 1
    Hadamard chain reaches both outputs through 2^{d-1} paths each."""
    g = W.ghz(6)
    N = oracle.valid_paths_per_output(6, 6, g)
    assert N[0] == 1 and N[63] == 1 and N.sum() == 2
    N = oracle.valid_paths_per_output(1, 6, W.hadamard_chain(6))
    assert list(N) == [32.0, 32.0]


# --------------------------------------------------------------------------
def test_thresholds_high_precision():
    sympy = pytest.importorskip("sympy")
    for J in (0.5, 1.0, 4.0, 5.7, 9.25):
        thr = oracle.thresholds(J)
        assert thr[0] == 2 ** 31
        for v in (1, 2, 3):
            exact = sympy.floor(sympy.Integer(2) ** 32 / (1 + sympy.exp(sympy.Float(J, 50) * v)))
            assert int(thr[v]) == int(exact)


@pytest.mark.parametrize("n,d,seed", [(3, 4, 0), (4, 4, 3), (4, 5, 21), (3, 6, 9)])
def test_colour_classes_share_no_factor(n, d, seed):
    """Two p-bits of one colour never interact: the violation count (Re E / J)
    has no cross term in them, for every state of the remaining bits."""
    g = W.random_circuit(n, d, seed=seed)
    col = oracle.colour(n, d, g)
    rng = np.random.default_rng(seed)
    states = rng.integers(0, 1 << n, size=(64, d), dtype=np.uint32)
    pbits = [(k, q) for k in range(1, d + 1) for q in range(n)]
    for i, (k1, q1) in enumerate(pbits):
        for (k2, q2) in pbits[i + 1:]:
            if col[k1 - 1, q1] != col[k2 - 1, q2]:
                continue
            es = []
            for b1 in (0, 1):
                for b2 in (0, 1):
                    st = states.copy()
                    st[:, k1 - 1] = (st[:, k1 - 1] & ~np.uint32(1 << q1)) | np.uint32(b1 << q1)
                    st[:, k2 - 1] = (st[:, k2 - 1] & ~np.uint32(1 << q2)) | np.uint32(b2 << q2)
                    es.append(oracle.violations(n, d, g, st).astype(np.int64))
            assert np.all(es[3] - es[2] - es[1] + es[0] == 0), ((k1, q1), (k2, q2))
