"""Pins of the oracle's general one-qubit-gate functions (Sec. 2 Eq. EB,
Sec. 4.2 Eq. HadT, Fig. 5) against closed forms, independent matrix
products, brute force and the already pinned Clifford+T oracle."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2007_07379_gb300 import workloads as W


def _kron_unitary(n, d, gates, mats, mats2=None):
    """Full 2^n x 2^n circuit matrix from numpy products of per-gate
    embeddings (basis index bit q = qubit q), independent of the oracle."""
    N = 1 << n
    std = {W.H: np.array([[1, 1], [1, -1]]) / np.sqrt(2), W.S: np.diag([1, 1j]),
           W.T: np.diag([1, np.exp(1j * np.pi / 4)]), W.X: np.array([[0, 1], [1, 0]])}
    Utot = np.eye(N, dtype=np.complex128)
    for layer in range(d):
        for i, (op, L, q0, q1) in enumerate(gates):
            if L != layer:
                continue
            G = np.zeros((N, N), dtype=np.complex128)
            for x in range(N):
                if op in (W.H, W.S, W.T, W.U, W.X):
                    m = mats[i] if op == W.U else std[op]
                    for yb in (0, 1):
                        y = (x & ~(1 << q0)) | (yb << q0)
                        G[y, x] += m[yb, (x >> q0) & 1]
                elif op == W.U2:
                    xl = ((x >> q0) & 1) | (((x >> q1) & 1) << 1)
                    for yl in range(4):
                        y = (x & ~(1 << q0) & ~(1 << q1)) | ((yl & 1) << q0) | ((yl >> 1) << q1)
                        G[y, x] += mats2[i][yl, xl]
                elif op == W.CNOT:
                    y = x ^ ((((x >> q0) & 1)) << q1)
                    G[y, x] = 1
                elif op == W.CZ:
                    G[x, x] = -1 if ((x >> q0) & 1) and ((x >> q1) & 1) else 1
            Utot = G @ Utot
    return Utot


def _path_weights(n, d, gates, mats, beta=0):
    """|U_C| of every path (s_1..s_d) by direct products (tests' own)."""
    out = {}
    per_layer = []
    for L in range(d):
        gl = [(i, r) for i, r in enumerate(gates) if r[1] == L]
        sub = np.array([r for _, r in gl], dtype=np.int32).reshape(-1, 4).copy()
        sub[:, 1] = 0
        m = np.stack([mats[i] for i, _ in gl]) if gl else np.zeros((0, 2, 2))
        per_layer.append(_kron_unitary(n, 1, sub, m))
    for path in itertools.product(range(1 << n), repeat=d):
        w = 1.0 + 0j
        prev = beta
        for L, s in enumerate(path):
            w *= per_layer[L][s, prev]
            prev = s
        if abs(w) > 0:
            out[path] = w
    return out


def test_statevector_matches_clifford_t_oracle():
    for n, d, seed in ((3, 6, 1), (5, 4, 2), (4, 8, 9)):
        g = W.random_circuit(n, d, seed)
        mats = np.zeros((len(g), 2, 2), dtype=np.complex128)
        assert np.allclose(oracle.u_statevector(n, d, g, mats), oracle.statevector(n, d, g),
                           atol=1e-12)


@pytest.mark.parametrize("theta", [0.1, 0.3, np.pi / 4, 1.2, np.pi / 2 - 0.01])
def test_rotated_h_chain_closed_form(theta):
    """RH(t)^2 = I, so an even chain returns |0> and an odd one gives
    (cos t, sin t)."""
    for d in (1, 2, 5, 6):
        g, m = W.rotated_h_chain(d, theta)
        psi = oracle.u_statevector(1, d, g, m)
        want = np.array([1.0, 0.0]) if d % 2 == 0 else np.array([np.cos(theta), np.sin(theta)])
        assert np.allclose(psi, want, atol=1e-12)


def test_u3_convention_rows_are_outputs():
    t, ph, la = 0.7, 1.1, -0.4
    g = np.array([[W.U, 0, 0, -1]], dtype=np.int32)
    m = W.u3(t, ph, la)[None]
    assert np.allclose(oracle.u_statevector(1, 1, g, m, beta=0),
                       [np.cos(t / 2), np.exp(1j * ph) * np.sin(t / 2)], atol=1e-14)
    assert np.allclose(oracle.u_statevector(1, 1, g, m, beta=1),
                       [-np.exp(1j * la) * np.sin(t / 2), np.exp(1j * (ph + la)) * np.cos(t / 2)],
                       atol=1e-14)


def test_statevector_against_matrix_products():
    for n, d, seed in ((2, 5, 3), (3, 6, 11), (4, 5, 5)):
        g, m = W.random_general_circuit(n, d, seed, frac_u=0.6)
        assert np.sum(g[:, 0] == W.U) >= 2
        want = _kron_unitary(n, d, g, m)[:, 0]
        assert np.allclose(oracle.u_statevector(n, d, g, m), want, atol=1e-12)


def test_path_sum_equals_state_vector():
    for n, d, seed in ((2, 5, 3), (3, 4, 12), (1, 9, 4)):
        g, m = W.random_general_circuit(n, d, seed, frac_u=0.7)
        ps = oracle.u_pathstats(n, d, g, m)
        assert np.allclose(ps["U"], oracle.u_statevector(n, d, g, m), atol=1e-12)


@pytest.mark.parametrize("theta", [0.2, 0.6, np.pi / 4, 1.3])
def test_rotated_chain_sums(theta):
    """Every column of |RH| sums to |cos|+|sin|: sum_C |U_C| = (|c|+|s|)^d,
    2^{d-1} paths reach each output, and log2 Z matches."""
    d = 8
    g, m = W.rotated_h_chain(d, theta)
    ps = oracle.u_pathstats(1, d, g, m)
    c, s = abs(np.cos(theta)), abs(np.sin(theta))
    assert np.isclose(ps["zabs"].sum(), (c + s) ** d, rtol=1e-12)
    assert np.all(ps["npath"] == 2 ** (d - 1))
    assert np.isclose(oracle.u_log2z(1, d, g, m), d * np.log2(c + s), rtol=1e-12)


def test_fig5_prefactor_pins():
    """d = 10 rotated Hadamards: at t = pi/4 the paths to |1> have equal
    magnitude and cancel, std = 2^{d/2} / 2 (the prefactor behind Eq. stdT),
    weighted and uniform alike; at t = pi/2 (classical) a single path
    survives and std vanishes; weighted never exceeds uniform
    (Cauchy-Schwarz, Fig. 5)."""
    d = 10
    g, m = W.rotated_h_chain(d, np.pi / 4)
    ps = oracle.u_pathstats(1, d, g, m)
    assert np.isclose(ps["std_weighted"][1], 2 ** (d / 2) / 2, rtol=1e-12)
    assert np.isclose(ps["std_uniform"][1], 2 ** (d / 2) / 2, rtol=1e-12)
    assert abs(ps["U"][1]) < 1e-12 and np.isclose(abs(ps["U"][0]), 1.0)
    g, m = W.rotated_h_chain(d, np.pi / 2)
    ps = oracle.u_pathstats(1, d, g, m)
    assert np.all(ps["std_weighted"] < 1e-6)
    for th in np.linspace(0.05, np.pi / 2 - 0.05, 12):
        g, m = W.rotated_h_chain(d, th)
        ps = oracle.u_pathstats(1, d, g, m)
        assert np.all(ps["std_weighted"] <= ps["std_uniform"] + 1e-9)
    # away from pi/4 weighting helps strictly on the |1> output
    g, m = W.rotated_h_chain(d, 0.3)
    ps = oracle.u_pathstats(1, d, g, m)
    assert ps["std_weighted"][1] < 0.9 * ps["std_uniform"][1]


def test_gibbs_reduces_to_clifford_t_sampler():
    """Without U gates the general sampler is the pinned orc_gibbs: the same
    states, the per-output counts, and phase sums equal to sum cnt w^b."""
    w = np.exp(1j * np.pi * np.arange(8) / 4)
    for n, d, seed in ((3, 5, 2), (5, 8, 21)):
        g = W.random_circuit(n, d, seed)
        mats = np.zeros((len(g), 2, 2))
        J = W.default_J(n, d, g)
        a = oracle.gibbs(n, d, g, J=J, seed=5, chains=96, sweeps=40)
        b = oracle.u_gibbs(n, d, g, mats, J=J, seed=5, chains=96, sweeps=40)
        assert np.array_equal(a["state"], b["state"])
        assert np.array_equal(a["cnt"].sum(axis=1), b["cnt"])
        assert a["valid"] == b["valid"] and a["samples"] == b["samples"]
        assert np.allclose(a["cnt"].astype(np.float64) @ w, b["sum"], atol=1e-9)
        h = int(np.sum(g[:, 0] == W.H))
        assert b["log2z"] == 0.5 * h


def test_rotated_pi4_chain_reproduces_hadamard_chain():
    """RH(pi/4) is H: K = ln(cos/sin) is one rounding away from 0, so the
    Metropolis step accepts (barring a 2^-32 draw) and the chain follows the
    H chain's proposals exactly."""
    d = 6
    g, m = W.rotated_h_chain(d, np.pi / 4)
    a = oracle.gibbs(1, d, W.hadamard_chain(d), J=2.0, seed=9, chains=128, sweeps=60)
    b = oracle.u_gibbs(1, d, g, m, J=2.0, seed=9, chains=128, sweeps=60)
    assert np.array_equal(a["state"], b["state"])
    assert np.array_equal(a["cnt"].sum(axis=1), b["cnt"])


def _batch_estimates(fn, n, d, g, m, nb, per, **kw):
    ests = []
    for b in range(nb):
        r = fn(n, d, g, m, chain0=b * per, chains=per, **kw)
        ests.append(oracle.u_estimate(r))
    ests = np.array(ests)
    return ests.mean(axis=0), ests.std(axis=0, ddof=1) / np.sqrt(nb)


@pytest.mark.parametrize("case", ["rotated", "general3", "general2"])
def test_gibbs_converges_to_state_vector(case):
    if case == "rotated":
        n, d = 1, 6
        g, m = W.rotated_h_chain(d, 0.35)
    elif case == "general3":
        n, d = 3, 5
        g, m = W.random_general_circuit(n, d, 7, frac_u=0.6)
    else:
        n, d = 2, 6
        g, m = W.random_general_circuit(n, d, 3, frac_u=0.7)
    exact = oracle.u_statevector(n, d, g, m)
    J = 3.0
    est, se = _batch_estimates(oracle.u_gibbs, n, d, g, m, 16, 64, J=J, seed=11, sweeps=600,
                               burn_in=50)
    assert np.all(np.abs(est - exact) <= 5 * np.maximum(se, 1e-3)), (est, exact, se)


def _path_index(state, n):
    idx = np.zeros(state.shape[0], dtype=np.int64)
    for k in range(state.shape[1]):
        idx = idx * (1 << n) + state[:, k].astype(np.int64)
    return idx


@pytest.mark.parametrize("theta", [0.4, 1.0])
def test_gibbs_stationary_law_is_abs_weight(theta):
    """Metropolis sign pin: after burn-in the chains' paths follow
    p_C = |U_C| / sum |U_C| (chi-square over the 8 paths of d = 3)."""
    from scipy.stats import chisquare
    d = 3
    g, m = W.rotated_h_chain(d, theta)
    pw = _path_weights(1, d, g, m)
    keys = sorted(pw)
    p = np.array([abs(pw[k]) for k in keys])
    p /= p.sum()
    r = oracle.u_gibbs(1, d, g, m, J=3.0, seed=4, chains=20000, sweeps=25)
    idx = _path_index(r["state"], 1)
    want_idx = np.array([_path_index(np.array([k]), 1)[0] for k in keys])
    counts = np.array([np.sum(idx == w) for w in want_idx])
    assert counts.sum() == 20000
    assert chisquare(counts, p * 20000).pvalue > 1e-4


def test_gibbs_stationary_law_with_links():
    """Two qubits with a CNOT and J-linked wires: the valid paths among the
    final states follow |U_C| restricted to valid paths."""
    from scipy.stats import chisquare
    n, d = 2, 3
    g = np.array([[W.U, 0, 0, -1], [W.H, 0, 1, -1], [W.CNOT, 1, 0, 1], [W.U, 2, 1, -1]],
                 dtype=np.int32)
    m = np.zeros((4, 2, 2), dtype=np.complex128)
    m[0] = W.u3(0.9, 0.3, 1.7)
    m[3] = W.rotated_h(0.5)
    pw = _path_weights(n, d, g, m)
    keys = sorted(pw)
    p = np.array([abs(pw[k]) for k in keys])
    p /= p.sum()
    # J-linked paths mix slowly (a move between valid paths crosses invalid
    # ones); 400 sweeps at J = 2 forget the uniform initial law
    r = oracle.u_gibbs(n, d, g, m, J=2.0, seed=2, chains=30000, sweeps=400)
    idx = _path_index(r["state"], n)
    key_idx = np.array([_path_index(np.array([k]), n)[0] for k in keys])
    counts = np.array([np.sum(idx == w) for w in key_idx])
    assert counts.sum() > 0.3 * 30000
    assert chisquare(counts, p * counts.sum()).pvalue > 1e-4


def test_elim_law_and_validity():
    from scipy.stats import chisquare
    n, d = 2, 3
    g = np.array([[W.U, 0, 0, -1], [W.H, 0, 1, -1], [W.CNOT, 1, 0, 1], [W.U, 2, 1, -1]],
                 dtype=np.int32)
    m = np.zeros((4, 2, 2), dtype=np.complex128)
    m[0] = W.u3(0.9, 0.3, 1.7)
    m[3] = W.rotated_h(0.5)
    pw = _path_weights(n, d, g, m)
    keys = sorted(pw)
    p = np.array([abs(pw[k]) for k in keys])
    assert np.isclose(p.sum(), 2 ** oracle.u_log2z(n, d, g, m), rtol=1e-12)
    p /= p.sum()
    r = oracle.u_elim(n, d, g, m, seed=6, chains=20000, sweeps=1)
    assert r["valid"] == r["samples"] == 20000
    idx = _path_index(r["state"], n)
    key_idx = np.array([_path_index(np.array([k]), n)[0] for k in keys])
    counts = np.array([np.sum(idx == w) for w in key_idx])
    assert counts.sum() == 20000
    assert chisquare(counts, p * 20000).pvalue > 1e-4


@pytest.mark.parametrize("n,d,seed", [(3, 5, 7), (2, 6, 3), (4, 4, 1)])
def test_elim_se_closed_form(n, d, seed):
    """i.i.d. draws with p_C = |U_C| / Z: X = Z e^{i arg U_C} [end = alpha]
    has Var X = Z Z_alpha - |U_alpha|^2."""
    g, m = W.random_general_circuit(n, d, seed, frac_u=0.6)
    exact = oracle.u_statevector(n, d, g, m)
    ps = oracle.u_pathstats(n, d, g, m)
    r = oracle.u_elim(n, d, g, m, seed=seed + 3, chains=2048, sweeps=60)
    Z = 2 ** r["log2z"]
    assert np.isclose(Z, ps["zabs"].sum(), rtol=1e-12)
    se = np.sqrt(np.maximum(Z * ps["zabs"] - np.abs(exact) ** 2, 0) / r["samples"])
    assert np.all(np.abs(oracle.u_estimate(r) - exact) <= 5 * se + 1e-12)


def test_diagonal_and_antidiagonal_gates():
    """A diagonal U is a J-linked copy with its phase (H Rz H: amplitudes
    (1 +- e^{i phi}) / 2 up to the gate's global phase), an anti-diagonal U
    a J-linked NOT."""
    phi = 0.77
    g = np.array([[W.H, 0, 0, -1], [W.U, 1, 0, -1], [W.H, 2, 0, -1]], dtype=np.int32)
    m = np.zeros((3, 2, 2), dtype=np.complex128)
    m[1] = np.diag([1.0, np.exp(1j * phi)])
    want = np.array([(1 + np.exp(1j * phi)) / 2, (1 - np.exp(1j * phi)) / 2])
    assert np.allclose(oracle.u_statevector(1, 3, g, m), want, atol=1e-14)
    r = oracle.u_elim(1, 3, g, m, seed=1, chains=4096, sweeps=20)
    se = np.sqrt(np.maximum(2 * 2 - np.abs(want) ** 2, 0) / r["samples"])  # Z = 2, Z_alpha <= 2
    assert np.all(np.abs(oracle.u_estimate(r) - want) <= 5 * se)
    x = np.array([[W.U, 0, 0, -1], [W.U, 1, 0, -1]], dtype=np.int32)
    mx = np.stack([np.array([[0, 1], [1, 0]], dtype=np.complex128),
                   np.array([[0, 1j], [1j, 0]], dtype=np.complex128)])
    assert np.allclose(oracle.u_statevector(1, 2, x[:1], mx[:1]), [0, 1])
    assert np.allclose(oracle.u_statevector(1, 2, x, mx), [1j, 0])
    r = oracle.u_gibbs(1, 2, x, mx, J=5.0, seed=3, chains=512, sweeps=100)
    est = oracle.u_estimate(r)
    assert np.allclose(est, [1j, 0], atol=1e-12)  # one valid path, phase i


def test_rejects_bad_matrices():
    g = np.array([[W.U, 0, 0, -1]], dtype=np.int32)
    for bad in (np.array([[1, 0], [0, 2]]), np.array([[1, 1], [1, 1]]) / 2,
                np.array([[0, 1], [1, 1]]) / np.sqrt(2)):
        with pytest.raises(ValueError):
            oracle.u_statevector(1, 1, g, bad[None].astype(np.complex128))



# ---- X and two-qubit permutations with phases (U2)

def test_two_qubit_gates_against_matrix_products():
    for n, d, seed in ((2, 4, 1), (3, 6, 3), (4, 6, 8), (5, 5, 11)):
        g, m2 = W.random_two_qubit_circuit(n, d, seed, frac=0.9)
        assert np.sum(g[:, 0] == W.U2) >= 1
        want = _kron_unitary(n, d, g, None, m2)[:, 0]
        assert np.allclose(oracle.u_statevector(n, d, g, None, mats2=m2), want, atol=1e-12)
        ps = oracle.u_pathstats(n, d, g, None, mats2=m2) if n * d <= 24 else None
        if ps is not None:
            assert np.allclose(ps["U"], want, atol=1e-12)


def test_exchange_operator_closed_form():
    """H on both qubits, then J12(g): amplitudes (1/2) e^{i g/2 (1-2 s1)(1-2 s2)}
    (the Appendix's energy of the exchange operator)."""
    gam = 0.83
    g = np.array([[W.H, 0, 0, -1], [W.H, 0, 1, -1], [W.U2, 1, 0, 1]], dtype=np.int32)
    m2 = np.zeros((3, 4, 4), dtype=np.complex128)
    m2[2] = W.exchange_matrix(gam)
    s1 = np.array([0, 1, 0, 1]); s2 = np.array([0, 0, 1, 1])
    want = 0.5 * np.exp(0.5j * gam * (1 - 2 * s1) * (1 - 2 * s2))
    assert np.allclose(oracle.u_statevector(2, 2, g, None, mats2=m2), want, atol=1e-14)


def test_u2_as_cnot_and_cz_reproduces_the_clifford_t_sampler():
    """A U2 holding the CNOT (or CZ) matrix has the same links, colouring and
    draws as the CNOT (CZ) gate: identical chain states; its phases equal the
    exact phase classes."""
    w = np.exp(1j * np.pi * np.arange(8) / 4)
    for n, d, seed in ((4, 6, 5), (6, 8, 21)):
        g = W.random_circuit(n, d, seed)
        gu = g.copy()
        m2 = np.zeros((len(g), 4, 4), dtype=np.complex128)
        for i in range(len(g)):
            if g[i, 0] == W.CNOT:
                gu[i, 0] = W.U2
                m2[i] = W.cnot_matrix(True)
            elif g[i, 0] == W.CZ:
                gu[i, 0] = W.U2
                m2[i] = np.diag([1, 1, 1, -1])
        assert np.sum(gu[:, 0] == W.U2) > 0
        assert np.array_equal(oracle.u_colour(n, d, gu, None, m2), oracle.colour(n, d, g))
        J = W.default_J(n, d, g)
        a = oracle.gibbs(n, d, g, J=J, seed=3, chains=96, sweeps=30)
        b = oracle.u_gibbs(n, d, gu, None, J=J, seed=3, chains=96, sweeps=30, mats2=m2)
        assert np.array_equal(a["state"], b["state"])
        assert np.array_equal(a["cnt"].sum(axis=1), b["cnt"])
        assert np.allclose(a["cnt"].astype(np.float64) @ w, b["sum"], atol=1e-9)


def test_u_colour_matches_the_clifford_t_colouring():
    for n, d, seed in ((3, 5, 2), (8, 12, 7), (12, 20, 1000)):
        g = W.random_circuit(n, d, seed)
        assert np.array_equal(oracle.u_colour(n, d, g), oracle.colour(n, d, g))


@pytest.mark.parametrize("n,d,seed", [(3, 5, 4), (4, 4, 9), (2, 6, 13)])
def test_two_qubit_circuits_converge(n, d, seed):
    g, m2 = W.random_two_qubit_circuit(n, d, seed, frac=0.9)
    exact = oracle.u_statevector(n, d, g, None, mats2=m2)
    ests = []
    for b in range(16):
        r = oracle.u_gibbs(n, d, g, None, J=3.0, seed=21, chains=64, chain0=64 * b, sweeps=500,
                           burn_in=50, mats2=m2)
        ests.append(oracle.u_estimate(r))
    ests = np.array(ests)
    est, se = ests.mean(axis=0), ests.std(axis=0, ddof=1) / 4
    assert np.all(np.abs(est - exact) <= 5 * np.maximum(se, 1e-3)), (est, exact, se)
    e = oracle.u_elim(n, d, g, None, seed=5, chains=2048, sweeps=40, mats2=m2)
    ps = oracle.u_pathstats(n, d, g, None, mats2=m2)
    Z = 2 ** e["log2z"]
    se_e = np.sqrt(np.maximum(Z * ps["zabs"] - np.abs(exact) ** 2, 0) / e["samples"])
    assert np.all(np.abs(oracle.u_estimate(e) - exact) <= 5 * se_e + 1e-12)


def test_rejects_unrepresentable_two_qubit_gates():
    g = np.array([[W.U2, 0, 0, 1]], dtype=np.int32)
    bad = []
    # output q0 = NOT(x1 XOR x2): y = (1 ^ x1 ^ x2) | x2 << 1
    m = np.zeros((4, 4), dtype=np.complex128)
    for x in range(4):
        x1, x2 = x & 1, x >> 1
        m[(1 ^ x1 ^ x2) | (x2 << 1), x] = 1
    bad.append(m)
    bad.append(2 * W.swap_matrix())  # not unitary
    for b in bad:
        with pytest.raises(ValueError):
            oracle.u_statevector(2, 1, g, None, mats2=b[None])



# ---- the Toffoli gate (CCX)

def _ccx_unitary(n, d, gates):
    """Circuit matrix with the CCX gates (rows (op, layer, q0, q1, q2))
    embedded directly; other gates through _kron_unitary, layer by layer."""
    N = 1 << n
    Utot = np.eye(N, dtype=np.complex128)
    for layer in range(d):
        lg = [r for r in gates if r[1] == layer]
        rest = np.array([r[:4] for r in lg if r[0] != W.CCX], dtype=np.int32).reshape(-1, 4).copy()
        rest[:, 1] = 0
        Utot = _kron_unitary(n, 1, rest, None) @ Utot
        for r in lg:
            if r[0] != W.CCX:
                continue
            G = np.zeros((N, N))
            for x in range(N):
                y = x ^ ((((x >> r[2]) & 1) & ((x >> r[3]) & 1)) << r[4])
                G[y, x] = 1
            Utot = G @ Utot
    return Utot


def test_ccx_truth_table():
    g = np.array([[W.CCX, 0, 0, 1, 2]], dtype=np.int32)
    for beta in range(8):
        want = np.zeros(8)
        want[beta ^ (4 if (beta & 1) and (beta & 2) else 0)] = 1
        assert np.allclose(oracle.u_statevector(3, 1, g, None, beta=beta), want)


@pytest.mark.parametrize("n,d,seed", [(3, 4, 1), (4, 5, 2), (5, 6, 7), (6, 4, 11)])
def test_ccx_circuits_against_matrix_products(n, d, seed):
    g = W.random_ccx_circuit(n, d, seed, frac=0.9)
    assert np.sum(g[:, 0] == W.CCX) >= 1
    want = _ccx_unitary(n, d, g)[:, 0]
    assert np.allclose(oracle.u_statevector(n, d, g, None), want, atol=1e-12)
    if n * d <= 24:
        assert np.allclose(oracle.u_pathstats(n, d, g, None)["U"], want, atol=1e-12)


@pytest.mark.parametrize("n,d,seed", [(4, 5, 2), (5, 6, 7), (8, 10, 3), (12, 20, 1000)])
def test_ccx_colouring_is_proper(n, d, seed):
    """No two p-bits of one colour class share a factor (a Toffoli target's
    factor holds four p-bits)."""
    g = W.random_ccx_circuit(n, d, seed, frac=0.7)
    col = oracle.u_colour(n, d, g)
    for r in g:
        if r[0] != W.CCX or r[1] == 0:
            continue
        k = r[1]  # p-bits (k, q) are row k - 1
        fac = [col[k, r[4]], col[k - 1, r[4]], col[k - 1, r[2]], col[k - 1, r[3]]]
        assert len(set(fac)) == 4


@pytest.mark.parametrize("n,d,seed", [(3, 4, 1), (4, 5, 2), (5, 4, 9)])
def test_ccx_circuits_converge(n, d, seed):
    g = W.random_ccx_circuit(n, d, seed, frac=0.9)
    exact = oracle.u_statevector(n, d, g, None)
    ests = []
    for b in range(16):
        r = oracle.u_gibbs(n, d, g, None, J=3.0, seed=31, chains=64, chain0=64 * b, sweeps=500,
                           burn_in=50)
        ests.append(oracle.u_estimate(r))
    ests = np.array(ests)
    est, se = ests.mean(axis=0), ests.std(axis=0, ddof=1) / 4
    assert np.all(np.abs(est - exact) <= 5 * np.maximum(se, 1e-3)), (est, exact, se)
    e = oracle.u_elim(n, d, g, None, seed=5, chains=2048, sweeps=40)
    ps = oracle.u_pathstats(n, d, g, None)
    Z = 2 ** e["log2z"]
    se_e = np.sqrt(np.maximum(Z * ps["zabs"] - np.abs(exact) ** 2, 0) / e["samples"])
    assert np.all(np.abs(oracle.u_estimate(e) - exact) <= 5 * se_e + 1e-12)



# ---- two-qubit tables (Eq. ET2): more than one nonzero per column

def _table_circuit(n, d, seed):
    g, m2 = W.random_table_circuit(n, d, seed)
    assert np.sum(g[:, 0] == W.U2) >= 1
    return g, m2


@pytest.mark.parametrize("n,d,seed", [(2, 4, 1), (3, 5, 2), (4, 5, 6)])
def test_table_gates_against_matrix_products(n, d, seed):
    g, m2 = _table_circuit(n, d, seed)
    want = _kron_unitary(n, d, g, None, m2)[:, 0]
    assert np.allclose(oracle.u_statevector(n, d, g, None, mats2=m2), want, atol=1e-12)
    assert np.allclose(oracle.u_pathstats(n, d, g, None, mats2=m2)["U"], want, atol=1e-12)
    assert np.isnan(oracle.u_log2z(n, d, g, None, mats2=m2))


@pytest.mark.parametrize("n,d,seed", [(2, 4, 1), (3, 4, 2), (3, 5, 9)])
def test_table_stationary_law_is_abs_weight(n, d, seed):
    """The factorised Metropolis step (table energy -ln|U| per entry) keeps
    p_C ~ |U_C| over the valid paths: chi-square of the final states."""
    from scipy.stats import chisquare
    g, m2 = _table_circuit(n, d, seed)
    # |U_C| of every valid path by the layer matrices (numpy)
    per_layer = []
    for L in range(d):
        gl = [(i, r) for i, r in enumerate(g) if r[1] == L]
        sub = np.array([r for _, r in gl], dtype=np.int32).reshape(-1, 4).copy()
        sub[:, 1] = 0
        mm = np.stack([m2[i] for i, _ in gl]) if gl else np.zeros((0, 4, 4))
        per_layer.append(_kron_unitary(n, 1, sub, None, mm))
    weights = {}
    for path in itertools.product(range(1 << n), repeat=d):
        w, prev = 1.0 + 0j, 0
        for L, s_ in enumerate(path):
            w *= per_layer[L][s_, prev]
            prev = s_
        if abs(w) > 1e-14:
            weights[path] = abs(w)
    keys = sorted(weights)
    p = np.array([weights[k] for k in keys])
    p /= p.sum()
    chains = 20000
    # a table with zero entries is crossed only through penalised states:
    # 1500 sweeps forget the initial law at J = 4
    r = oracle.u_gibbs(n, d, g, None, J=4.0, seed=17, chains=chains, sweeps=1500, mats2=m2)
    idx = _path_index(r["state"], n)
    key_idx = np.array([_path_index(np.array([k]), n)[0] for k in keys])
    counts = np.array([np.sum(idx == w) for w in key_idx])
    assert counts.sum() > 0.3 * chains
    assert chisquare(counts, p * counts.sum()).pvalue > 1e-4


@pytest.mark.parametrize("n,d,seed", [(3, 5, 2), (4, 5, 6)])
def test_table_circuits_converge_l2(n, d, seed):
    """No closed-form scale: the L2-normalised estimate (Fig. 2 Step 4)
    approaches the normalised state vector."""
    g, m2 = _table_circuit(n, d, seed)
    exact = oracle.u_statevector(n, d, g, None, mats2=m2)
    blocks = []
    for b in range(16):
        r = oracle.u_gibbs(n, d, g, None, J=4.0, seed=5, chains=128, chain0=128 * b, sweeps=600,
                           burn_in=100, mats2=m2)
        blocks.append(r["sum"])
    blocks = np.array(blocks)
    tot = blocks.sum(axis=0)
    est = tot / np.linalg.norm(tot)
    # batch means of the normalised estimate (normalised per block)
    per = blocks / np.linalg.norm(blocks, axis=1, keepdims=True)
    se = per.std(axis=0, ddof=1) / np.sqrt(len(per))
    assert np.all(np.abs(est - exact) <= 5 * se + 1e-3), (est, exact, se)
    with pytest.raises(ValueError):  # the exact sampler needs closed-form column sums
        oracle.u_elim(n, d, g, None, seed=1, chains=32, sweeps=2, mats2=m2)
