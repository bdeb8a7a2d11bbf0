"""General one-qubit gates (PB_U; Eq. EB, Eq. HadT) on the GPU against the
oracle's orc_u_gibbs / orc_u_elim: identical Philox draws give identical
chain states and per-output sample counts (bit-exact), and the FP64 phase
sums agree within the bound of the device's fixed-point angles."""
import numpy as np
import pytest

import oracle
from paper_2007_07379_gb300 import build, pbits
from paper_2007_07379_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pbits.load()


def _sum_tol(counts, n_u):
    """Per bin: each sample's angle is a sum of n_u phases rounded to 2^-32
    turn (error <= n_u 2^-33 turn = n_u pi 2^-32 rad) plus the class angle
    (exact); the device rounds the angle to FP32 (<= pi 2^-24 = 1.9e-7 rad)
    and takes sincospif (about one ulp, 6e-8), then sums in FP64 in another
    order (~1e-16 per term): |delta| <= count (n_u * 7.4e-10 + 3e-7) + 1e-12."""
    return counts.astype(np.float64) * (n_u * 7.4e-10 + 3e-7) + 1e-12


def _circuit(kind, n, d, seed):
    if kind == "rot":
        return W.rotated_h_chain(d, 0.3 + 0.01 * seed)
    return W.random_general_circuit(n, d, seed, frac_u=0.35)


CASES = [("gen", 3, 5, 7, 256, 40), ("gen", 5, 8, 21, 100, 33), ("rot", 1, 10, 0, 64, 50),
         ("gen", 12, 20, 1000, 4096, 6), ("gen", 32, 64, 3, 40, 3), ("gen", 6, 1, 4, 33, 7)]


@pytest.mark.parametrize("kind,n,d,seed,chains,sweeps", CASES)
def test_gibbs_bit_exact_vs_oracle(kind, n, d, seed, chains, sweeps):
    g, mats = _circuit(kind, n, d, seed)
    J = 3.0
    alphas = np.arange(16, dtype=np.uint32) if n > 20 else None
    m = pbits.Model(n, d, g, J, mats=mats)
    inf = m.info()
    assert inf["n_u"] == int(np.sum(g[:, 0] == W.U))
    r = pbits.Run([m], [pbits.RunCfg(seed=77, chains=chains, alphas=alphas)])
    r.sweeps(sweeps)
    r.wait()
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_gibbs(n, d, g, mats, J=J, seed=77, chains=chains, sweeps=sweeps, alphas=alphas)
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    assert samples == ref["samples"] and valid == ref["valid"]
    assert np.array_equal(cnt, ref["cnt"])
    assert np.all(np.abs(sums - ref["sum"]) <= _sum_tol(cnt, inf["n_u"]))
    assert np.isclose(inf["log2z"], ref["log2z"], rtol=0, atol=1e-12)
    psi, _ = r.amplitudes()
    want = oracle.u_estimate(ref)
    scale = 2.0 ** ref["log2z"] / max(valid, 1)
    assert np.all(np.abs(psi - want) <= scale * _sum_tol(cnt, inf["n_u"]) + 1e-12)


@pytest.mark.parametrize("n_alphas", [1, 3, 5])
def test_odd_output_lists_bit_exact(n_alphas):
    """An output list of odd length: the shared histogram holds 40 bytes a
    bin, so the tables after it start at a 16-byte boundary only because
    the histogram is rounded up to one; results as the oracle's."""
    n, d, chains, sweeps = 5, 8, 100, 21
    g, mats = _circuit("gen", n, d, 21)
    alphas = np.array([3, 17, 30, 8, 21][:n_alphas], dtype=np.uint32)
    m = pbits.Model(n, d, g, 3.0, mats=mats)
    r = pbits.Run([m], [pbits.RunCfg(seed=78, chains=chains, alphas=alphas)])
    r.sweeps(sweeps)
    r.wait()
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_gibbs(n, d, g, mats, J=3.0, seed=78, chains=chains, sweeps=sweeps, alphas=alphas)
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    assert samples == ref["samples"] and valid == ref["valid"]
    assert np.array_equal(cnt, ref["cnt"])
    assert np.all(np.abs(sums - ref["sum"]) <= _sum_tol(cnt, m.info()["n_u"]))


def test_plain_and_general_models_share_a_run():
    """The general-gate kernel runs plain models unchanged (8 exact phase
    classes), and both match their oracles bit-exactly."""
    n, d = 5, 8
    gp = W.random_circuit(n, d, 21)
    gu, mats = W.random_general_circuit(n, d, 22, frac_u=0.5)
    mp = pbits.Model(n, d, gp, W.default_J(n, d, gp))
    mu = pbits.Model(n, d, gu, 2.5, mats=mats)
    r = pbits.Run([mp, mu], [pbits.RunCfg(seed=5, chains=96), pbits.RunCfg(seed=6, chains=70)])
    r.sweeps(17)
    cp, vp, sp = r.histogram(0)
    refp = oracle.gibbs(n, d, gp, J=W.default_J(n, d, gp), seed=5, chains=96, sweeps=17)
    assert np.array_equal(cp, refp["cnt"]) and vp == refp["valid"] and sp == refp["samples"]
    assert np.array_equal(pbits.unslice_state(r.get_state(0), 96), refp["state"])
    sums, cnt, vu, su = r.phase_sums(1)
    refu = oracle.u_gibbs(n, d, gu, mats, J=2.5, seed=6, chains=70, sweeps=17)
    assert np.array_equal(cnt, refu["cnt"]) and vu == refu["valid"] and su == refu["samples"]
    assert np.array_equal(pbits.unslice_state(r.get_state(1), 70), refu["state"])
    assert np.all(np.abs(sums - refu["sum"]) <= _sum_tol(cnt, int(np.sum(gu[:, 0] == W.U))))
    with pytest.raises(pbits.PbError):
        r.histogram(1)


def test_shape_invariance_with_large_classes():
    """32 consumers: most colour classes exceed them, so the coupled p-bits
    beyond the first 32 take the out-of-line path; results are unchanged."""
    n, d = 12, 20
    g, mats = W.random_general_circuit(n, d, 1000, frac_u=0.35)
    m = pbits.Model(n, d, g, 3.0, mats=mats)
    r = pbits.Run([m], [pbits.RunCfg(seed=9, chains=256)])
    r.set_shape(32, 96)
    r.sweeps(9)
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_gibbs(n, d, g, mats, J=3.0, seed=9, chains=256, sweeps=9)
    assert np.array_equal(pbits.unslice_state(r.get_state(), 256), ref["state"])
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"]


def test_global_histogram_path():
    """n = 14: 2^14 bins do not fit the shared-memory histogram; the record
    adds to global memory directly."""
    n, d = 14, 6
    g, mats = W.random_general_circuit(n, d, 5, frac_u=0.4)
    m = pbits.Model(n, d, g, 3.0, mats=mats)
    r = pbits.Run([m], [pbits.RunCfg(seed=3, chains=64, burn_in=2, record_every=2)])
    r.sweeps(11)
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_gibbs(n, d, g, mats, J=3.0, seed=3, chains=64, sweeps=11, burn_in=2, record_every=2)
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"] and samples == ref["samples"]
    assert np.all(np.abs(sums - ref["sum"]) <= _sum_tol(cnt, int(np.sum(g[:, 0] == W.U))))


# 9600 / 12800 chains: 300 / 400 groups, the 16- and 8-warp exact-sampler kernels
@pytest.mark.parametrize("kind,n,d,seed,chains,sweeps", [("gen", 3, 5, 7, 300, 20), ("rot", 1, 10, 1, 64, 30),
                                                         ("gen", 12, 20, 1000, 4096, 4),
                                                         ("gen", 5, 8, 11, 9600, 9), ("gen", 5, 8, 12, 12800, 7)])
def test_elim_bit_exact_vs_oracle(kind, n, d, seed, chains, sweeps):
    g, mats = _circuit(kind, n, d, seed)
    m = pbits.Model(n, d, g, 3.0, mats=mats)
    r = pbits.Run([m], [pbits.RunCfg(seed=41, chains=chains, sampler=pbits.PB_ELIM)])
    r.sweeps(sweeps)
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_elim(n, d, g, mats, seed=41, chains=chains, sweeps=sweeps)
    assert samples == valid == ref["samples"] == chains * sweeps
    assert np.array_equal(cnt, ref["cnt"])
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    assert np.all(np.abs(sums - ref["sum"]) <= _sum_tol(cnt, int(np.sum(g[:, 0] == W.U))))


def test_compensated_phase_sums():
    """Phase sums of general gates are compensated: every FP64 atomic add's
    rounding error is carried exactly into a second word.  The same samples
    (a four-qubit circuit of random one-qubit unitaries; the exact sampler,
    2^23 samples, and Gibbs, 2^22 records) summed in one launch and in many
    launches -- another grouping and order of the adds -- give sums equal to
    within 8 ulp of their size (a plain FP64 sum of ~5e5 unit phasors per bin
    drifts by hundreds of half-ulps between orders), and the sums agree with
    the oracle's exact phasors within the per-term bound."""
    n, d = 4, 12
    g, mats = W.random_general_circuit(n, d, 5, frac_u=1.0)
    m = pbits.Model(n, d, g, 3.0, mats=mats)
    n_u = m.info()["n_u"]
    for sampler, total, parts in ((pbits.PB_ELIM, 2048, 16), (pbits.PB_GIBBS, 1024, 8)):
        cfg = pbits.RunCfg(seed=31, chains=4096, sampler=sampler)
        a = pbits.Run([m], [cfg])
        a.sweeps(total)
        b = pbits.Run([m], [cfg])
        for _ in range(parts):
            b.sweeps(total // parts)
        sa, ca, va, _ = a.phase_sums()
        sb, cb, vb, _ = b.phase_sums()
        assert np.array_equal(ca, cb) and va == vb and ca.max() > 50_000
        for x, y in ((sa.real, sb.real), (sa.imag, sb.imag)):
            assert np.all(np.abs(x - y) <= 8 * np.spacing(np.abs(x) + 1.0)), (sampler, np.abs(x - y))
        if sampler == pbits.PB_ELIM:
            ref = oracle.u_elim(n, d, g, mats, seed=31, chains=4096, sweeps=total)
        else:
            ref = oracle.u_gibbs(n, d, g, mats, J=3.0, seed=31, chains=4096, sweeps=total)
        assert np.array_equal(ca, ref["cnt"])
        assert np.all(np.abs(sa - ref["sum"]) <= _sum_tol(ca, n_u))


def test_rotated_chain_converges():
    """d = 10 rotated Hadamards (t = 0.3): the Gibbs estimate of both
    amplitudes lies within 5 batch-means SE of (1, 0), and the exact
    sampler's SE matches its closed form sqrt((Z Z_alpha - |U|^2) / T)."""
    d, th = 10, 0.3
    g, mats = W.rotated_h_chain(d, th)
    m = pbits.Model(1, d, g, 3.0, mats=mats)
    r = pbits.Run([m], [pbits.RunCfg(seed=1, chains=4096, burn_in=100, n_batches=32)])
    r.sweeps(3000)
    psi, se = r.amplitudes()
    exact = oracle.u_statevector(1, d, g, mats)
    assert np.all(np.abs(psi - exact) <= 5 * se + 1e-9), (psi, se)
    assert np.all(se < 0.05)
    e = pbits.Run([m], [pbits.RunCfg(seed=2, chains=4096, n_batches=32, sampler=pbits.PB_ELIM)])
    e.sweeps(500)
    psi_e, se_e = e.amplitudes()
    ps = oracle.u_pathstats(1, d, g, mats)
    Z = 2 ** m.info()["log2z"]
    _, _, _, T = e.phase_sums()
    se_closed = np.sqrt(np.maximum(Z * ps["zabs"] - np.abs(exact) ** 2, 0) / T)
    assert np.all(np.abs(psi_e - exact) <= 5 * se_closed + 1e-12)
    assert np.all(np.abs(se_e / se_closed - 1) < 0.5)


def test_rejections():
    n, d = 4, 6
    g, mats = W.random_general_circuit(n, d, 2, frac_u=0.9)
    assert np.sum(g[:, 0] == W.U) > 0
    m = pbits.Model(n, d, g, 3.0, mats=mats)
    assert m.info()["n_coupled"] > 0
    with pytest.raises(pbits.PbError):  # clamping assumes uniform free outputs
        pbits.Run([m], [pbits.RunCfg(seed=1, chains=32, alphas=np.array([0], np.uint32),
                                     sampler=pbits.PB_ELIM_CLAMP)])
    r = pbits.Run([m], [pbits.RunCfg(seed=1, chains=64)])
    net = pbits.Mlp(n, d, hidden=64, batch=128, seed=1)
    with pytest.raises(Exception):
        pbits.Learned(r, net)
    bad = mats.copy()
    i = int(np.flatnonzero(g[:, 0] == W.U)[0])
    bad[i] = np.array([[1, 0], [0, 2]])
    with pytest.raises(pbits.PbError):
        pbits.Model(n, d, g, 3.0, mats=bad)


# ---- X and two-qubit permutations with phases (PB_X, PB_U2)

TWO_Q = [(3, 5, 4, 256, 40), (5, 8, 21, 100, 33), (12, 20, 1000, 4096, 6), (32, 64, 3, 40, 3),
         (6, 1, 4, 33, 7)]


@pytest.mark.parametrize("n,d,seed,chains,sweeps", TWO_Q)
def test_two_qubit_gates_bit_exact_vs_oracle(n, d, seed, chains, sweeps):
    g, m2 = W.random_two_qubit_circuit(n, d, seed, frac=0.8)
    alphas = np.arange(16, dtype=np.uint32) if n > 20 else None
    m = pbits.Model(n, d, g, 3.0, mats2=m2)
    r = pbits.Run([m], [pbits.RunCfg(seed=13, chains=chains, alphas=alphas)])
    r.sweeps(sweeps)
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_gibbs(n, d, g, None, J=3.0, seed=13, chains=chains, sweeps=sweeps, alphas=alphas,
                         mats2=m2)
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"] and samples == ref["samples"]
    n_u = int(np.sum(g[:, 0] == W.U2))
    assert np.all(np.abs(sums - ref["sum"]) <= _sum_tol(cnt, n_u))


def test_x_gates_run_on_the_plain_kernel():
    """X without matrices: a plain model (exact phase classes), identical to
    the general oracle's sampler."""
    n, d = 6, 10
    g, _ = W.random_two_qubit_circuit(n, d, 8, frac=0.0)
    g = g.copy()
    for i in range(0, len(g), 3):
        if g[i, 0] in (W.S, W.T):
            g[i, 0] = W.X
    assert np.sum(g[:, 0] == W.X) > 0
    m = pbits.Model(n, d, g, 3.0)
    assert m.info()["n_u"] == 0
    r = pbits.Run([m], [pbits.RunCfg(seed=4, chains=200)])
    r.sweeps(15)
    cnt, valid, samples = r.histogram()
    ref = oracle.u_gibbs(n, d, g, None, J=3.0, seed=4, chains=200, sweeps=15)
    assert np.array_equal(pbits.unslice_state(r.get_state(), 200), ref["state"])
    assert np.array_equal(cnt.sum(axis=1), ref["cnt"]) and valid == ref["valid"]
    w = np.exp(1j * np.pi * np.arange(8) / 4)
    assert np.allclose(cnt.astype(np.float64) @ w, ref["sum"], atol=1e-9)


@pytest.mark.parametrize("n,d,seed,chains,sweeps", [(3, 5, 4, 300, 20), (12, 20, 1000, 4096, 4)])
def test_two_qubit_gates_exact_sampler(n, d, seed, chains, sweeps):
    g, m2 = W.random_two_qubit_circuit(n, d, seed, frac=0.8)
    m = pbits.Model(n, d, g, 3.0, mats2=m2)
    r = pbits.Run([m], [pbits.RunCfg(seed=41, chains=chains, sampler=pbits.PB_ELIM)])
    r.sweeps(sweeps)
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_elim(n, d, g, None, seed=41, chains=chains, sweeps=sweeps, mats2=m2)
    assert samples == valid == ref["samples"]
    assert np.array_equal(cnt, ref["cnt"])
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    assert np.all(np.abs(sums - ref["sum"]) <= _sum_tol(cnt, int(np.sum(g[:, 0] == W.U2))))


def test_exchange_operator_circuit_converges():
    """H on two qubits, the exchange operator J12(g), H again: the Gibbs
    estimate lies within 5 SE of the state vector."""
    gam = 1.3
    g = np.array([[W.H, 0, 0, -1], [W.H, 0, 1, -1], [W.U2, 1, 0, 1], [W.H, 2, 0, -1],
                  [W.H, 2, 1, -1]], dtype=np.int32)
    m2 = np.zeros((5, 4, 4), dtype=np.complex128)
    m2[2] = W.exchange_matrix(gam)
    exact = oracle.u_statevector(2, 3, g, None, mats2=m2)
    m = pbits.Model(2, 3, g, 3.0, mats2=m2)
    r = pbits.Run([m], [pbits.RunCfg(seed=9, chains=4096, burn_in=50, n_batches=32)])
    r.sweeps(2000)
    psi, se = r.amplitudes()
    assert np.all(np.abs(psi - exact) <= 5 * se + 1e-9), (psi, exact, se)
    assert np.all(se < 0.02)


# ---- the Toffoli gate (PB_CCX)

CCX_CASES = [(4, 5, 2, 256, 40), (6, 8, 3, 100, 25), (12, 20, 1000, 4096, 6), (5, 6, 7, 33, 9)]


@pytest.mark.parametrize("n,d,seed,chains,sweeps", CCX_CASES)
def test_toffoli_bit_exact_vs_oracle(n, d, seed, chains, sweeps):
    g = W.random_ccx_circuit(n, d, seed, frac=0.9)
    assert np.sum(g[:, 0] == W.CCX) > 0
    m = pbits.Model(n, d, g, 3.0)
    r = pbits.Run([m], [pbits.RunCfg(seed=23, chains=chains)])
    r.sweeps(sweeps)
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_gibbs(n, d, g, None, J=3.0, seed=23, chains=chains, sweeps=sweeps)
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"] and samples == ref["samples"]
    assert np.all(np.abs(sums - ref["sum"]) <= _sum_tol(cnt, 0))


def test_toffoli_shape_invariance_and_exact_sampler():
    n, d = 12, 20
    g = W.random_ccx_circuit(n, d, 1000, frac=0.7)
    m = pbits.Model(n, d, g, 3.0)
    r = pbits.Run([m], [pbits.RunCfg(seed=9, chains=256)])
    r.set_shape(32, 96)  # classes beyond 32 p-bits: the out-of-line path
    r.sweeps(9)
    _, cnt, valid, _ = r.phase_sums()
    ref = oracle.u_gibbs(n, d, g, None, J=3.0, seed=9, chains=256, sweeps=9)
    assert np.array_equal(pbits.unslice_state(r.get_state(), 256), ref["state"])
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"]
    e = pbits.Run([m], [pbits.RunCfg(seed=41, chains=300, sampler=pbits.PB_ELIM)])
    e.sweeps(12)
    sums, cnt, valid, samples = e.phase_sums()
    refe = oracle.u_elim(n, d, g, None, seed=41, chains=300, sweeps=12)
    assert np.array_equal(cnt, refe["cnt"]) and samples == valid == refe["samples"]
    assert np.array_equal(pbits.unslice_state(e.get_state(), 300), refe["state"])
    with pytest.raises(pbits.PbError):
        pbits.Run([m], [pbits.RunCfg(seed=1, chains=32, alphas=np.array([0], np.uint32),
                                     sampler=pbits.PB_ELIM_CLAMP)])


def test_toffoli_circuit_converges():
    g = W.random_ccx_circuit(4, 5, 2, frac=0.9)
    exact = oracle.u_statevector(4, 5, g, None)
    m = pbits.Model(4, 5, g, 3.0)
    r = pbits.Run([m], [pbits.RunCfg(seed=3, chains=4096, burn_in=50, n_batches=32)])
    r.sweeps(2000)
    psi, se = r.amplitudes()
    assert np.all(np.abs(psi - exact) <= 5 * se + 1e-9), (psi, exact, se)


def test_general_run_checkpoint_tune_and_mixed_with_toffoli():
    """A run holding a coupled-U model, a U2 model and a Toffoli model:
    checkpoint / restore gives the same states and counters (the FP64 sums
    to rounding), the
    autotuner keeps shapes of at most 512 threads and leaves the results
    unchanged."""
    n, d = 6, 8
    gu, mu = W.random_general_circuit(n, d, 5, frac_u=0.5)
    g2, m2 = W.random_two_qubit_circuit(n, d, 6, frac=0.8)
    gc = W.random_ccx_circuit(n, d, 3, frac=0.9)
    models = [pbits.Model(n, d, gu, 3.0, mats=mu), pbits.Model(n, d, g2, 3.0, mats2=m2),
              pbits.Model(n, d, gc, 3.0)]
    cfgs = [pbits.RunCfg(seed=11 + i, chains=64 + 17 * i) for i in range(3)]
    a = pbits.Run(models, cfgs)
    a.sweeps(7)
    blob = a.checkpoint()
    a.sweeps(9)
    b = pbits.Run(models, cfgs)
    b.restore(blob)
    b.sweeps(9)
    for i in range(3):
        sa, ca, va, na = a.phase_sums(i)
        sb, cb, vb, nb = b.phase_sums(i)
        assert np.array_equal(ca, cb) and va == vb and na == nb
        # FP64 atomic adds land in any order: equal to rounding
        assert np.allclose(sa, sb, rtol=0, atol=1e-9 * max(1.0, float(np.abs(sa).max())))
        assert np.array_equal(a.get_state(i), b.get_state(i))
    c = pbits.Run(models, cfgs)
    c.tune(trial_sweeps=5)
    sh = c.shape()
    assert sh["consumers"] + sh["producers"] + 32 <= 512
    c.sweeps(16)
    refs = [oracle.u_gibbs(n, d, gu, mu, J=3.0, seed=11, chains=64, sweeps=16),
            oracle.u_gibbs(n, d, g2, None, J=3.0, seed=12, chains=81, sweeps=16, mats2=m2),
            oracle.u_gibbs(n, d, gc, None, J=3.0, seed=13, chains=98, sweeps=16)]
    for i, ref in enumerate(refs):
        _, cnt, valid, _ = c.phase_sums(i)
        assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"]
        assert np.array_equal(pbits.unslice_state(c.get_state(i), cfgs[i].chains), ref["state"])


# ---- two-qubit tables (Eq. ET2): a second Metropolis factor on -ln|U|

def _table_with_u(n, d, seed):
    """A table circuit whose one-qubit gates are partly random unitaries:
    p-bits with both a coupling and a table factor."""
    g, m2 = W.random_table_circuit(n, d, seed)
    g = g.copy()
    rng = np.random.default_rng(seed)
    m1 = np.zeros((len(g), 2, 2), dtype=np.complex128)
    for i in range(len(g)):
        if g[i, 0] in (W.H, W.S, W.T) and rng.random() < 0.5:
            g[i, 0] = W.U
            m1[i] = W.u3(*(2 * np.pi * rng.random(3)))
    return g, m1, m2


TABLE_CASES = [(3, 5, 2, 256, 30, False), (6, 8, 5, 100, 25, False), (12, 20, 1000, 4096, 5, False),
               (6, 8, 5, 96, 20, True), (12, 20, 1000, 512, 6, True)]


@pytest.mark.parametrize("n,d,seed,chains,sweeps,with_u", TABLE_CASES)
def test_table_gates_bit_exact_vs_oracle(n, d, seed, chains, sweeps, with_u):
    if with_u:
        g, m1, m2 = _table_with_u(n, d, seed)
    else:
        (g, m2), m1 = W.random_table_circuit(n, d, seed), None
    m = pbits.Model(n, d, g, 4.0, mats=m1, mats2=m2)
    r = pbits.Run([m], [pbits.RunCfg(seed=29, chains=chains)])
    r.sweeps(sweeps)
    sums, cnt, valid, samples = r.phase_sums()
    ref = oracle.u_gibbs(n, d, g, m1, J=4.0, seed=29, chains=chains, sweeps=sweeps, mats2=m2)
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"] and samples == ref["samples"]
    n_ph = int(np.sum(g[:, 0] == W.U2) + np.sum(g[:, 0] == W.U))
    assert np.all(np.abs(sums - ref["sum"]) <= _sum_tol(cnt, n_ph))


def test_table_gates_l2_amplitudes_and_rejections():
    n, d = 3, 5
    g, m2 = W.random_table_circuit(n, d, 2)
    exact = oracle.u_statevector(n, d, g, None, mats2=m2)
    m = pbits.Model(n, d, g, 4.0, mats2=m2)
    r = pbits.Run([m], [pbits.RunCfg(seed=5, chains=4096, burn_in=100, n_batches=32)])
    r.sweeps(1500)
    psi, se = r.amplitudes(l2_normalize=True)
    assert np.all(np.abs(psi - exact) <= 5 * se + 2e-3), (psi, exact, se)
    with pytest.raises(pbits.PbError):  # no closed-form scale
        r.amplitudes(l2_normalize=False)
    with pytest.raises(pbits.PbError):  # the exact sampler needs closed-form column sums
        pbits.Run([m], [pbits.RunCfg(seed=1, chains=32, sampler=pbits.PB_ELIM)])
