"""GPU parity of the plain Gibbs path against the CPU oracle, through the C ABI.

Chain words, histograms and counters must be bit-identical to the oracle's
for identical Philox streams (all couplings are exact multiples of J and the
thresholds are the same u32 table); amplitudes must sit within 5 standard
errors of the FP64 state vector.
"""
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


def _gpu_run(n, d, g, J, seed, chains, sweeps=(), alphas=None, beta=0, burn_in=0, record_every=1,
             n_batches=0):
    m = pbits.Model(n, d, g, J, input_bits=beta)
    r = pbits.Run([m], [pbits.RunCfg(seed=seed, chains=chains, alphas=alphas, burn_in=burn_in,
                                     record_every=record_every, n_batches=n_batches)])
    for s in sweeps:
        r.sweeps(s)
    r.wait()
    return m, r


def test_philox_device_matches_oracle():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(512, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    for key in [(0, 0), (0xA4093822, 0x299F31D0), (0xFFFFFFFF, 0xFFFFFFFF), (0x5EED, 0)]:
        got = pbits.philox_fill(ctr, key)
        for i in range(0, 512, 37):
            assert np.array_equal(got[i], oracle.philox4x32_10(ctr[i], key))
    kat = pbits.philox_fill(np.zeros((1, 4), np.uint32), (0, 0))[0]
    assert [int(x) for x in kat] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


CASES = [
    # name, n, d, seed, chains, J, beta
    ("tiny", 3, 4, 0, 1024, 4.0, 0),
    ("ragged", 5, 7, 17, 40, 3.0, 0),
    ("mid_shape", 12, 20, 1000, 96, None, 0),
    ("one_chain", 7, 13, 5, 1, 2.5, 0),
    ("hchain", 1, 6, None, 64, 3.0, 0),
    ("ghz", 6, 6, None, 64, 3.5, 0),
    ("input_bits", 4, 9, 23, 64, 3.0, 0b1011),
    ("wide", 32, 3, 9, 64, 4.0, 0),
    ("deep", 2, 64, 31, 32, 3.0, 0),
    ("max", 32, 64, 3, 40, None, 0),     # the largest model: 2048 p-bits
    ("one_layer", 6, 1, 4, 64, 3.0, 0),  # no two p-bits interact: one class
    ("no_h", 5, 8, 12, 64, 3.0, 0b101),  # h = 0: a single valid path
]


def _circuit(name, n, d, seed):
    if name == "hchain":
        return W.hadamard_chain(d)
    if name == "ghz":
        return W.ghz(n)
    g = W.random_circuit(n, d, seed)
    if name == "no_h":
        g = np.array(g)
        g[g[:, 0] == W.H, 0] = W.T
    return g


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_init_and_sweeps_bit_exact(case):
    name, n, d, seed, chains, J, beta = case
    g = _circuit(name, n, d, seed)
    J = W.default_J(n, d, g) if J is None else J
    key = 0x5EED + 7
    sweeps = 6 if n * d > 200 else 25
    alphas = None if n <= 20 else np.arange(16, dtype=np.uint32)
    m, r = _gpu_run(n, d, g, J, key, chains, beta=beta, alphas=alphas)
    init = pbits.unslice_state(r.get_state(), chains)
    ref0 = oracle.gibbs(n, d, g, J=J, seed=key, chains=chains, sweeps=0, beta=beta, alphas=alphas)
    assert np.array_equal(init, ref0["state"]), "initial valid paths differ"
    assert np.all(oracle.violations(n, d, g, init, beta=beta) == 0)
    r.sweeps(sweeps)
    r.wait()
    got = pbits.unslice_state(r.get_state(), chains)
    cnt, valid, samples = r.histogram()
    ref = oracle.gibbs(n, d, g, J=J, seed=key, chains=chains, sweeps=sweeps, beta=beta,
                       alphas=alphas)
    assert np.array_equal(got, ref["state"])
    assert samples == ref["samples"] == chains * sweeps
    assert valid == ref["valid"]
    assert np.array_equal(cnt, ref["cnt"])


@pytest.mark.parametrize("case", [c for c in CASES if c[0] in ("tiny", "ragged", "mid_shape", "one_chain")],
                         ids=lambda c: c[0])
def test_two_buffer_production_bit_exact(case, monkeypatch):
    """Plain runs whose tables fit take 16 planes ahead per p-bit, produced
    evenly over the colour steps in three buffers; the others (the largest
    models) 12 planes in two buffers, made one step ahead.  The second form
    is forced here (PB_BALANCED=0) on models that would take the first: both
    must give the oracle's chains and histogram (the planes are the same
    Philox outputs, only computed at another time)."""
    monkeypatch.setenv("PB_BALANCED", "0")
    name, n, d, seed, chains, J, beta = case
    g = _circuit(name, n, d, seed)
    J = W.default_J(n, d, g) if J is None else J
    key = 0x5EED + 8
    m, r = _gpu_run(n, d, g, J, key, chains, sweeps=(9,), beta=beta)
    ref = oracle.gibbs(n, d, g, J=J, seed=key, chains=chains, sweeps=9, beta=beta)
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    cnt, valid, _ = r.histogram()
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"]


def test_graph_replays_continue_the_stream():
    """sweeps(7) + sweeps(11) + sweeps(7) == the oracle's 25 sweeps."""
    n, d = 6, 9
    g = W.random_circuit(n, d, 44)
    _, r = _gpu_run(n, d, g, 3.0, 99, 128, sweeps=(7, 11, 7))
    ref = oracle.gibbs(n, d, g, J=3.0, seed=99, chains=128, sweeps=25)
    assert np.array_equal(pbits.unslice_state(r.get_state(), 128), ref["state"])
    cnt, valid, samples = r.histogram()
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"]
    assert r.stats()["sweeps_done"] == 25


def test_burn_in_and_thinning():
    n, d = 4, 6
    g = W.random_circuit(n, d, 3)
    _, r = _gpu_run(n, d, g, 3.0, 5, 64, sweeps=(30,), burn_in=7, record_every=4)
    ref = oracle.gibbs(n, d, g, J=3.0, seed=5, chains=64, sweeps=30, burn_in=7, record_every=4)
    cnt, valid, samples = r.histogram()
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"] and samples == ref["samples"]


def test_alpha_subset():
    n, d = 6, 8
    g = W.random_circuit(n, d, 12)
    al = np.array([9, 0, 63, 17], dtype=np.uint32)  # unsorted on purpose
    _, r = _gpu_run(n, d, g, 3.0, 8, 96, sweeps=(20,), alphas=al)
    ref = oracle.gibbs(n, d, g, J=3.0, seed=8, chains=96, sweeps=20)
    cnt, valid, _ = r.histogram()
    assert np.array_equal(cnt, ref["cnt"][al]) and valid == ref["valid"]


def test_checkpoint_restore_bit_identical():
    n, d = 5, 8
    g = W.random_circuit(n, d, 77)
    _, a = _gpu_run(n, d, g, 3.0, 4, 96, sweeps=(10,))
    blob = a.checkpoint()
    a.sweeps(15)
    a.wait()
    _, b = _gpu_run(n, d, g, 3.0, 4, 96)
    b.restore(blob)
    b.sweeps(15)
    b.wait()
    assert np.array_equal(a.get_state(), b.get_state())
    ca, va, sa = a.histogram()
    cb, vb, sb = b.histogram()
    assert np.array_equal(ca, cb) and va == vb and sa == sb


def test_batched_run_equals_separate_runs():
    """Several circuits in one persistent launch give each circuit's own stream."""
    specs = [(4, 6, 1, 64), (7, 11, 2, 200), (3, 4, 3, 32), (9, 8, 4, 96)]
    models, cfgs, refs = [], [], []
    for n, d, s, ch in specs:
        g = W.random_circuit(n, d, s)
        models.append(pbits.Model(n, d, g, 3.0))
        cfgs.append(pbits.RunCfg(seed=0x5EED + s, chains=ch))
        refs.append(oracle.gibbs(n, d, g, J=3.0, seed=0x5EED + s, chains=ch, sweeps=12))
    r = pbits.Run(models, cfgs)
    r.sweeps(12)
    r.wait()
    for i, ref in enumerate(refs):
        assert np.array_equal(pbits.unslice_state(r.get_state(i), cfgs[i].chains), ref["state"])
        cnt, valid, _ = r.histogram(i)
        assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"]


def test_amplitude_kernel_matches_counts():
    n, d = 5, 6
    g = W.random_circuit(n, d, 21)
    m, r = _gpu_run(n, d, g, 3.0, 2, 512, sweeps=(200,), n_batches=8)
    cnt, valid, _ = r.histogram()
    h = m.info()["h"]
    psi, se = r.amplitudes()
    want = oracle.estimate_amplitudes(cnt, valid, h)
    assert np.allclose(psi, want, rtol=1e-12, atol=1e-14)
    assert np.all(se >= 0) and np.all(np.isfinite(se))
    psin, _ = r.amplitudes(l2_normalize=True)
    assert abs(np.sum(np.abs(psin) ** 2) - 1) < 1e-12
    assert np.allclose(psin, want / np.sqrt(np.sum(np.abs(want) ** 2)), rtol=1e-12, atol=1e-14)


def test_amplitude_kernel_many_batches():
    """More batches than a warp has lanes (the amplitude kernel's lanes take
    batches b, b + 32, ...): amplitudes equal the oracle's estimate of the
    same counts."""
    n, d = 4, 5
    g = W.random_circuit(n, d, 22)
    m, r = _gpu_run(n, d, g, 3.0, 3, 45 * 32, sweeps=(60,), n_batches=45)
    cnt, valid, _ = r.histogram()
    psi, se = r.amplitudes()
    want = oracle.estimate_amplitudes(cnt, valid, m.info()["h"])
    assert np.allclose(psi, want, rtol=1e-12, atol=1e-14)
    assert np.all(se >= 0) and np.all(np.isfinite(se))
    reached = cnt.sum(axis=1) > 0
    assert np.all(se[reached] > 0)


def test_tiny_workload_amplitudes():
    """Tiny workload at its budget (1024 chains x 1e4 sweeps): every amplitude
    within 5 batch-means standard errors of the FP64 state vector."""
    wl = W.tiny()
    m, r = _gpu_run(wl.n, wl.d, wl.gates, wl.J, wl.seed, wl.chains, sweeps=(wl.sweeps,),
                    n_batches=32)
    psi, se = r.amplitudes()
    exact = oracle.statevector(wl.n, wl.d, wl.gates)
    err = np.abs(psi - exact)
    assert np.all(err <= 5 * se + 1e-12), (err, se)
    assert se.max() < 3e-3


def test_tiny_workload_converges_to_1e_3():
    """After convergence (the tiny circuit run 20x its budget, 1024 chains x
    2e5 sweeps) every amplitude is within 1e-3 of the state vector."""
    wl = W.tiny()
    m, r = _gpu_run(wl.n, wl.d, wl.gates, wl.J, wl.seed + 1, wl.chains, sweeps=(200_000,),
                    n_batches=32)
    psi, se = r.amplitudes()
    exact = oracle.statevector(wl.n, wl.d, wl.gates)
    err = np.abs(psi - exact)
    assert err.max() < 1e-3, (err.max(), se.max())
    assert np.all(err <= 5 * se + 1e-12)


def test_mid_workload_sampled_parity():
    """Mid workload in the launch configuration the benchmark times (4096
    chains, one CTA per 32-chain group): after 300 sweeps, sampled groups are
    continued by the oracle for 3 sweeps from the GPU's state and must match
    the GPU's next 3 sweeps bit for bit."""
    wl = W.mid()
    m, r = _gpu_run(wl.n, wl.d, wl.gates, wl.J, wl.seed, wl.chains, sweeps=(300,))
    before = pbits.unslice_state(r.get_state(), wl.chains)
    r.sweeps(3)
    r.wait()
    after = pbits.unslice_state(r.get_state(), wl.chains)
    for grp in (0, 57, 127):
        c0 = grp * 32
        ref = oracle.gibbs(wl.n, wl.d, wl.gates, J=wl.J, seed=wl.seed, chains=32, chain0=c0,
                           sweep0=300, sweeps=3, state=before[c0:c0 + 32])
        assert np.array_equal(after[c0:c0 + 32], ref["state"]), grp
    _, valid, samples = r.histogram()
    assert samples == wl.chains * 303
    # stationary valid fraction (1 + e^{-J})^{-M} is reached from a valid start
    p = (1 + np.exp(-wl.J)) ** (-m.info()["M"])
    assert 0.3 * p < valid / samples <= 1.0


def test_sharded_runs_sum_to_the_single_run():
    """Rank-style sharding on one GPU: the chain ranges of two ranks (global
    group offsets) run separately; their integer histograms add up to the
    single run of all chains bit for bit."""
    from paper_2007_07379_gb300 import dist as D
    n, d, chains = 6, 9, 200
    g = W.random_circuit(n, d, 8)
    _, full = _gpu_run(n, d, g, 3.0, 33, chains, sweeps=(20,))
    want = full.histogram()
    tot_cnt, tot_valid, tot_samples = 0, 0, 0
    states = []
    for rank in range(2):
        c, g0 = D.shard(chains, rank, 2)
        m = pbits.Model(n, d, g, 3.0)
        r = pbits.Run([m], [pbits.RunCfg(seed=33, chains=c, group0=g0)])
        r.sweeps(20)
        cnt, valid, samples = r.histogram()
        tot_cnt = tot_cnt + cnt
        tot_valid += valid
        tot_samples += samples
        states.append(pbits.unslice_state(r.get_state(), c))
    assert np.array_equal(tot_cnt, want[0]) and tot_valid == want[1] and tot_samples == want[2]
    assert np.array_equal(np.concatenate(states), pbits.unslice_state(full.get_state(), chains))


def test_zero_sweeps_and_the_single_path_of_an_h_free_circuit():
    """h = 0: the only valid path is the deterministic one, so every valid
    sample lands in one (alpha, phase) bin and |psi_alpha| = 1 exactly."""
    n, d = 5, 8
    g = np.array(W.random_circuit(n, d, 12))
    g[g[:, 0] == W.H, 0] = W.T
    m, r = _gpu_run(n, d, g, 3.0, 99, 256, beta=0b101)
    r.sweeps(0)
    cnt0, v0, s0 = r.histogram()
    assert v0 == 0 and s0 == 0 and cnt0.sum() == 0
    r.sweeps(50)
    cnt, valid, samples = r.histogram()
    assert samples == 256 * 50 and valid > 0
    nz = np.argwhere(cnt > 0)
    assert len(nz) == 1 and cnt[tuple(nz[0])] == valid
    psi, se = r.amplitudes()
    # every batch estimates the same exact value: SE is rounding residue only
    assert abs(abs(psi[nz[0][0]]) - 1.0) < 1e-12 and np.all(se < 1e-15)
    assert np.allclose(psi, oracle.statevector(n, d, g, beta=0b101), atol=1e-12)
