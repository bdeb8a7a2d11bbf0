"""Exact path sampler on the eliminated network (PB_ELIM) on the GPU against
the oracle's orc_elim: identical Philox draws give identical paths and
counters (bit-exact), and the i.i.d. estimator converges to the state
vector at its closed-form standard error."""
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


def _elim_run(n, d, g, seed, chains, alphas=None, burn_in=0, record_every=1, n_batches=8):
    m = pbits.Model(n, d, g, W.default_J(n, d, g))
    cfg = pbits.RunCfg(seed=seed, chains=chains, alphas=alphas, burn_in=burn_in,
                       record_every=record_every, n_batches=n_batches, sampler=pbits.PB_ELIM)
    return m, pbits.Run([m], [cfg])


@pytest.mark.parametrize("n,d,cseed,chains,sweeps", [(3, 4, 0, 1024, 50), (5, 8, 21, 100, 33),
                                                     (12, 20, 1000, 4096, 6), (1, 6, -1, 64, 40)])
def test_bit_exact_vs_oracle(n, d, cseed, chains, sweeps):
    g = W.hadamard_chain(d) if cseed < 0 else W.random_circuit(n, d, cseed)
    m, r = _elim_run(n, d, g, seed=77, chains=chains)
    r.sweeps(sweeps)
    r.wait()
    cnt, valid, samples = r.histogram()
    state = pbits.unslice_state(r.get_state(), chains)
    ref = oracle.elim(n, d, g, seed=77, chains=chains, sweeps=sweeps)
    assert samples == ref["samples"] == chains * sweeps
    assert valid == ref["valid"] == samples
    assert np.array_equal(cnt, ref["cnt"])
    assert np.array_equal(state, ref["state"])


def test_launches_compose_and_record_rule():
    n, d = 6, 10
    g = W.random_circuit(n, d, 5)
    m, r = _elim_run(n, d, g, seed=3, chains=200, burn_in=4, record_every=3)
    r.sweeps(8)
    r.sweeps(12)
    r.wait()
    cnt, valid, samples = r.histogram()
    ref = oracle.elim(n, d, g, seed=3, chains=200, sweeps=20, burn_in=4, record_every=3)
    assert samples == ref["samples"] and valid == ref["valid"]
    assert np.array_equal(cnt, ref["cnt"])
    assert np.array_equal(pbits.unslice_state(r.get_state(), 200), ref["state"])


def test_output_subset():
    n, d = 8, 12
    g = W.random_circuit(n, d, 9)
    al = np.array([0, 5, 17, 255, 128], dtype=np.uint32)
    m, r = _elim_run(n, d, g, seed=11, chains=512, alphas=al)
    r.sweeps(16)
    cnt, valid, samples = r.histogram()
    ref = oracle.elim(n, d, g, seed=11, chains=512, sweeps=16, alphas=al)
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"] and samples == ref["samples"]


def test_tiny_converges_to_the_state_vector():
    """i.i.d. paths: SE = sqrt((N_alpha - |psi|^2) / T) exactly, so 1e7 samples
    reach 1e-3 on the tiny circuit."""
    wl = W.tiny()
    exact = oracle.statevector(wl.n, wl.d, wl.gates)
    h, rank = oracle.gf2_rank(wl.n, wl.d, wl.gates)
    m, r = _elim_run(wl.n, wl.d, wl.gates, seed=wl.seed, chains=wl.chains, n_batches=32)
    r.sweeps(10_000)
    psi, se = r.amplitudes()
    cnt, valid, _ = r.histogram()
    # N_alpha = 2^{h - rank} valid paths end at a reachable output, none at
    # the others (their estimate is exactly 0)
    reach = cnt.sum(axis=1) > 0
    Na = np.where(reach, 2.0 ** (h - rank), 0.0)
    se_closed = np.sqrt(np.maximum(Na - np.abs(exact) ** 2, 0.0) / valid)
    err = np.abs(psi - exact)
    assert np.all(err <= 5 * se_closed + 1e-12), (err, se_closed)
    assert err.max() < 1e-3
    # batch-means SE agrees with the closed form (i.i.d. draws)
    big = se_closed > 1e-6
    assert big.any() and np.all(np.abs(se[big] / se_closed[big] - 1.0) < 0.5)
    assert np.all(psi[~reach] == 0) and np.all(np.abs(exact[~reach]) < 1e-12)


def test_learned_moves_reject_an_elim_run():
    n, d = 4, 6
    g = W.random_circuit(n, d, 2)
    m, r = _elim_run(n, d, g, seed=1, chains=64)
    net = pbits.Mlp(n, d, hidden=64, batch=128, seed=1)
    with pytest.raises(Exception):
        pbits.Learned(r, net)
