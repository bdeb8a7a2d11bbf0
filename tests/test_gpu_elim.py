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


# chain groups (chains / 32) against the SM count (152 on GB300) pick the
# kernel's warps per CTA: up to 152 groups 32 warps, up to 304 16, else 8;
# 9600 and 12800 chains (300, 400 groups) take the 16- and 8-warp kernels
@pytest.mark.parametrize("n,d,cseed,chains,sweeps", [(3, 4, 0, 1024, 50), (5, 8, 21, 100, 33),
                                                     (12, 20, 1000, 4096, 6), (1, 6, -1, 64, 40),
                                                     (32, 64, 3, 40, 3), (6, 1, 4, 33, 7),
                                                     (5, 8, 22, 9600, 37), (5, 8, 23, 12800, 13)])
def test_bit_exact_vs_oracle(n, d, cseed, chains, sweeps):
    g = W.hadamard_chain(d) if cseed < 0 else W.random_circuit(n, d, cseed)
    alphas = np.arange(16, dtype=np.uint32) if n > 20 else None
    m, r = _elim_run(n, d, g, seed=77, chains=chains, alphas=alphas)
    r.sweeps(sweeps)
    r.wait()
    cnt, valid, samples = r.histogram()
    state = pbits.unslice_state(r.get_state(), chains)
    ref = oracle.elim(n, d, g, seed=77, chains=chains, sweeps=sweeps, alphas=alphas)
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


# ---- output-clamped exact sampler (PB_ELIM_CLAMP)

def _clamp_cfg(seed, chains, alpha, n_batches=8, sampler=None):
    return pbits.RunCfg(seed=seed, chains=chains, alphas=np.array([alpha], dtype=np.uint32),
                        n_batches=n_batches, sampler=pbits.PB_ELIM_CLAMP if sampler is None else sampler)


@pytest.mark.parametrize("n,d,cseed,chains,sweeps", [(4, 8, 17, 300, 20), (5, 6, 3, 64, 9),
                                                     (12, 20, 1000, 4096, 4), (4, 8, 18, 9600, 19),
                                                     (4, 8, 19, 12800, 11)])
def test_clamped_bit_exact_vs_oracle(n, d, cseed, chains, sweeps):
    g = W.random_circuit(n, d, cseed)
    exact = oracle.statevector(n, d, g)
    h, rank = oracle.gf2_rank(n, d, g)
    reach = [a for a in range(1 << n) if abs(exact[a]) > 1e-9][:2]
    unreach = [a for a in range(1 << n)
               if not oracle.elim_clamped(n, d, g, alpha=a, seed=1, chains=1, sweeps=0)["consistent"]][:1]
    for a in reach + unreach:
        m = pbits.Model(n, d, g, W.default_J(n, d, g))
        r = pbits.Run([m], [_clamp_cfg(41 + a, chains, a)])
        r.sweeps(sweeps)
        r.wait()
        cnt, valid, samples = r.histogram()
        ref = oracle.elim_clamped(n, d, g, alpha=a, seed=41 + a, chains=chains, sweeps=sweeps)
        assert samples == ref["samples"] == valid
        assert np.array_equal(cnt[0], ref["cnt"])
        psi, se = r.amplitudes()
        want = oracle.clamped_amplitude(ref["cnt"], ref["samples"], h, rank)
        assert abs(psi[0] - want) <= 1e-12 * max(1.0, abs(want))
        if ref["consistent"]:
            assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
        else:
            assert samples == 0 and psi[0] == 0


def test_clamped_se_is_2_to_the_r_over_2_smaller_on_mid():
    """Mid (h = 33, r = 12): the clamped estimator of psi_0 has SE
    sqrt((2^{h-2r} - |psi|^2) / T), 2^{r/2} = 64 times the unclamped one's
    sqrt((2^{h-r} - |psi|^2) / T); the batch-means SE agrees with it."""
    wl = W.mid()
    h, rank = oracle.gf2_rank(wl.n, wl.d, wl.gates)
    m = pbits.Model(wl.n, wl.d, wl.gates, wl.J)
    r = pbits.Run([m], [_clamp_cfg(wl.seed, wl.chains, 0, n_batches=32)])
    r.sweeps(2000)
    psi, se = r.amplitudes()
    _, _, samples = r.histogram()
    psi0 = oracle.statevector(wl.n, wl.d, wl.gates)[0]
    se_closed = np.sqrt(max(2.0 ** (h - 2 * rank) - abs(psi0) ** 2, 0.0) / samples)
    assert abs(se[0] / se_closed - 1.0) < 0.5
    assert abs(psi[0] - psi0) <= 5 * se_closed
    # the unclamped exact sampler over the same samples: 64x the SE on psi_0
    ru = pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains, n_batches=32,
                                      sampler=pbits.PB_ELIM)])
    ru.sweeps(2000)
    _, se_u = ru.amplitudes()
    ratio = se_u[0] / se[0]
    assert 2 ** (rank / 2) * 0.6 < ratio < 2 ** (rank / 2) * 1.6, ratio


def test_clamped_and_unclamped_models_share_a_run():
    n, d = 4, 8
    g = W.random_circuit(n, d, 17)
    m1 = pbits.Model(n, d, g, W.default_J(n, d, g))
    m2 = pbits.Model(n, d, g, W.default_J(n, d, g))
    r = pbits.Run([m1, m2], [_clamp_cfg(5, 100, 3), pbits.RunCfg(seed=6, chains=70, sampler=pbits.PB_ELIM)])
    r.sweeps(11)
    c1, v1, s1 = r.histogram(0)
    c2, v2, s2 = r.histogram(1)
    ref1 = oracle.elim_clamped(n, d, g, alpha=3, seed=5, chains=100, sweeps=11)
    ref2 = oracle.elim(n, d, g, seed=6, chains=70, sweeps=11)
    assert np.array_equal(c1[0], ref1["cnt"]) and s1 == ref1["samples"]
    assert np.array_equal(c2, ref2["cnt"]) and s2 == ref2["samples"]
