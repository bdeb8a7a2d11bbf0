"""Large workload (n=24, d=32, 792 p-bits, 65536 chains, 64 output bins) in
the launch configuration the benchmark uses: sampled groups continue bit for
bit in the oracle; learned suffix moves run at this size; the amplitude
reduction of the 64 bins equals the FP64 estimator of the run's own
histogram.  (With h ~ 110 H outputs the estimator's variance, 2^{h-rank}
per sample, puts any comparison with the 2^24-entry state vector far below
the noise: the sign problem of Sec. 4.1.)"""
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


def test_large_workload():
    wl = W.large()
    m = pbits.Model(wl.n, wl.d, wl.gates, wl.J)
    r = pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=wl.chains, alphas=wl.alphas, n_batches=32)])
    r.sweeps(40)
    before = pbits.unslice_state(r.get_state(), wl.chains)
    r.sweeps(2)
    r.wait()
    after = pbits.unslice_state(r.get_state(), wl.chains)
    for grp in (0, 1000, 2047):
        c0 = grp * 32
        ref = oracle.gibbs(wl.n, wl.d, wl.gates, J=wl.J, seed=wl.seed, chains=32, chain0=c0,
                           sweep0=40, sweeps=2, state=before[c0:c0 + 32], alphas=wl.alphas)
        assert np.array_equal(after[c0:c0 + 32], ref["state"]), grp
    # learned moves at this size (untrained network; the MH correction keeps
    # the distribution)
    net = pbits.Mlp(wl.n, wl.d, hidden=256, batch=4096, seed=3)
    L = pbits.Learned(r, net)
    for _ in range(3):
        L.step(1)
        r.sweeps(1)
    mv, acc = L.stats()
    assert mv == 3 and 0 <= acc <= 3 * wl.chains
    r.sweeps(300)
    psi, se = r.amplitudes()
    cnt, valid, samples = r.histogram()
    assert samples == wl.chains * 345 and 0 < valid <= samples
    assert cnt.sum() <= valid
    want = oracle.estimate_amplitudes(cnt, valid, m.info()["h"])
    # the two sides sum the same integer counts times e^{i pi phi/4} in a
    # different order: exact zeros may come out as rounding residue of the
    # largest terms (relative 1e-16)
    assert np.allclose(psi, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    assert np.all(np.isfinite(se)) and np.all(se >= 0)
