"""Batched workload: 256 uneven random circuits (n in [6,20], d in [8,40],
chains max(256, 2^ceil(n/2))) in one persistent, graph-captured launch with
an autotuned CTA shape.  Sampled circuits must match the oracle bit for bit;
tuning and the shape must not change any result."""
import os
import tempfile

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


def _batched_run(wls):
    models = [pbits.Model(w.n, w.d, w.gates, w.J) for w in wls]
    cfgs = [pbits.RunCfg(seed=w.seed, chains=w.chains) for w in wls]
    return models, pbits.Run(models, cfgs)


def test_full_batch_sampled_parity():
    wls = W.batched()
    assert len(wls) == 256
    models, r = _batched_run(wls)
    assert r.shape()["grid"] > 0  # persistent launch
    sweeps = 4
    r.sweeps(sweeps)
    r.wait()
    for i in (0, 37, 101, 255):
        w = wls[i]
        got = pbits.unslice_state(r.get_state(i), w.chains)
        # the oracle continues 32 chains of this circuit from the initial state
        ref = oracle.gibbs(w.n, w.d, w.gates, J=w.J, seed=w.seed, chains=32, sweeps=sweeps,
                           alphas=np.arange(4, dtype=np.uint32))
        assert np.array_equal(got[:32], ref["state"]), i


def test_tuning_does_not_change_results():
    wls = W.batched(24)
    _, a = _batched_run(wls)
    _, b = _batched_run(wls)
    cache = os.path.join(tempfile.mkdtemp(), "tune.txt")
    ms = b.tune(trial_sweeps=20, cache_path=cache)
    assert ms > 0 and os.path.exists(cache)
    shape = b.shape()
    a.sweeps(30)
    b.sweeps(30)
    for i, w in enumerate(wls):
        assert np.array_equal(a.get_state(i), b.get_state(i)), i
        assert np.array_equal(a.histogram(i)[0], b.histogram(i)[0]), i
    # a second tuning of the same shapes is a cache hit with the same choice
    _, c = _batched_run(wls)
    c.tune(trial_sweeps=20, cache_path=cache)
    assert c.shape()["consumers"] == shape["consumers"] and c.shape()["producers"] == shape["producers"]


@pytest.mark.parametrize("cons,prod", [(32, 32), (64, 96), (224, 352)])
def test_shape_does_not_change_results(cons, prod):
    n, d = 10, 16
    g = W.random_circuit(n, d, 5)
    m = pbits.Model(n, d, g, 3.0)
    r = pbits.Run([m], [pbits.RunCfg(seed=4, chains=256)])
    r.set_shape(cons, prod)
    r.sweeps(12)
    ref = oracle.gibbs(n, d, g, J=3.0, seed=4, chains=256, sweeps=12)
    assert np.array_equal(pbits.unslice_state(r.get_state(), 256), ref["state"])
    assert np.array_equal(r.histogram()[0], ref["cnt"])


def test_two_buffer_persistent_launch_matches(monkeypatch):
    """The persistent launch in both plane-buffer forms (three buffers with
    16 planes ahead, the default; two with 12, forced by PB_BALANCED=0):
    identical chains and histograms for 16 uneven circuits."""
    wls = W.batched()[:16]
    _, a = _batched_run(wls)
    a.sweeps(9)
    a.wait()
    monkeypatch.setenv("PB_BALANCED", "0")
    _, b = _batched_run(wls)
    b.sweeps(9)
    b.wait()
    for i in range(len(wls)):
        assert np.array_equal(a.get_state(i), b.get_state(i)), i
        assert np.array_equal(a.histogram(i)[0], b.histogram(i)[0]), i
