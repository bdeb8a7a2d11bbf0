"""Learned proposal (Metropolis-Hastings suffix move with the network) on the GPU.

The move must keep the sampled distribution whatever the network (the MH
correction), so an untrained network still gives amplitudes within 5 SE of
the state vector; a network trained on collected valid paths must be
accepted often and must lower the error at an equal number of steps.
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


def _run(n, d, g, J, chains, seed, n_batches=32):
    m = pbits.Model(n, d, g, J)
    r = pbits.Run([m], [pbits.RunCfg(seed=seed, chains=chains, n_batches=n_batches)])
    return m, r


def test_mh_with_untrained_network_keeps_the_distribution():
    wl = W.tiny()
    m, r = _run(wl.n, wl.d, wl.gates, wl.J, 1024, wl.seed + 5)
    net = pbits.Mlp(wl.n, wl.d, hidden=64, batch=1024, seed=11)
    L = pbits.Learned(r, net)
    for _ in range(2000):
        L.step(1)
        r.sweeps(1)
    psi, se = r.amplitudes()
    exact = oracle.statevector(wl.n, wl.d, wl.gates)
    err = np.abs(psi - exact)
    assert np.all(err <= 5 * se + 1e-9), (err, se)
    _, valid, samples = r.histogram()
    M_ = m.info()["M"]
    p = (1 + np.exp(-wl.J)) ** (-M_)
    assert abs(valid / samples - p) < 0.05
    assert 0 < L.accepted < L.proposed


def _train(r, net, n, d, sweeps=200, steps=400):
    import torch
    cap = 1 << 17
    paths = torch.zeros((cap, d), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    L = pbits.Learned(r, net)
    for _ in range(sweeps):
        r.sweeps(1)
        L.collect(paths, count)
    n_paths = min(int(count.item()), cap)
    assert n_paths > 1000
    losses = pbits.train_on_paths(net, paths, n_paths, 0, steps=steps, rows=1024, lr=2e-3, seed=7)
    torch.cuda.synchronize()
    return losses.cpu().numpy(), n_paths


def test_training_on_collected_paths_raises_acceptance():
    n, d = 6, 8
    g = W.random_circuit(n, d, 61)
    J = W.default_J(n, d, g)
    m, r = _run(n, d, g, J, 1024, 99)
    net = pbits.Mlp(n, d, hidden=128, batch=1024, seed=12)
    L0 = pbits.Learned(r, net)
    for i in range(20):
        L0.step(1)
    acc_untrained = L0.accepted / L0.proposed
    losses, n_paths = _train(r, net, n, d)
    h = m.info()["h"]
    # a perfect network pays log 2 per H output and nothing else
    assert losses[-20:].mean() < losses[:5].mean()
    L1 = pbits.Learned(r, net)
    for i in range(20):
        L1.step(1)
        r.sweeps(1)
    acc_trained = L1.accepted / L1.proposed
    # the collected paths land in slots taken by an atomic counter, so their
    # order, the training batches and the trained network differ from run to
    # run: acceptance has been seen from about 0.49 up; untrained about 0.0015
    assert acc_trained > 0.4 and acc_trained > 20 * acc_untrained, (acc_untrained, acc_trained)


def test_trained_proposal_lowers_the_error_at_equal_steps():
    """What the trained network gains: the same number of steps (sweeps) with
    and without a suffix move per step; the error against the state vector
    (mean over amplitudes) is lower with the move."""
    n, d = 6, 12
    g = W.random_circuit(n, d, 71)
    J = W.default_J(n, d, g)
    exact = oracle.statevector(n, d, g)
    steps = 600
    _, plain = _run(n, d, g, J, 1024, 5)
    plain.sweeps(steps)
    psi_p, se_p = plain.amplitudes()
    _, lr = _run(n, d, g, J, 1024, 5)
    net = pbits.Mlp(n, d, hidden=128, batch=1024, seed=13)
    _train(lr, net, n, d)
    _, learned = _run(n, d, g, J, 1024, 5)
    L = pbits.Learned(learned, net)
    for _ in range(steps):
        L.step(1)
        learned.sweeps(1)
    psi_l, se_l = learned.amplitudes()
    err_p = np.mean(np.abs(psi_p - exact))
    err_l = np.mean(np.abs(psi_l - exact))
    assert np.all(np.abs(psi_l - exact) <= 5 * se_l + 1e-9)
    assert err_l < err_p and np.mean(se_l) < np.mean(se_p), (err_p, err_l, np.mean(se_p), np.mean(se_l))


def test_mh_keeps_the_distribution_with_x_gates():
    """X gates are deterministic links the proposal replays (the suffix's X
    bits flip): with an untrained network the move still keeps the law, so
    the amplitudes stay within 5 SE of the general oracle's state vector."""
    n, d = 4, 6
    g = W.random_circuit(n, d, 17).copy()
    for i in range(0, len(g), 2):
        if g[i, 0] in (W.S, W.T):
            g[i, 0] = W.X
    assert np.sum(g[:, 0] == W.X) > 0
    m, r = _run(n, d, g, W.default_J(n, d, g), 1024, 0x5EED + 17)
    net = pbits.Mlp(n, d, hidden=64, batch=1024, seed=12)
    L = pbits.Learned(r, net)
    for _ in range(2000):
        L.step(1)
        r.sweeps(1)
    psi, se = r.amplitudes()
    exact = oracle.u_statevector(n, d, g, None)
    err = np.abs(psi - exact)
    assert np.all(err <= 5 * se + 1e-9), (err, se)
    assert 0 < L.accepted < L.proposed
