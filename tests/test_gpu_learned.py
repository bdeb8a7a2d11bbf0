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


def _trained_network(n, d, g, J):
    """A network trained on paths collected from a fresh run (same seeds
    every call), and that run."""
    m, r = _run(n, d, g, J, 1024, 99)
    net = pbits.Mlp(n, d, hidden=128, batch=1024, seed=12)
    L0 = pbits.Learned(r, net)
    for i in range(20):
        L0.step(1)
    acc_untrained = L0.accepted / L0.proposed
    losses, n_paths = _train(r, net, n, d)
    return m, r, net, losses, acc_untrained


def test_training_on_collected_paths_raises_acceptance():
    """Collected paths are written in chain order and every reduction of the
    training step runs in a fixed order, so two trainings from the same
    seeds give bit-identical weights; the trained network is accepted about
    half the time (an untrained one about 0.0015)."""
    n, d = 6, 8
    g = W.random_circuit(n, d, 61)
    J = W.default_J(n, d, g)
    m, r, net, losses, acc_untrained = _trained_network(n, d, g, J)
    _, _, net2, losses2, _ = _trained_network(n, d, g, J)
    p1, p2 = net.params(), net2.params()
    for name in p1:
        assert np.array_equal(p1[name], p2[name]), f"{name} differs between two trainings"
    assert np.array_equal(losses, losses2)
    # a perfect network pays log 2 per H output and nothing else
    assert losses[-20:].mean() < losses[:5].mean()
    L1 = pbits.Learned(r, net)
    for i in range(20):
        L1.step(1)
        r.sweeps(1)
    acc_trained = L1.accepted / L1.proposed
    assert acc_trained > 0.5 and acc_trained > 20 * acc_untrained, (acc_untrained, acc_trained)


def _learned_cfg(seed, chains, net, mh_every, **kw):
    return pbits.RunCfg(seed=seed, chains=chains, n_batches=32, sampler=pbits.PB_LEARNED, proposal=net,
                        mh_every=mh_every, **kw)


def test_learned_run_mode_equals_manual_moves():
    """PB_LEARNED: pb_run_sweeps(2 * 60 + 1) with mh_every = 2 (60 device-side
    periods of a move and 2 sweeps, then one sweep) is bit for bit the same
    run as a PB_GIBBS run driven from the host: 60 x (one pb_mh move, 2
    sweeps), then one sweep -- chain words, histogram, move and acceptance
    counts; a second call continues both alike."""
    n, d = 6, 8
    g = W.random_circuit(n, d, 61)
    J = W.default_J(n, d, g)
    _, _, net, _, _ = _trained_network(n, d, g, J)
    m = pbits.Model(n, d, g, J)
    a = pbits.Run([m], [_learned_cfg(77, 1000, net, 2)])
    b = pbits.Run([m], [pbits.RunCfg(seed=77, chains=1000, n_batches=32)])
    L = pbits.Learned(b, net)
    for call in range(2):
        a.sweeps(121)
        for _ in range(60):
            L.step(1)
            b.sweeps(2)
        b.sweeps(1)
        a.wait()
        b.wait()
        assert np.array_equal(a.get_state(), b.get_state()), call
        ca, va, sa = a.histogram()
        cb, vb, sb = b.histogram()
        assert np.array_equal(ca, cb) and va == vb and sa == sb, call
        mv, acc = a.moves()
        assert mv == 60 * (call + 1) and (mv, acc) == L.stats(), (mv, acc, L.stats())
    assert acc > 0


def test_learned_run_mode_checkpoint_restore():
    """A learned run restored from a checkpoint (chain words, counters and
    the move counters) continues bit-identically."""
    n, d = 5, 7
    g = W.random_circuit(n, d, 62)
    J = W.default_J(n, d, g)
    net = pbits.Mlp(n, d, hidden=64, batch=1024, seed=3)
    m = pbits.Model(n, d, g, J)
    a = pbits.Run([m], [_learned_cfg(5, 256, net, 3)])
    a.sweeps(30)
    blob = a.checkpoint()
    a.sweeps(31)
    b = pbits.Run([m], [_learned_cfg(5, 256, net, 3)])
    b.restore(blob)
    b.sweeps(31)
    assert np.array_equal(a.get_state(), b.get_state())
    assert np.array_equal(a.histogram()[0], b.histogram()[0])
    assert a.moves() == b.moves() and a.moves()[0] == 20


def test_learned_run_mode_rejects_bad_configs():
    n, d = 5, 7
    g = W.random_circuit(n, d, 63)
    m = pbits.Model(n, d, g, 3.0)
    net = pbits.Mlp(n, d, hidden=64, batch=1024, seed=3)
    other = pbits.Mlp(n, d + 1, hidden=64, batch=1024, seed=3)
    gu, mats = W.random_general_circuit(n, d, 3, frac_u=0.5)
    mu = pbits.Model(n, d, gu, 3.0, mats=mats)
    bad = [(m, _learned_cfg(1, 64, None, 1)), (m, _learned_cfg(1, 64, net, 0)),
           (m, _learned_cfg(1, 64, other, 1)), (mu, _learned_cfg(1, 64, net, 1))]
    for model, cfg in bad:
        with pytest.raises(pbits.PbError) as e:
            pbits.Run([model], [cfg])
        assert e.value.code == pbits.PB_EINVAL
    plain = pbits.Run([m], [pbits.RunCfg(seed=1, chains=64)])
    with pytest.raises(pbits.PbError) as e:
        plain.moves()
    assert e.value.code == pbits.PB_ESTATE


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
