"""Amplitude parity of the GPU Gibbs sampler with the FP64 state vector on
every workload, in each workload's launch configuration (Eq. U23 estimator,
Eqs. U26 / U30 error law).

Standard errors.  Per output alpha the per-sample estimator
X = 2^{h/2} [end = alpha] w^phi has E X = psi_alpha and E|X|^2 = N_alpha,
the number of valid paths ending at alpha (2^{h - rank} or 0, from the
oracle), so i.i.d. samples give the closed-form error
se_cf = sqrt((N_alpha - |psi_alpha|^2) / T), T = valid samples.  A Gibbs
chain's records are correlated: the run's batch means over chain groups
(se_bm) include that, and the pooled ratio rho = rms(se_bm) / rms(se_cf)
over the reached outputs measures it (rho^2 = the integrated
autocorrelation time in records).  The error a bin is tested against is
SE = max(se_bm, rho' se_cf), rho' = max(rho, 1): the closed form scaled by
the pooled autocorrelation factor, never below the bin's own batch-means
estimate.  Acceptance:
  * |psi_hat - psi| <= 5 SE for every reached output whose expected count
    T N_alpha / 2^h is at least 16 (a sum of that many unit phasors is close
    enough to normal for a per-bin test); sparser outputs are tested
    together: their mean squared error is at most 25 times their mean SE^2;
  * outputs no valid path reaches read exactly 0;
  * rho >= 0.8 always (the batch means never fall below the i.i.d. floor),
    and 0.8 <= rho <= 1.2 where the records are independent: the learned and
    large workloads as run, the mid workload with records every 8th sweep;
  * within 1e-3 absolute where 5 SE reaches 1e-3: the batched circuits with
    the fewest paths per output, run to convergence (at the batched budget
    of 1e4 sweeps no circuit gets there: the smallest 5 SE is about 6e-3).
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


def _check(name, psi, se_bm, exact, N, valid, h, iid=None):
    """The acceptance above for one model; returns (rho, max z)."""
    reach = N > 0
    assert np.all(psi[~reach] == 0), f"{name}: an unreachable output has a nonzero estimate"
    se_cf = np.sqrt(np.maximum(N - np.abs(exact) ** 2, 0.0) / valid)
    rho = float(np.sqrt(np.mean(se_bm[reach] ** 2) / np.mean(se_cf[reach] ** 2)))
    se = np.maximum(se_bm, max(rho, 1.0) * se_cf)
    err = np.abs(psi - exact)
    dense = reach & (valid * N / 2.0 ** h >= 16)
    sparse = reach & ~dense
    z = err[dense] / se[dense]
    zmax = float(z.max()) if z.size else 0.0
    print(f"{name}: valid {valid}, reached {int(reach.sum())}, dense {int(dense.sum())}, "
          f"rho {rho:.4f}, max z {zmax:.2f}")
    assert zmax <= 5.0, f"{name}: max |psi_hat - psi| / SE = {zmax:.2f}"
    if sparse.any():
        ms = float(np.mean(err[sparse] ** 2) / np.mean(se[sparse] ** 2))
        assert ms <= 25.0, f"{name}: sparse outputs, mean squared error / SE^2 = {ms:.2f}"
    assert rho >= 0.8, f"{name}: batch-means SE below the i.i.d. floor ({rho:.3f})"
    if iid:
        assert rho <= 1.2, f"{name}: batch-means and closed-form SE differ by more than 20% ({rho:.3f})"
    return rho, zmax


def _run(wl, chains=None, sweeps=None, n_batches=32, record_every=1, alphas=None, seed=None):
    m = pbits.Model(wl.n, wl.d, wl.gates, wl.J)
    r = pbits.Run([m], [pbits.RunCfg(seed=wl.seed if seed is None else seed,
                                     chains=chains or wl.chains, n_batches=n_batches,
                                     record_every=record_every, alphas=alphas)])
    if sweeps:
        r.sweeps(sweeps)
        r.wait()
    return m, r


def test_mid_workload_amplitudes():
    """Mid workload at its budget (4096 chains x 1e5 sweeps): all 4096
    amplitudes, psi_0 among them, within 5 SE of the state vector; the
    chain's records are correlated (rho about 1.3), and with every 8th
    sweep recorded the two error estimates agree within 20%."""
    wl = W.mid()
    exact = oracle.statevector(wl.n, wl.d, wl.gates)
    N = oracle.valid_paths_per_output(wl.n, wl.d, wl.gates)
    m, r = _run(wl, sweeps=100_000)
    h = m.info()["h"]
    psi, se = r.amplitudes()
    _, valid, samples = r.histogram()
    assert samples == wl.chains * 100_000
    rho, _ = _check("mid", psi, se, exact, N, valid, h)
    se0 = max(se[0], max(rho, 1.0) * np.sqrt((N[0] - abs(exact[0]) ** 2) / valid))
    assert abs(psi[0] - exact[0]) <= 5 * se0
    m, r = _run(wl, sweeps=100_000, record_every=8, seed=wl.seed + 1)
    psi, se = r.amplitudes()
    _, valid, _ = r.histogram()
    _check("mid, every 8th sweep", psi, se, exact, N, valid, h, iid=True)


def _train(r, net, d, sweeps=60, steps=300):
    import torch
    cap = 1 << 18
    paths = torch.zeros((cap, d), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    L = pbits.Learned(r, net)
    r.sweeps(100)
    for _ in range(sweeps):
        r.sweeps(2)
        L.collect(paths, count)
    n_paths = min(int(count.item()), cap)
    pbits.train_on_paths(net, paths, n_paths, 0, steps=steps, rows=4096, lr=1e-3, seed=5)
    torch.cuda.synchronize()
    L.close()


def test_learned_workload_amplitudes_plain_and_learned():
    """Learned workload (n=16, d=24, 4096 chains): plain Gibbs (2e4 sweeps)
    and the PB_LEARNED run mode with a suffix move per sweep from a trained
    network (1e4 moves and sweeps in one pb_run_sweeps call), each against
    the 65,536-amplitude state vector."""
    wl = W.learned()
    exact = oracle.statevector(wl.n, wl.d, wl.gates)
    N = oracle.valid_paths_per_output(wl.n, wl.d, wl.gates)
    m, r = _run(wl, sweeps=20_000)
    h = m.info()["h"]
    psi, se = r.amplitudes()
    _, valid, _ = r.histogram()
    _check("learned, plain", psi, se, exact, N, valid, h, iid=True)

    _, src = _run(wl, seed=wl.seed + 100)
    net = pbits.Mlp(wl.n, wl.d, hidden=256, batch=4096, seed=21)
    _train(src, net, wl.d)
    # the learned sampler as a run mode: one graph, a move before every sweep
    r = pbits.Run([m], [pbits.RunCfg(seed=wl.seed + 2, chains=wl.chains, n_batches=32,
                                     sampler=pbits.PB_LEARNED, proposal=net, mh_every=1)])
    r.sweeps(10_000)
    r.wait()
    moves, acc = r.moves()
    assert moves == 10_000 and acc > 0
    print(f"learned move acceptance {acc / (moves * wl.chains):.4f}")
    psi, se = r.amplitudes()
    _, valid, _ = r.histogram()
    _check("learned, with moves", psi, se, exact, N, valid, h)


def test_large_workload_amplitudes():
    """Large workload (n=24, d=32, 65536 chains, 1e4 sweeps): the 64 output
    amplitudes against the 2^24-entry FP64 state vector."""
    wl = W.large()
    exact = oracle.statevector(wl.n, wl.d, wl.gates)[wl.alphas]
    N = oracle.valid_paths_per_output(wl.n, wl.d, wl.gates, alphas=wl.alphas)
    m, r = _run(wl, sweeps=10_000, alphas=wl.alphas)
    psi, se = r.amplitudes()
    _, valid, _ = r.histogram()
    _check("large", psi, se, exact, N, valid, m.info()["h"], iid=True)


def test_batched_workload_amplitudes():
    """Batched workload (256 circuits in one persistent launch, 1e4 sweeps,
    16 batches per circuit where it has that many chain groups): every
    circuit's amplitudes against its own state vector."""
    wls = W.batched()
    models = [pbits.Model(w.n, w.d, w.gates, w.J) for w in wls]
    r = pbits.Run(models, [pbits.RunCfg(seed=w.seed, chains=w.chains, n_batches=16) for w in wls])
    r.sweeps(10_000)
    r.wait()
    rhos, smallest = [], []
    for i, w in enumerate(wls):
        exact = oracle.statevector(w.n, w.d, w.gates)
        N = oracle.valid_paths_per_output(w.n, w.d, w.gates)
        psi, se = r.amplitudes(i)
        _, valid, samples = r.histogram(i)
        assert samples == w.chains * 10_000
        h = models[i].info()["h"]
        rho, _ = _check(f"batched[{i}] n={w.n} d={w.d}", psi, se, exact, N, valid, h)
        rhos.append(rho)
        smallest.append(5 * max(rho, 1.0) * np.sqrt(N[N > 0].min() / valid))
    print(f"batched rho min/median/max {min(rhos):.3f}/{np.median(rhos):.3f}/{max(rhos):.3f}; "
          f"smallest 5 SE at budget {min(smallest):.2e}")


def test_batched_small_circuits_converge_to_1e_3():
    """The three batched circuits with the fewest valid paths per output,
    run alone to convergence (65536 chains x 1e5 sweeps): 5 SE falls below
    1e-3 and every amplitude is within 1e-3 of the state vector."""
    wls = W.batched()
    ranked = sorted(range(len(wls)), key=lambda i: (lambda hr: hr[0] - hr[1])(
        oracle.gf2_rank(wls[i].n, wls[i].d, wls[i].gates)))
    for i in ranked[:3]:
        w = wls[i]
        exact = oracle.statevector(w.n, w.d, w.gates)
        N = oracle.valid_paths_per_output(w.n, w.d, w.gates)
        m, r = _run(w, chains=65536, sweeps=100_000)
        psi, se = r.amplitudes()
        _, valid, _ = r.histogram()
        rho, _ = _check(f"batched[{i}] converged", psi, se, exact, N, valid, m.info()["h"])
        se_max = max(rho, 1.0) * np.sqrt(N[N > 0].max() / valid)
        err = np.abs(psi - exact).max()
        print(f"batched[{i}]: 5 SE {5 * se_max:.2e}, max error {err:.2e}")
        assert 5 * se_max <= 1e-3 and err <= 1e-3
