"""Column sampling of the period-finding circuit (Sec. 5.2) on the GPU
against the oracle's orc_shor_columns / orc_shor_prob_at."""
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


def _tol(N, a, n, x):
    """Per k: each FP32 phasor is within about 5e-7 of e^{i angle} (an exact
    integer phase rounded to FP32 and sincospif, times an FP32-rounded table
    entry), so |group sum|^2 moves by at most about 1e-6 g^2; the bound used,
    1e-5 sum_y g_y^2 / (2^n T), leaves a factor of ten."""
    y = np.array([pow(a, int(v), N) for v in x])
    _, g = np.unique(y, return_counts=True)
    return 1e-5 * float(np.sum(g.astype(np.float64) ** 2)) / (2 ** n * len(x)) + 1e-12


CASES = [(51, 2, 6, "all"), (21, 2, 5, 100), (15, 7, 4, "all"), (5, 2, 3, 7), (4001, 3, 12, 1),
         (60013, 7, 16, 300), (255, 2, 8, 1000)]


@pytest.mark.parametrize("N,a,n,T", CASES)
def test_full_vector_vs_oracle(N, a, n, T):
    rng = np.random.default_rng(N)
    x = (np.arange(2 ** n) if T == "all" else rng.integers(0, 2 ** n, T)).astype(np.uint32)
    sc = pbits.ShorColumns(n, len(x))
    y = sc.run(N, a, x, want_y=True)
    assert np.array_equal(y, [pow(a, int(v), N) for v in x])
    got = sc.prob.cpu().numpy()
    want, _ = oracle.shor_columns(N, a, n, x)
    assert np.all(np.abs(got - want) <= _tol(N, a, n, x))


def test_paper_case_sampled_and_peaks():
    """f(x) = 10424^x mod 98743069 (27 bits), 250 columns: sampled k (every
    peak neighbourhood and random k) against the oracle, total probability
    1, and the peak count at a threshold between the background and the
    peaks is the order 78."""
    wl = W.shor_paper()
    x = wl.columns()
    sc = pbits.ShorColumns(wl.n, wl.T)
    sc.run(wl.N, wl.a, x)
    M = 2 ** wl.n
    rng = np.random.default_rng(2)
    ks = np.unique(np.concatenate([
        [(int(round(j * M / wl.r)) + dd) % M for j in range(wl.r) for dd in (-1, 0, 1)],
        rng.integers(0, M, 3000)])).astype(np.uint64)
    import torch
    got = sc.prob[torch.as_tensor(ks.astype(np.int64), device=sc.prob.device)].cpu().numpy()
    want = oracle.shor_prob_at(wl.N, wl.a, wl.n, x, ks)
    assert np.all(np.abs(got - want) <= _tol(wl.N, wl.a, wl.n, x))
    assert abs(float(sc.prob.sum()) - 1.0) < 1e-4
    # background level 1/M; the peaks stand above 2.2/M at this sample count
    count, pos, mx = sc.peaks(2.2 / M, 4096)
    print("peaks", count, "max*M", mx * M)
    assert count == wl.r
    assert np.all(np.abs(pos.astype(np.float64) - np.arange(wl.r) * M / wl.r) <= 1.0)
