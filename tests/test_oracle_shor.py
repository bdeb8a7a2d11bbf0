"""Pins of the column-sampling oracle (Sec. 5.2) against Python's modular
power, the closed form of the order-finding distribution when r divides
2^n, Parseval, and an explicit psi table built in numpy."""
import numpy as np
import pytest

import oracle
from paper_2007_07379_gb300 import workloads as W


def test_modexp_matches_python_pow():
    rng = np.random.default_rng(3)
    for _ in range(200):
        N = int(rng.integers(2, 2 ** 32))
        a = int(rng.integers(0, N))
        x = int(rng.integers(0, 2 ** 32))
        assert oracle.modexp(a, x, N) == pow(a, x, N)
    assert oracle.modexp(10424, 78, 98743069) == 1          # the order of Sec. 5.3
    assert oracle.modexp(5, 479568, 961307) == 1            # the order of Table 1
    assert oracle.modexp(10424, 39, 98743069) != 1 and oracle.modexp(10424, 26, 98743069) != 1


@pytest.mark.parametrize("N,a,n,r", [(15, 7, 4, 4), (51, 2, 6, 8), (255, 2, 8, 8), (17, 3, 5, 16)])
def test_all_columns_give_the_exact_distribution(N, a, n, r):
    """Every column once (T = 2^n) with r | 2^n: probability 1/r at each
    multiple of 2^n / r, zero elsewhere."""
    assert pow(a, r, N) == 1 and (2 ** n) % r == 0
    prob, y = oracle.shor_columns(N, a, n, np.arange(2 ** n, dtype=np.uint32))
    want = np.zeros(2 ** n)
    want[:: 2 ** n // r] = 1.0 / r
    assert np.allclose(prob, want, atol=1e-12)
    assert np.array_equal(y, [pow(a, x, N) for x in range(2 ** n)])


def test_parseval_for_distinct_columns():
    rng = np.random.default_rng(5)
    for N, a, n in ((21, 2, 5), (391, 5, 9), (4001, 3, 12)):
        x = rng.choice(2 ** n, size=min(2 ** n, 97), replace=False).astype(np.uint32)
        prob, _ = oracle.shor_columns(N, a, n, x)
        assert abs(prob.sum() - 1.0) < 1e-12


def test_against_an_explicit_psi_table():
    """psi[k, y] += 2^{-n/2} e^{2 pi i k x / 2^n} per sample (duplicates
    included), prob = sum_y |psi|^2 / T -- built here directly."""
    rng = np.random.default_rng(7)
    for N, a, n, T in ((21, 2, 5, 40), (35, 3, 6, 25), (15, 2, 4, 9)):
        x = rng.integers(0, 2 ** n, T).astype(np.uint32)
        psi = np.zeros((2 ** n, N), dtype=np.complex128)
        k = np.arange(2 ** n)
        for xi in x:
            psi[:, pow(a, int(xi), N)] += 2 ** (-n / 2) * np.exp(2j * np.pi * k * int(xi) / 2 ** n)
        want = (np.abs(psi) ** 2).sum(axis=1) / T
        prob, _ = oracle.shor_columns(N, a, n, x)
        assert np.allclose(prob, want, atol=1e-12)
        at = oracle.shor_prob_at(N, a, n, x, np.array([0, 3, 2 ** n - 1], dtype=np.uint64))
        assert np.allclose(at, prob[[0, 3, 2 ** n - 1]], atol=1e-15)


def test_peaks_when_r_does_not_divide():
    """N = 21, a = 2 (r = 6), n = 5: all columns put r bumps near j 32 / 6."""
    prob, _ = oracle.shor_columns(21, 2, 5, np.arange(32, dtype=np.uint32))
    left, right = np.roll(prob, 1), np.roll(prob, -1)
    peaks = np.nonzero((prob >= left) & (prob > right) & (prob > 0.5 * prob.max()))[0]
    assert len(peaks) == 6
    assert np.all(np.abs(peaks - np.round(np.arange(6) * 32 / 6)) <= 1)


def test_workload_columns_are_reproducible():
    wl = W.shor_paper()
    x1, x2 = wl.columns(), wl.columns()
    assert np.array_equal(x1, x2) and len(x1) == 250 and x1.max() < 2 ** 27
    assert len(np.unique(x1)) == 250
