"""The no-allocation run (pb_gibbs_run_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory at the call site, so
its scratch is the library's fixed device array.  Two calls in a row must
each reproduce the histogram and totals of the regular run (pb_run_create +
pb_run_sweeps) bit for bit: the counts are integers, so the tolerance the
other parity tests use for integers, exact equality, applies.  The file is
named to run last, after every other test, and also passes alone.
"""
import numpy as np
import pytest

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


def test_noalloc_matches_regular_run_twice():
    import torch
    n, d, chains, sweeps = 7, 11, 200, 30
    g = W.random_circuit(n, d, seed=77)
    m = pbits.Model(n, d, g, 3.0)
    cfg = pbits.RunCfg(seed=0x5EED + 9, chains=chains)
    r = pbits.Run([m], [cfg])
    r.sweeps(sweeps)
    want_cnt, want_valid, want_samples = r.histogram()
    for call in range(2):
        counts = torch.full(((1 << n) * 8,), -1, dtype=torch.int64, device="cuda")
        totals = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        pbits.gibbs_run_noalloc(m, cfg, sweeps, counts, totals)
        torch.cuda.synchronize()
        got = counts.cpu().numpy().view(np.uint64).reshape(-1, 8)
        tot = totals.cpu().numpy()
        assert np.array_equal(got, want_cnt), f"call {call}: histogram differs"
        assert int(tot[0]) == want_valid and int(tot[1]) == want_samples, f"call {call}"


def test_noalloc_global_histogram_matches_regular_run():
    """n = 14: the 2^14-bin histogram does not fit in shared memory, so the
    recorders add every count to the array's histogram in global memory
    (cleared by the call itself); still bit-identical to the regular run,
    on two calls in a row."""
    import torch
    n, d, chains, sweeps = 14, 5, 96, 12
    g = W.random_circuit(n, d, seed=78)
    m = pbits.Model(n, d, g, 3.0)
    cfg = pbits.RunCfg(seed=0x5EED + 10, chains=chains)
    r = pbits.Run([m], [cfg])
    r.sweeps(sweeps)
    want_cnt, want_valid, want_samples = r.histogram()
    assert want_valid > 0
    for call in range(2):
        counts = torch.full(((1 << n) * 8,), -1, dtype=torch.int64, device="cuda")
        totals = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        pbits.gibbs_run_noalloc(m, cfg, sweeps, counts, totals)
        torch.cuda.synchronize()
        got = counts.cpu().numpy().view(np.uint64).reshape(-1, 8)
        tot = totals.cpu().numpy()
        assert np.array_equal(got, want_cnt), f"call {call}: histogram differs"
        assert int(tot[0]) == want_valid and int(tot[1]) == want_samples, f"call {call}"


def test_noalloc_refuses_stream_capture():
    """The call copies host tables, so it cannot be recorded into a graph:
    on a capturing stream it returns PB_ESTATE and enqueues nothing."""
    import torch
    n, d = 5, 6
    m = pbits.Model(n, d, W.random_circuit(n, d, seed=79), 3.0)
    cfg = pbits.RunCfg(seed=3, chains=64)
    counts = torch.zeros((1 << n) * 8, dtype=torch.int64, device="cuda")
    totals = torch.zeros(2, dtype=torch.int64, device="cuda")
    pbits.gibbs_run_noalloc(m, cfg, 2, counts, totals)  # first call on the device: set-up
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(graph, stream=s):
        try:
            pbits.gibbs_run_noalloc(m, cfg, 2, counts, totals, stream=s)
        except pbits.PbError as e:
            err = e
    assert err is not None and err.code == pbits.PB_ESTATE


def test_noalloc_rejects_oversize():
    import torch
    g = W.random_circuit(12, 20, seed=1)
    m = pbits.Model(12, 20, g, 3.0)
    counts = torch.zeros(4096 * 8, dtype=torch.int64, device="cuda")
    totals = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(pbits.PbError) as e:
        pbits.gibbs_run_noalloc(m, pbits.RunCfg(seed=1, chains=1 << 20), 1, counts, totals)
    assert e.value.code == pbits.PB_ERANGE


def test_noalloc_rejects_general_gate_models():
    """Models with general one-qubit gates carry complex phase sums, which
    the fixed scratch does not hold: the call is refused before any launch."""
    import torch
    g, mats = W.random_general_circuit(5, 8, 3, frac_u=0.5)
    m = pbits.Model(5, 8, g, 3.0, mats=mats)
    assert m.info()["n_u"] > 0
    counts = torch.zeros(32 * 8, dtype=torch.int64, device="cuda")
    totals = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(pbits.PbError) as e:
        pbits.gibbs_run_noalloc(m, pbits.RunCfg(seed=1, chains=64), 1, counts, totals)
    assert e.value.code == pbits.PB_EINVAL
