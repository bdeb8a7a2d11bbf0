"""Failure detection without a GPU fault.

Every wait the tensor-core kernels make (for an MMA commit or a bulk copy)
is bounded; one that runs out ends the kernel and records PB_ETIMEOUT in the
network's status word.  The wait itself is exercised by the library's
self-test on an mbarrier that nothing arrives at (no MMA, copy or tensor
memory in flight), after which the context must still compute bit-exact
results; the status of a network after forward, backward, training and MH
moves must stay PB_OK.
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


def test_bounded_wait_completes_when_arrived_on():
    assert pbits.selftest_wait(True, 1000) == pbits.PB_OK


def test_bounded_wait_runs_out_and_the_context_survives():
    assert pbits.selftest_wait(False, 64) == pbits.PB_ETIMEOUT
    assert pbits.selftest_wait(False, 1) == pbits.PB_ETIMEOUT
    # the same process then computes as before: a small run bit-exact vs the oracle
    n, d, chains, sweeps = 5, 7, 96, 20
    g = W.random_circuit(n, d, seed=17)
    m = pbits.Model(n, d, g, 3.0)
    r = pbits.Run([m], [pbits.RunCfg(seed=0x5EED, chains=chains)])
    r.sweeps(sweeps)
    r.wait()
    cnt, valid, _ = r.histogram()
    ref = oracle.gibbs(n, d, g, J=3.0, seed=0x5EED, chains=chains, sweeps=sweeps)
    assert np.array_equal(pbits.unslice_state(r.get_state(), chains), ref["state"])
    assert np.array_equal(cnt, ref["cnt"]) and valid == ref["valid"]
    assert pbits.selftest_wait(True, 1000) == pbits.PB_OK


def test_network_status_stays_ok_through_forward_backward_and_moves():
    import torch
    wl = W.tiny()
    m = pbits.Model(wl.n, wl.d, wl.gates, wl.J)
    r = pbits.Run([m], [pbits.RunCfg(seed=wl.seed, chains=256)])
    net = pbits.Mlp(wl.n, wl.d, hidden=64, batch=256, seed=3)
    assert net.status() == pbits.PB_OK
    x = torch.zeros((256, net.k_in), dtype=torch.bfloat16, device="cuda")
    x[:, : wl.n] = 1.0
    x[:, wl.n] = 1.0
    target = torch.zeros((256, wl.n), dtype=torch.float32, device="cuda")
    net.forward(x)
    net.forward_fused(x)
    net.backward(x, target)
    net.adam(1e-3)
    L = pbits.Learned(r, net)
    for _ in range(20):
        L.step(1)
        r.sweeps(1)
    r.wait()
    torch.cuda.synchronize()
    assert net.status() == pbits.PB_OK
    assert 0 < L.proposed
