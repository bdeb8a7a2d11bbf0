"""GPU proposal network (tcgen05 GEMMs) against the FP64 oracle of oracle/mlp.py.

The oracle computes in FP64 on the same bf16-rounded weights, inputs and
hidden activations the GPU feeds its tensor cores, so what remains is fp32
accumulation order and the bf16 rounding of backward intermediates: logits
within 2e-2 absolute; gradients per tensor within 2e-2 relative (L2) and
cosine >= 0.999; one Adam step within 1e-5 relative.
"""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2007_07379_gb300 import build, pbits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pbits.load()


def _batch(net, rows, seed):
    import torch
    rng = np.random.default_rng(seed)
    prev = rng.integers(0, 1 << net.n, size=rows, dtype=np.int64)
    layer = rng.integers(1, net.d + 1, size=rows)
    x = M.make_input(prev, layer, net.n, net.d, net.k_in)
    target = (rng.random((rows, net.n)) < 0.5).astype(np.float64)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda").to(torch.bfloat16)
    tt = torch.tensor(target, dtype=torch.float32, device="cuda")
    return x, target, xt, tt


def _oracle_params(net):
    p = net.params()
    return {k: v for k, v in p.items()}


@pytest.mark.parametrize("n,d,hidden,rows", [(16, 24, 256, 512), (5, 7, 64, 128), (24, 32, 256, 256)])
def test_forward_matches_oracle(n, d, hidden, rows):
    net = pbits.Mlp(n, d, hidden=hidden, batch=max(rows, 128), seed=3)
    x, _, xt, _ = _batch(net, rows, 1)
    got = net.forward(xt).cpu().numpy()
    p = _oracle_params(net)
    want, _ = M.forward({k: (v[:n] if k in ("W3", "b3") else v) for k, v in p.items()}, x)
    assert np.abs(got - want).max() < 2e-2 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("n,d,hidden,rows", [(16, 24, 256, 1024), (5, 7, 64, 256)])
def test_backward_matches_oracle(n, d, hidden, rows):
    net = pbits.Mlp(n, d, hidden=hidden, batch=rows, seed=4)
    x, target, xt, tt = _batch(net, rows, 2)
    loss = net.backward(xt, tt).item()
    g = net.grads()
    p = _oracle_params(net)
    po = {k: (v[:n] if k in ("W3", "b3") else v) for k, v in p.items()}
    want = M.backward(po, x, target)
    assert abs(loss - M.bce_loss(M.forward(po, x)[0], target)) < 1e-3 * max(1.0, loss)
    for name in want:
        a = g[name][:n] if name in ("W3", "b3") else g[name]
        b = want[name]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = np.sum(a * b) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        assert rel < 2e-2 and cos > 0.999, (name, rel, cos)


def test_adam_step_matches_oracle():
    net = pbits.Mlp(5, 7, hidden=64, batch=256, seed=5)
    x, target, xt, tt = _batch(net, 256, 3)
    net.backward(xt, tt)
    g = net.grads()
    p0 = net.params()
    net.adam(1e-3)
    p1 = net.params()
    want = {k: v.copy() for k, v in p0.items()}
    M.adam_step(want, g, {}, lr=1e-3, t=1)
    for k in want:
        assert np.allclose(p1[k], want[k], rtol=1e-5, atol=1e-6), k


def test_training_fits_a_deterministic_map():
    """Learning q(s_j | s_{j-1}) for a fixed bit map (target = permuted input
    bits): the loss must fall far below its initial log 2 per bit."""
    import torch
    n, d = 8, 4
    net = pbits.Mlp(n, d, hidden=64, batch=512, seed=6)
    rng = np.random.default_rng(9)
    losses = []
    for step in range(300):
        prev = rng.integers(0, 1 << n, size=512, dtype=np.int64)
        layer = rng.integers(1, d + 1, size=512)
        x = M.make_input(prev, layer, n, d, net.k_in)
        nxt = ((prev << 1) | (prev >> (n - 1))) & ((1 << n) - 1)
        tgt = np.stack([(nxt >> q) & 1 for q in range(n)], 1).astype(np.float32)
        loss = net.backward(torch.tensor(x, dtype=torch.float32, device="cuda").to(torch.bfloat16),
                            torch.tensor(tgt, device="cuda"))
        net.adam(3e-3)
        losses.append(loss.item())
    assert losses[0] > 0.5 * n * np.log(2)
    assert np.mean(losses[-20:]) < 0.05 * n * np.log(2), losses[-20:]


@pytest.mark.parametrize("n,d,hidden,rows", [(16, 24, 256, 4096), (24, 32, 256, 300), (5, 7, 64, 128),
                                             (6, 12, 128, 1024), (3, 4, 48, 130)])
def test_fused_forward_matches_layered_and_oracle(n, d, hidden, rows):
    net = pbits.Mlp(n, d, hidden=hidden, batch=((rows + 127) // 128) * 128, seed=8)
    x, _, xt, _ = _batch(net, rows, 4)
    fused = net.forward_fused(xt).cpu().numpy()
    layered = net.forward(xt).cpu().numpy()
    p = _oracle_params(net)
    want, _ = M.forward({k: (v[:n] if k in ("W3", "b3") else v) for k, v in p.items()}, x)
    scale = max(1.0, np.abs(want).max())
    assert np.abs(fused - want).max() < 2e-2 * scale
    assert np.abs(fused - layered).max() < 1e-3 * scale
