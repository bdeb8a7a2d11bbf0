"""FP64 reference of the learned proposal network (test infrastructure only).

The paper trains nothing (its weights are "one-shot", from the gate
matrices); the proposal network is an addition to the sampler of
Fig. 2 Step 1, so its reference is the textbook definition, written plainly:

  q(s_j | s_{j-1}, j) = prod_q sigma(l_q)^{s_j[q]} sigma(-l_q)^{1-s_j[q]},
  l = W3 relu(W2 relu(W1 x + b1) + b2) + b3,
  x = [2 s_{j-1} - 1 (n entries), onehot(j-1) (d entries), zeros] (K_in),

loss = mean over the batch of the binary cross-entropy
-sum_q [t_q log sigma(l_q) + (1 - t_q) log sigma(-l_q)], gradients by the chain
rule, and one Adam step (Kingma & Ba, 2015).  Precision policy: the GPU feeds
bf16 inputs, weights and hidden activations to the tensor cores; the
reference takes the same bf16-rounded values (`bf16` below) and computes in
FP64, so the remaining difference is the GPU's fp32 accumulation.

Pinned by tests/test_oracle_mlp.py against central finite differences and
closed forms of the loss.
"""
from __future__ import annotations

import numpy as np


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) and return as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def make_input(prev_bits: np.ndarray, layer: np.ndarray, n: int, d: int, k_in: int) -> np.ndarray:
    """Rows x = [2 s_{j-1} - 1, onehot(j-1), 0...]; prev_bits[B] are n-bit words, layer[B] = j."""
    B = len(prev_bits)
    x = np.zeros((B, k_in))
    for q in range(n):
        x[:, q] = 2.0 * ((prev_bits >> q) & 1) - 1.0
    x[np.arange(B), n + (np.asarray(layer) - 1)] = 1.0
    return x


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def forward(params: dict, x: np.ndarray, round_bf16: bool = True):
    """Logits and the hidden activations (as the GPU stores them)."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3 = r(params["W1"]), r(params["W2"]), r(params["W3"])
    x = r(x)
    z1 = x @ W1.T + params["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + params["b2"]
    h2 = r(np.maximum(z2, 0.0))
    logits = h2 @ W3.T + params["b3"]
    return logits, (x, h1, h2)


def bce_loss(logits: np.ndarray, target: np.ndarray) -> float:
    """Mean over rows of -sum_q [t log sigma(l) + (1-t) log sigma(-l)]."""
    # log sigma(l) = -log(1 + e^{-l}), evaluated stably
    ls = -np.logaddexp(0.0, -logits)
    lns = -np.logaddexp(0.0, logits)
    return float(-np.mean(np.sum(target * ls + (1.0 - target) * lns, axis=1)))


def backward(params: dict, x: np.ndarray, target: np.ndarray, round_bf16: bool = True) -> dict:
    """Gradients of bce_loss w.r.t. the fp32 master parameters (chain rule)."""
    logits, (xr, h1, h2) = forward(params, x, round_bf16)
    B = x.shape[0]
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W2, W3 = r(params["W2"]), r(params["W3"])
    dl = (sigmoid(logits) - target) / B
    g = {"W3": dl.T @ h2, "b3": dl.sum(0)}
    dh2 = dl @ W3
    dz2 = dh2 * (h2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (h1 > 0)
    g["W1"] = dz1.T @ xr
    g["b1"] = dz1.sum(0)
    return g


def adam_step(params: dict, grads: dict, state: dict, lr: float, t: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place; state holds m, v per parameter; t = step (1-based)."""
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)


def log_q(logits: np.ndarray, bits: np.ndarray) -> np.ndarray:
    """log q of n-bit words under the logits (per row)."""
    n = logits.shape[1]
    t = np.stack([((bits >> q) & 1) for q in range(n)], axis=1).astype(np.float64)
    return np.sum(t * -np.logaddexp(0.0, -logits) + (1 - t) * -np.logaddexp(0.0, logits), axis=1)
