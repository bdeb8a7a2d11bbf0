"""Pins of the FP64 MLP reference (oracle/mlp.py): finite differences,
closed forms of the loss, the Adam update on a case worked by hand."""
import numpy as np

from oracle import mlp as M


def _params(rng, k_in=24, h=32, n=5):
    return {"W1": rng.normal(0, 0.3, (h, k_in)), "b1": rng.normal(0, 0.1, h),
            "W2": rng.normal(0, 0.2, (h, h)), "b2": rng.normal(0, 0.1, h),
            "W3": rng.normal(0, 0.2, (n, h)), "b3": rng.normal(0, 0.1, n)}


def test_bce_closed_forms():
    # logits 0: each bit costs log 2
    assert abs(M.bce_loss(np.zeros((3, 4)), np.ones((3, 4))) - 4 * np.log(2)) < 1e-12
    # large correct logits cost ~0, large wrong logits cost ~|l|
    assert M.bce_loss(np.array([[30.0, -30.0]]), np.array([[1.0, 0.0]])) < 1e-12
    assert abs(M.bce_loss(np.array([[-30.0]]), np.array([[1.0]])) - 30.0) < 1e-9


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    x = rng.normal(0, 1, (7, 24))
    t = (rng.random((7, 5)) < 0.5).astype(float)
    g = M.backward(p, x, t, round_bf16=False)
    eps = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = M.bce_loss(M.forward(p, x, False)[0], t)
            flat[idx] = old - eps
            lm = M.bce_loss(M.forward(p, x, False)[0], t)
            flat[idx] = old
            num = (lp - lm) / (2 * eps)
            assert abs(num - g[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(num)), (name, idx)


def test_input_encoding():
    x = M.make_input(np.array([0b101, 0b010]), np.array([1, 3]), n=3, d=4, k_in=8)
    assert np.array_equal(x[0], [1, -1, 1, 1, 0, 0, 0, 0])
    assert np.array_equal(x[1], [-1, 1, -1, 0, 0, 1, 0, 0])


def test_adam_first_step_is_signed_lr():
    """With zero state, the bias-corrected first Adam step is -lr * g/(|g| + eps')."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    st = {}
    M.adam_step(p, g, st, lr=0.01, t=1)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(p["w"], want, atol=1e-12)


def test_bf16_rounding():
    assert M.bf16(np.array([1.0]))[0] == 1.0
    # 1 + 2^-8 is exactly halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert M.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert M.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert M.bf16(np.array([-3.14159]))[0] == -3.140625


def test_log_q_sums_to_one():
    rng = np.random.default_rng(2)
    logits = rng.normal(0, 2, (1, 4))
    total = sum(np.exp(M.log_q(logits, np.array([b])))[0] for b in range(16))
    assert abs(total - 1.0) < 1e-12
