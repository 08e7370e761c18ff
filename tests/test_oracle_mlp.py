"""Pins for the oracle MLP: gradients against central finite differences, and Adam."""
import numpy as np

from oracle import mlp


def test_mlp_gradients_finite_difference():
    rng = np.random.default_rng(4)
    n_in, n_h, n_out, B = 12, 7, 5, 3
    p = mlp.init_params(n_in, n_h, n_out, seed=1)
    for k in p:
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)  # nonzero biases, no ReLU kinks at 0
    X = rng.standard_normal((B, n_in))
    T = rng.standard_normal((B, n_out))
    mask = np.ones((B, n_out))
    mask[2, 3:] = 0.0
    L, g = mlp.loss_and_grads(p, X, T, mask)
    eps = 1e-6
    for k in p:
        flat = p[k].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            Lp, _ = mlp.loss_and_grads(p, X, T, mask)
            flat[idx] = old - eps
            Lm, _ = mlp.loss_and_grads(p, X, T, mask)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * eps)
            assert abs(fd - g[k].ravel()[idx]) < 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_is_sign_times_lr():
    # with bias correction the first Adam step moves every parameter by lr * sign(grad)
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    mlp.adam_step(p, g, {}, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p["w"], [0.99, -1.99, 2.99], rtol=1e-12)


def test_bf16_rounding_is_torchs():
    """The oracle's bfloat16 rounding equals the library conversion float32 -> bfloat16
    (round to nearest, ties to even), including ties, subnormals and large values."""
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 1e-40, 3.4e38])])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_bf16_network_gradients_are_those_of_the_rounded_products():
    """With bf16=True every product operand is rounded: the gradients equal those of the
    FP64 network evaluated with the same rounded operands, which a hand expansion of one
    layer confirms (dW3 = bf16(dY)^T bf16(H2))."""
    rng = np.random.default_rng(6)
    n_in, n_h, n_out, B = 10, 6, 4, 5
    p = mlp.init_params(n_in, n_h, n_out, seed=2)
    X = rng.standard_normal((B, n_in))
    T = rng.standard_normal((B, n_out))
    mask = np.ones((B, n_out))
    L, g = mlp.loss_and_grads(p, X, T, mask, bf=True)
    W = {k: mlp.bf16(p[k]) for k in ("W1", "W2", "W3")}
    h1 = mlp.bf16(np.maximum(mlp.bf16(X) @ W["W1"].T + p["b1"], 0))
    h2 = mlp.bf16(np.maximum(h1 @ W["W2"].T + p["b2"], 0))
    y = h2 @ W["W3"].T + p["b3"]
    dy = 2 * (y - T) / mask.sum()
    np.testing.assert_allclose(g["W3"], mlp.bf16(dy).T @ h2, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(L, ((y - T) ** 2).sum() / mask.sum(), rtol=1e-14)
    # rounding changes the gradients at the bfloat16 level, not more
    _, g64 = mlp.loss_and_grads(p, X, T, mask)
    for k in g:
        assert np.max(np.abs(g[k] - g64[k])) <= 0.05 * np.max(np.abs(g64[k])) + 1e-12, k
