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
