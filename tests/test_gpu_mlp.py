"""Learned initial guess on the GPU: gradients against the FP64 oracle, and its gain."""
import numpy as np
import pytest

import synth
from oracle import mlp

pytestmark = pytest.mark.gpu


def _solver(name, **opt):
    from paper_2101_02959_gb300 import binding, build
    build.build()
    return binding.Solver(synth.workload(name), synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, **opt)


@pytest.mark.parametrize("name", ["ragged", "slab128"])
def test_mlp_loss_and_gradients_match_oracle(name):
    """The tensor-core network (bf16 operands, FP32 accumulation) against the oracle's
    FP64 network with the same bf16 rounding points: loss, and every gradient entry
    against its block's largest entry.  What remains is FP32 accumulation order and the
    rare bf16 rounding of an activation that lands on the other side of a midpoint."""
    s = _solver(name, learned_guess=1, precision="mixed")
    sz = s.mlp_sizes()
    n_in, H, n_out, B = sz["n_in"], sz["n_hidden"], sz["n_out"], sz["batch"]
    assert n_in % 6 == 0 and n_out * 3 == n_in
    if name == "slab128":  # the 128x128x32 slab: 386 interface nodes per H/h = 8 subdomain
        assert (n_in, H, n_out, B) == (2316, 256, 772, 1024)
    rng = np.random.default_rng(7)
    p = mlp.init_params(n_in, H, n_out, seed=3)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.01 * rng.standard_normal(p[k].shape)
    for k in ("W1", "W2", "W3"):
        p[k] = mlp.bf16(p[k])  # the GPU's masters are FP32; these are exact in bf16 already
    w = np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])
    s.mlp_params(w.astype(np.float32))
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    T = (0.1 * rng.standard_normal((B, n_out))).astype(np.float32)
    mask = (rng.random((B, n_out)) < 0.8).astype(np.float32)
    loss, g = s.mlp_loss_grad(X, T, mask)
    L, gr = mlp.loss_and_grads(p, X.astype(np.float64), T.astype(np.float64), mask.astype(np.float64), bf=True)
    assert abs(loss - L) < 1e-4 * L
    # bars: a bf16 rounding point whose FP32 value (GPU) and FP64 value (oracle) fall on the
    # two sides of a rounding midpoint rounds 2^-8 apart; over a batch the number of such
    # flips grows, and a numpy FP32 run of the same network differs from the oracle by
    # 1e-8 (batch 18) and 2.3e-4 (batch 1,024, 2,316 inputs) in the W1 gradient's norm;
    # the tensor cores' FP32 accumulation order adds a factor of about 3
    tol_norm, tol_max = (5e-4, 2e-3) if B <= 64 else (2e-3, 5e-3)
    off = 0
    for k, shape in (("W1", (H, n_in)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (n_out, H)),
                     ("b3", (n_out,))):
        n = int(np.prod(shape))
        got = g[off:off + n].astype(np.float64)
        ref = gr[k].ravel()
        assert np.linalg.norm(got - ref) <= tol_norm * np.linalg.norm(ref), k
        assert np.max(np.abs(got - ref)) <= tol_max * np.max(np.abs(ref)), k  # entry by entry
        off += n
    assert off == g.size
    s.close()


def test_adam_matches_oracle_over_steps():
    """The GPU's Adam update (FP32) against the oracle's adam_step (FP64) over six steps
    with gradients spanning three decades, entry by entry."""
    s = _solver("cube8ve", learned_guess=1)
    w0 = s.mlp_params()
    rng = np.random.default_rng(11)
    p = {"w": w0.astype(np.float64)}
    st = {}
    for _ in range(6):
        g = (rng.choice([-1.0, 1.0], w0.size) * 10.0 ** rng.uniform(-3, 0, w0.size)).astype(np.float32)
        s.mlp_adam_step(g, 1e-3)
        mlp.adam_step(p, {"w": g.astype(np.float64)}, st, lr=1e-3)
    got = s.mlp_params().astype(np.float64)
    moved = np.abs(p["w"] - w0)
    assert np.median(moved) > 1e-3  # the steps really moved the weights (about lr each)
    # FP32 weights: a few units in the last place of each weight, plus FP32 rounding of
    # the updates (each about lr in size)
    ulp = np.spacing(np.maximum(np.abs(w0), np.abs(got)).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(got - p["w"]) <= 8 * ulp + 6 * 1e-3 * 1e-6)
    s.mlp_reset()
    np.testing.assert_array_equal(s.mlp_params(), w0)  # back to the initial draw


def _run(name, steps, **opt):
    s = _solver(name, **opt)
    ui, ue, w = synth.initial_state(s.N, 0)
    s.set_state(ui, ue, w, 0.0)
    stats = [s.step(synth.STIMULUS) for _ in range(steps)]
    out = s.get_state()
    s.close()
    return stats, out


def test_learned_guess_gain_and_agreement():
    """Trained online, the guess beats the previous-step state and saves Krylov iterations."""
    steps = 40
    base, (bi, be, _, _) = _run("cube8ve", steps)
    lg, (li, le, _, _) = _run("cube8ve", steps, learned_guess=1, mlp_train_steps=steps, mlp_warmup=5)
    assert all(st["reason"] == 0 for st in base + lg)
    late = lg[15:]
    used = [st for st in late if st["guess_used"]]
    assert len(used) >= 0.6 * len(late)
    ratio = np.median([st["res_guess"] / st["res0"] for st in late])
    assert ratio < 0.6
    kry_base = sum(st["krylov_its"] for st in base[15:])
    kry_lg = sum(st["krylov_its"] for st in late)
    assert kry_lg < kry_base
    # both runs satisfy the same anchored Newton test: states agree to the SNES tolerance level
    assert np.linalg.norm(le - be) / np.linalg.norm(be) < 1e-3
    assert np.linalg.norm((li - le) - (bi - be)) / np.linalg.norm(bi - be) < 1e-3
    print(f"krylov its (last {len(late)} steps): previous-step guess {kry_base}, learned guess {kry_lg}; "
          f"median residual ratio {ratio:.3f}")
