"""Pins of oracle parts whose correctness a plain re-run cannot show.

* The cubic backtracking line search of the Newton step (Section 6 uses the PETSc
  SNES defaults; the published algorithm is Dennis and Schnabel A6.3.1): on
  functions that are exactly a quadratic or a cubic in the step length, the first
  backtrack must land on the quadratic's minimiser and the second on the cubic's,
  whose values are worked out by hand below.  A wrong coefficient, sign or root
  branch moves them.
* The same line search on a real Newton step of the method that does backtrack
  (tau = 0.3 ms, a state near the excitation threshold).
* Adam (Kingma and Ba, Algorithm 1) for two steps against values worked out in
  exact decimal arithmetic, and its bias correction for t > 1 by the invariant
  that a constant gradient moves every step by lr g / (|g| + eps).
* Optimality (Section 5, Theorem; Section 6, Test 3): the condition number of the
  BDDC deluxe operator with vertex and edge constraints grows at most like
  (1 + log H/h)^2 and the vertex-only one much faster.
"""
import os

import numpy as np
import pytest

import synth
from oracle import bidomain, mlp
from oracle.bidomain import Problem, direct_solve, line_search_bt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


class _Cubic:
    """trial(lam) = ||R(u + lam s)||^2 = 2 f(lam) with f = 1 - 2 lam + b lam^2 + a lam^3:
    f(0) = 1 and f'(0) = -2 = -||R||^2, the values the line search assumes."""

    def __init__(self, a, b):
        self.a, self.b, self.calls = a, b, []

    def __call__(self, lam):
        self.calls.append(lam)
        return 2.0 * (1.0 - 2.0 * lam + self.b * lam ** 2 + self.a * lam ** 3)


def test_line_search_first_backtrack_is_the_quadratic_minimiser():
    # f = 1 - 2 lam + 4 lam^2: f(1) = 3 fails the test; the quadratic through f(0), f'(0),
    # f(1) is f itself, minimised at lam = 2 / (2 * 4) = 0.25, where f = 0.75 passes.
    tr = _Cubic(0.0, 4.0)
    lam, g, ok = line_search_bt(2.0, tr)
    assert ok and tr.calls == [1.0, 0.25]
    assert lam == 0.25 and abs(g - 1.5) < 1e-15


@pytest.mark.parametrize("a,b,lam2", [
    # f = 1 - 2 lam + 1000 lam^3: f(1) fails, the quadratic step 1 / 1000 is raised to the
    # floor 0.1, f(0.1) = 1.8 fails; the cubic through f(0), f'(0), f(1), f(0.1) is f, whose
    # minimiser solves f' = -2 + 3000 lam^2 = 0: lam = sqrt(6 / 1000) / 3.
    (1000.0, 0.0, 0.025819888974716113),
    # f = 1 - 2 lam + 50 lam^2 + 500 lam^3: f' = -2 + 100 lam + 1500 lam^2 = 0 gives
    # lam = (-50 + sqrt(2500 + 3000)) / 1500.
    (500.0, 50.0, 0.016107989913971087),
])
def test_line_search_second_backtrack_is_the_cubic_minimiser(a, b, lam2):
    tr = _Cubic(a, b)
    lam, g, ok = line_search_bt(2.0, tr)
    assert ok
    assert tr.calls[:2] == [1.0, 0.1]
    assert abs(tr.calls[2] - lam2) < 1e-12 * lam2 and lam == tr.calls[2]
    # the accepted step satisfies the sufficient-decrease test f <= f0 + 1e-4 lam f'(0)
    assert 0.5 * g <= 1.0 - 2e-4 * lam


def test_line_search_gives_up_below_the_minimum_step():
    # f rises in every direction (a positive slope would never be produced by Newton);
    # the step shrinks by at least 10x per backtrack until it falls below 1e-12
    lam, g, ok = line_search_bt(2.0, lambda lam: 2.0 * (1.0 + lam), minlambda=1e-12)
    assert not ok and lam < 1e-12


def test_newton_step_that_backtracks():
    """A real step of the method with backtracking: tau = 0.3 ms (below the 0.37 ms bound
    of the coercivity remark), V near the threshold v_th = 13 mV with 5 mV noise."""
    w = synth.workload("cube8")
    prob = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, 0.3, synth.stimulus(w))
    ui, ue, wv = synth.initial_state(prob.N, 0, sigma_mv=5.0)
    ui = ui + 13.0
    seen = []

    def spy(fn2, trial, **kw):
        out = line_search_bt(fn2, trial, **kw)
        seen.append((fn2, out))
        return out

    orig = bidomain.line_search_bt
    bidomain.line_search_bt = spy
    try:
        ui1, ue1, w1, st = bidomain.time_step(prob, ui, ue, wv, 0,
                                              lambda kc, a, b: direct_solve(prob, kc, a, b),
                                              rtol=1e-10, atol=1e-16)
    finally:
        bidomain.line_search_bt = orig
    back = [(fn2, lam, g) for fn2, (lam, g, ok) in seen if lam < 1.0]
    assert back, "the full Newton step was always accepted"
    for fn2, lam, g in back:
        assert 1e-6 <= lam <= 0.5 and g <= fn2 * (1.0 - 2e-4 * lam)
    assert st["reason"] in ("fnorm", "snorm")
    r_i, r_e = prob.residual(ui1, ue1, w1, ui, ue, prob.tau)  # the gauge shift leaves F - G unchanged
    assert np.sqrt(r_i @ r_i + r_e @ r_e) <= 1e-8 * st["res0"]


def test_adam_two_steps_hand_computed():
    # p0 = (0.5, -1, 2), g1 = (1, -2, 0.001), g2 = (-2, 1, 0.001), lr 0.1: the values were
    # worked out in 40-digit decimal arithmetic from m_t = 0.9 m + 0.1 g, v_t = 0.999 v +
    # 0.001 g^2, p -= lr (m_t / (1 - 0.9^t)) / (sqrt(v_t / (1 - 0.999^t)) + 1e-8)
    p = {"w": np.array([0.5, -1.0, 2.0])}
    st = {}
    mlp.adam_step(p, {"w": np.array([1.0, -2.0, 0.001])}, st, lr=0.1)
    np.testing.assert_allclose(p["w"], [0.40000000099999999, -0.90000000050000000, 1.9000009999900001],
                               rtol=0, atol=1e-15)
    mlp.adam_step(p, {"w": np.array([-2.0, 1.0, 0.001])}, st, lr=0.1)
    np.testing.assert_allclose(p["w"], [0.43661035347207509, -0.87336629670243136, 1.8000019999800002],
                               rtol=0, atol=1e-14)


def test_adam_constant_gradient_steps_are_equal():
    # bias correction makes m_hat = g and v_hat = g^2 at every t for a constant g, so each
    # step moves by exactly lr g / (|g| + eps)
    g = np.array([0.3, -7.0, 2e-4])
    p = {"w": np.zeros(3)}
    st = {}
    for t in range(1, 8):
        mlp.adam_step(p, {"w": g}, st, lr=0.01)
        np.testing.assert_allclose(p["w"], -t * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def _slab_optimality():
    rows = {}
    with open(os.path.join(GOLDEN, "slab_optimality.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            hh, prim, its, cond = line.split()
            rows[(int(hh), prim)] = (int(its), float(cond))
    return rows


def test_stored_slab_optimality_is_the_oracles():
    """The stored sweep is the oracle's: H/h = 4 recomputed here."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_slab_optimality",
                                                  os.path.join(GOLDEN, "make_slab_optimality.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    rows = _slab_optimality()
    its, cond = mod.first_newton_solve(4, "VE")
    assert its == rows[(4, "VE")][0]
    assert abs(cond - rows[(4, "VE")][1]) < 1e-5 * cond


def test_condition_number_grows_polylogarithmically():
    """Section 5: cond(M^-1 S) <= C (1 + log H/h)^2 with vertex + edge constraints; with
    vertices alone the bound is lost and the growth is close to linear in H/h
    (Section 6, Test 3 remarks)."""
    rows = _slab_optimality()
    hs = sorted({h for h, _ in rows})
    assert hs == [4, 8, 12]
    ve = np.array([rows[(h, "VE")][1] for h in hs])
    v = np.array([rows[(h, "V")][1] for h in hs])
    L = (1.0 + np.log(np.array(hs, float))) ** 2
    # growth between any two sizes within the ratio of the bound's (1 + log)^2
    for i in range(3):
        for j in range(i + 1, 3):
            assert ve[j] / ve[i] <= L[j] / L[i]
    # a least-squares fit cond = a + b (1 + log H/h)^2 has b > 0 and a small residual
    A = np.stack([np.ones(3), L], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, ve, rcond=None)
    assert b > 0 and np.max(np.abs(A @ [a, b] - ve)) < 0.05 * ve.max()
    # iteration counts stay nearly flat (the paper's Table 7: 10 -> 17 over H/h 4 -> 24)
    its = [rows[(h, "VE")][0] for h in hs]
    assert its[-1] - its[0] <= 6
    # vertex only: faster than the (1 + log)^2 bound, at least half of linear growth
    assert v[1] / v[0] > L[1] / L[0] and v[2] / v[0] > 0.5 * 12 / 4
    assert np.all(v > 5 * ve)
