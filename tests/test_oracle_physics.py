"""Pins for the oracle's ionic model, residual, Jacobian and Newton (Sections 2-3)."""
import numpy as np
import pytest

import synth
from conftest import oracle_problem
from oracle import ionic
from oracle.bidomain import direct_solve, newton, time_step

P = synth.IONIC


def test_gating_solves_backward_euler():
    rng = np.random.default_rng(1)
    v, w = rng.uniform(-10, 110, 50), rng.uniform(0, 1, 50)
    tau = 0.05
    w1 = ionic.gating_step(v, w, tau, P)
    # defining equation of Step 1: w1 - tau R(v, w1) = w
    R = P["eta2"] * (v / P["vp"] - w1)
    np.testing.assert_allclose(w1 - tau * R, w, rtol=1e-14, atol=1e-15)


def test_di_ion_finite_difference():
    v = np.linspace(-20, 120, 57)
    w = np.linspace(0, 1, 57)
    eps = 1e-5
    fd = (ionic.i_ion(v + eps, w, P) - ionic.i_ion(v - eps, w, P)) / (2 * eps)
    np.testing.assert_allclose(ionic.di_ion_dv(v, w, P), fd, rtol=1e-7, atol=1e-8)


def test_coercivity_remark_tau_037():
    """Remark after the coercivity lemma: chi Cm + tau dI/dv >= 0 for tau <= 0.37 ms.

    The minimum of dI/dv (w = 0) is G (1 - (a+b)^2 / (3ab)) at v = (a+b)/(3ab),
    a = 1/v_th, b = 1/v_p: -2.73 at v = 37.67 mV, so tau_max = 1/2.73 = 0.366.
    """
    v = np.linspace(-50, 150, 200001)
    d = ionic.di_ion_dv(v, 0.0, P)
    k = np.argmin(d)
    assert abs(v[k] - 37.67) < 0.01
    assert abs(d[k] + 2.73) < 0.005
    assert np.all(P["chi_cm"] + 0.36 * d > 0)
    assert np.any(P["chi_cm"] + 0.37 * d < 0)


def _state(prob, seed=0):
    ui, ue, w = synth.initial_state(prob.N, seed)
    ue = 0.3 * synth.random_vector(prob.N, seed + 7)
    ui = ui + ue + 20.0 * np.exp(-np.sum(prob.mesh.coords ** 2, axis=1) / 0.02)
    w = np.abs(synth.random_vector(prob.N, seed + 9)) * 0.01
    return ui, ue, w


@pytest.mark.parametrize("name", ["ragged", "ell10"])
def test_residual_compatibility_and_rest(name):
    prob = oracle_problem(name)
    ui, ue, w = _state(prob)
    r_i, r_e = prob.residual(ui, ue, w, ui * 0.9, ue * 1.1, 0.5)
    assert abs(r_i.sum() + r_e.sum()) < 1e-13 * np.abs(np.r_[r_i, r_e]).sum()
    # rest state, no stimulus: nothing moves
    z = np.zeros(prob.N)
    r_i, r_e = prob.residual(z, z, z, z, z, 5.0)
    assert np.all(r_i == 0) and np.all(r_e == 0)


def _tiny_ellipsoid():
    from oracle.bidomain import Problem
    w = dict(n=(2, 2, 2), ellipsoid=synth.ELLIPSOID, s=(1, 1, 1), primal="V", name="tiny_ell")
    return Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, synth.stimulus(w))


@pytest.mark.parametrize("geometry", ["box", "ellipsoid"])
def test_jacobian_fd_symmetry_nullspace(geometry):
    prob = oracle_problem("tiny") if geometry == "box" else _tiny_ellipsoid()
    ui, ue, w = _state(prob, 3)
    kc = prob.kc(ui, ue, w)
    J = prob.jacobian(kc).toarray()
    N = prob.N
    eps = 1e-4
    Jfd = np.zeros_like(J)
    for k in range(2 * N):
        d = np.zeros(2 * N)
        d[k] = eps
        rp = np.concatenate(prob.residual(ui + d[:N], ue + d[N:], w, ui, ue, 0.5))
        rm = np.concatenate(prob.residual(ui - d[:N], ue - d[N:], w, ui, ue, 0.5))
        Jfd[:, k] = (rp - rm) / (2 * eps)
    np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-9 * np.abs(J).max())
    scale = np.abs(J).max()
    np.testing.assert_allclose(J, J.T, atol=1e-15 * scale)
    np.testing.assert_allclose(J @ np.ones(2 * N), 0.0, atol=1e-13 * scale)
    keep = np.ones(2 * N, bool)
    keep[N + prob.part.gauge_node] = False
    assert np.linalg.eigvalsh(J[np.ix_(keep, keep)]).min() > 0


def test_newton_direct_quadratic():
    prob = oracle_problem("cube8")
    ui, ue, w = _state(prob)
    w1 = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    _, _, st = newton(prob, ui, ue, w1, prob.tau,
                      lambda kc, a, b: direct_solve(prob, kc, a, b), rtol=1e-13, atol=1e-18)
    assert st["reason"] in ("fnorm", "snorm")
    assert st["newton_its"] <= 4


def test_time_step_gauge_and_rest():
    prob = oracle_problem("tiny")
    z = np.zeros(prob.N)
    prob.stim = dict(prob.stim, amp=0.0)
    ui, ue, w, st = time_step(prob, z, z, z, 30, lambda kc, a, b: direct_solve(prob, kc, a, b))
    assert np.all(ui == 0) and np.all(ue == 0) and st["newton_its"] == 0
    prob.stim = dict(synth.STIMULUS)
    ui0, ue0, w0 = _state(prob)
    ui, ue, w, st = time_step(prob, ui0, ue0, w0, 0,
                              lambda kc, a, b: direct_solve(prob, kc, a, b))
    assert abs(prob.fem.M @ ue) < 1e-15
    # stimulus on: the corner cube depolarises
    assert (ui - ue)[0] > (ui0 - ue0)[0]
