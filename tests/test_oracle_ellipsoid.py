"""Pins for the oracle's truncated-ellipsoid geometry (Section 6) and its
isoparametric Q1 elements, checked against facts fixed outside the oracle."""
import math

import numpy as np
import pytest

import synth
from conftest import oracle_problem
from oracle import ionic
from oracle.bidomain import direct_solve
from oracle.dd import DDSolver
from oracle.fem import conductivity, fibre_frame_ellipsoid, q1_element_iso, q1_stiffness_gauss
from oracle.mesh import Mesh, ellipsoid_map

AXES = synth.ELLIPSOID["axes"]


def _box_corners(h):
    return np.array([[(a & 1) * h[0], ((a >> 1) & 1) * h[1], ((a >> 2) & 1) * h[2]] for a in range(8)])


def _spd(rng, sig=(3e-3, 3.1525e-4, 3.1525e-5)):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q @ np.diag(sig) @ Q.T


def _distorted_hex(rng):
    return _box_corners((0.05, 0.04, 0.07)) + 0.008 * rng.standard_normal((8, 3))


def test_iso_element_reduces_to_box():
    """On a box the isoparametric element is the box element, with masses vol/8."""
    rng = np.random.default_rng(0)
    h = (0.05, 0.04, 0.07)
    D = _spd(rng)
    K, m = q1_element_iso(_box_corners(h), D)
    np.testing.assert_allclose(K, q1_stiffness_gauss(h, D), rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(m, np.full(8, h[0] * h[1] * h[2] / 8.0), rtol=1e-13)


def test_iso_element_rigid_motion_and_scaling():
    """K(R X + t, R D R^T) = K(X, D); K(s X, D) = s K(X, D) and masses scale by s^3."""
    rng = np.random.default_rng(1)
    X = _distorted_hex(rng)
    D = _spd(rng)
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(R) < 0:
        R[:, 0] = -R[:, 0]
    K, m = q1_element_iso(X, D)
    K2, m2 = q1_element_iso(X @ R.T + np.array([0.3, -1.0, 2.0]), R @ D @ R.T)
    np.testing.assert_allclose(K2, K, rtol=1e-10, atol=1e-16)
    np.testing.assert_allclose(m2, m, rtol=1e-12)
    K3, m3 = q1_element_iso(2.5 * X, D)
    np.testing.assert_allclose(K3, 2.5 * K, rtol=1e-10, atol=1e-16)
    np.testing.assert_allclose(m3, 2.5 ** 3 * m, rtol=1e-12)


def test_iso_element_linear_fields():
    """Trilinear hexahedra reproduce linear fields and 2x2x2 Gauss integrates their
    energy exactly: u_a = c . X_a gives u^T K u = c^T D c vol; constants are in the kernel."""
    rng = np.random.default_rng(2)
    X = _distorted_hex(rng)
    D = _spd(rng)
    K, m = q1_element_iso(X, D)
    c = rng.standard_normal(3)
    u = X @ c
    assert math.isclose(u @ K @ u, c @ D @ c * m.sum(), rel_tol=1e-11)
    np.testing.assert_allclose(K @ np.ones(8), 0.0, atol=1e-15 * np.abs(K).max())
    np.testing.assert_allclose(K, K.T, atol=1e-18)
    assert np.linalg.eigvalsh(K)[1] > 0  # one zero mode only


def test_nodes_lie_on_the_ellipsoids():
    """Every node with depth r satisfies x^2/a(r)^2 + y^2/b(r)^2 + z^2/c(r)^2 = 1."""
    m = Mesh((6, 5, 4), ellipsoid=synth.ELLIPSOID)
    a1, a2, b1, b2, c1, c2 = AXES
    phi, th, r = m.pcoords.T
    x, y, z = m.coords.T
    q = (x / (a1 + r * (a2 - a1))) ** 2 + (y / (b1 + r * (b2 - b1))) ** 2 + (z / (c1 + r * (c2 - c1))) ** 2
    np.testing.assert_allclose(q, 1.0, rtol=1e-13)
    assert np.isclose(phi.min(), -np.pi / 2) and np.isclose(phi.max(), 0.0)
    assert np.isclose(th.min(), -3 * np.pi / 8) and np.isclose(th.max(), np.pi / 8)
    assert r.min() == 0.0 and r.max() == 1.0


def _shell_volume():
    """Exact volume of the truncated shell: the Jacobian determinant of the map,
    derived by hand, det = cos(t) (a' b c cos^2 t cos^2 p + a b' c cos^2 t sin^2 p
    + a b c' sin^2 t), integrated with 24-point Gauss-Legendre per direction."""
    a1, a2, b1, b2, c1, c2 = AXES
    (p0, p1), (t0, t1) = synth.ELLIPSOID["phi"], synth.ELLIPSOID["theta"]
    g, w = np.polynomial.legendre.leggauss(24)
    P = 0.5 * (p1 - p0) * (g + 1) + p0
    T = 0.5 * (t1 - t0) * (g + 1) + t0
    Rr = 0.5 * (g + 1)
    W = np.einsum("i,j,k->ijk", w, w, w) * 0.125 * (p1 - p0) * (t1 - t0)
    p, t, r = np.meshgrid(P, T, Rr, indexing="ij")
    a, b, c = a1 + r * (a2 - a1), b1 + r * (b2 - b1), c1 + r * (c2 - c1)
    ct, st = np.cos(t), np.sin(t)
    det = ct * ((a2 - a1) * b * c * ct ** 2 * np.cos(p) ** 2 + a * (b2 - b1) * c * ct ** 2 * np.sin(p) ** 2
                + a * b * (c2 - c1) * st ** 2)
    return float((W * det).sum())


def _mesh_volume(n):
    m = Mesh(n, ellipsoid=synth.ELLIPSOID)
    return sum(q1_element_iso(m.coords[m.conn[e]], np.eye(3))[1].sum() for e in range(m.n_elem))


def test_mesh_volume_converges_to_the_shell():
    """The Q1 mesh (straight-edged in physical space) approximates the curved shell
    to O(h^2) in the angles: halving h divides the volume error by about 4."""
    exact = _shell_volume()
    e1 = abs(_mesh_volume((4, 4, 2)) - exact) / exact
    e2 = abs(_mesh_volume((8, 8, 2)) - exact) / exact
    e3 = abs(_mesh_volume((16, 16, 2)) - exact) / exact
    assert 3.5 < e1 / e2 < 4.5 and 3.5 < e2 / e3 < 4.5
    assert e3 < 5e-3


def test_patch_test_on_the_ellipsoid():
    """With one constant tensor everywhere, a linear field u = c . x is discretely
    harmonic: (A u)_x = 0 at every node off the boundary."""
    rng = np.random.default_rng(4)
    m = Mesh((5, 4, 4), ellipsoid=synth.ELLIPSOID)
    D = _spd(rng)
    c = rng.standard_normal(3)
    u = m.coords @ c
    Au = np.zeros(m.n_node)
    scale = 0.0
    for e in range(m.n_elem):
        K, _ = q1_element_iso(m.coords[m.conn[e]], D)
        Au[m.conn[e]] += K @ u[m.conn[e]]
        scale = max(scale, np.abs(K).max() * np.abs(u).max())
    ijk = m.node_ijk
    inner = np.all((ijk > 0) & (ijk < np.array(m.n)), axis=1)
    assert inner.sum() == 4 * 3 * 3
    assert np.abs(Au[inner]).max() < 1e-13 * scale
    assert np.abs(Au[~inner]).max() > 1e-6 * scale  # boundary rows carry the flux


@pytest.mark.parametrize("pc", [(-0.3, -0.2, 0.0), (-1.2, 0.3, 0.5), (-0.1, -1.0, 1.0)])
def test_fibre_frame_on_the_ellipsoid(pc):
    """Orthonormal frame; a_n along the gradient of the implicit ellipsoid equation
    (outward); the fibre angle from the phi tangent is 60 degrees at r = 0 and
    -60 degrees at r = 1 (120 degrees through the wall, Section 6)."""
    a_l, a_t, a_n = fibre_frame_ellipsoid(pc, AXES)
    F = np.stack([a_l, a_t, a_n])
    np.testing.assert_allclose(F @ F.T, np.eye(3), atol=1e-14)
    assert np.linalg.det(F) > 0
    a1, a2, b1, b2, c1, c2 = AXES
    r = pc[2]
    X = ellipsoid_map(np.array(pc), AXES)
    grad = X / np.array([a1 + r * (a2 - a1), b1 + r * (b2 - b1), c1 + r * (c2 - c1)]) ** 2
    grad /= np.linalg.norm(grad)
    np.testing.assert_allclose(a_n, grad, atol=1e-13)
    t_phi = np.array([-math.sin(pc[0]), math.cos(pc[0]), 0.0])  # d/dphi direction when a = b
    alpha = math.degrees(math.atan2(a_l @ np.cross(a_n, t_phi), a_l @ t_phi))
    assert math.isclose(alpha, -60.0 + 120.0 * (1.0 - r), abs_tol=1e-9)
    D = conductivity((3.0, 2.0, 1.0), (a_l, a_t, a_n))
    np.testing.assert_allclose(np.linalg.eigvalsh(D), [1.0, 2.0, 3.0])


def test_ellipsoid_problem_mass_stimulus_and_matrices():
    prob = oracle_problem("ell8")
    m = prob.mesh
    # lumped mass: every element's masses sum to its Gauss volume, all positive
    assert np.all(prob.fem.Me > 0)
    assert np.isclose(prob.fem.M.sum(), prob.fem.Me.sum())
    assert abs(prob.fem.M.sum() - _shell_volume()) / _shell_volume() < 0.02
    # the stimulus covers the endocardial surface r = 0: one 9 x 9 node layer
    assert prob.stim_mask.sum() == 81 and np.all(m.node_ijk[prob.stim_mask, 2] == 0)
    for A in (prob.fem.A_i, prob.fem.A_e):
        assert abs(A - A.T).max() < 1e-15 * abs(A).max()
        np.testing.assert_allclose(np.asarray(A.sum(axis=1)).ravel(), 0.0, atol=1e-14 * abs(A).max())
    # the subassembled local masses add up to the global one
    tot = np.zeros(prob.N)
    for j in range(prob.part.n_sub):
        nodes = prob.part.sub_nodes[j]
        _, _, Ml = prob.fem.local(prob.part.sub_elems[j], nodes)
        tot[nodes] += Ml
    np.testing.assert_allclose(tot, prob.fem.M, rtol=1e-13)


def _jacobian_system(prob, seed=0):
    ui, ue, w = synth.initial_state(prob.N, seed)
    ui = ui + 30.0 * (prob.mesh.node_ijk[:, 2] == 0)
    w1 = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    r_i, r_e = prob.residual(ui, ue, w1, ui - 1.0, ue, prob.tau)
    return prob.kc(ui, ue, w1), -r_i, -r_e


@pytest.mark.parametrize("name,scaling", [("ell8", "deluxe"), ("ell10", "deluxe"), ("ell8", "rho")])
@pytest.mark.parametrize("method", ["bddc", "fetidp"])
def test_dd_on_the_ellipsoid_matches_direct(name, scaling, method):
    prob = oracle_problem(name)
    kc, f_i, f_e = _jacobian_system(prob)
    si, se, _ = direct_solve(prob, kc, f_i, f_e)
    dd = DDSolver(prob, method=method, rtol=1e-13, atol=0.0, scaling=scaling)
    ai, ae, info = dd.solve(kc / prob.fem.M, f_i, f_e)
    assert info["reason"] == "converged"
    err = np.linalg.norm(np.r_[ai - si, ae - se]) / np.linalg.norm(np.r_[si, se])
    assert err < 1e-10
