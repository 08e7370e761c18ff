"""Oracle: fibre field, conductivity tensors, Q1 stiffness and lumped mass.

Section 2: D_{i,e}(x) = sum over l, t, n of sigma_* a_* a_*^T (the printed
formula drops the second a_*; the outer product is the standard reading).
Section 6: fibres rotate linearly with depth by 120 degrees, counter-clockwise
from epicardium to endocardium.  Slab reading: endocardium at z = 0,
epicardium at z = L_z, fibre angle alpha(z) = -60 + 120 (1 - z / L_z) degrees
in the x-y plane, a_n = e_z.  D is evaluated at the element centroid.

Section 3a: A_{nm} = integral of grad(phi_n)^T D grad(phi_m) over Q1 elements
(2x2x2 Gauss, exact for box elements with element-constant D); the mass is
lumped by row sums, so every node of an element receives vol/8.

Truncated ellipsoid (Section 6): the same 120 degree rotation with the depth r,
alpha(r) = -60 + 120 (1 - r) degrees, measured in the tangent plane of the
surface r = const from the unit tangent along phi towards n x t_phi, with a_n
the outward unit normal of that surface; D is evaluated at the element's
parametric centroid.  The elements are isoparametric Q1 hexahedra: stiffness
and lumped mass (row sums of the consistent mass, i.e. the integral of phi_a)
by 2x2x2 Gauss on the reference cube through the trilinear map.

Pinned by: the tensor-product closed form of the box-element stiffness (tests),
zero row sums, symmetry, and total lumped mass = volume; for the ellipsoid by
the isoparametric element reducing to the box element on a box, invariance
under a rigid rotation, the linear-field energy identity and patch test, the
total mass converging at O(h^2) to the volume of the exact shell, and the
fibre normal against the gradient of the implicit ellipsoid equation.
"""
from __future__ import annotations

import math

import numpy as np


def fibre_frame_slab(z, lz):
    """Orthonormal (a_l, a_t, a_n) at depth z of a slab of thickness lz."""
    alpha = math.radians(-60.0 + 120.0 * (1.0 - z / lz))
    a_l = np.array([math.cos(alpha), math.sin(alpha), 0.0])
    a_t = np.array([-math.sin(alpha), math.cos(alpha), 0.0])
    a_n = np.array([0.0, 0.0, 1.0])
    return a_l, a_t, a_n


def fibre_frame_ellipsoid(pc, axes):
    """Orthonormal (a_l, a_t, a_n) at parametric point pc = (phi, theta, r)."""
    a1, a2, b1, b2, c1, c2 = axes
    phi, th, r = (float(v) for v in pc)
    a, b, c = a1 + r * (a2 - a1), b1 + r * (b2 - b1), c1 + r * (c2 - c1)
    cp, sp_, ct, st = math.cos(phi), math.sin(phi), math.cos(th), math.sin(th)
    x_phi = np.array([-a * ct * sp_, b * ct * cp, 0.0])
    x_th = np.array([-a * st * cp, -b * st * sp_, c * ct])
    x_r = np.array([(a2 - a1) * ct * cp, (b2 - b1) * ct * sp_, (c2 - c1) * st])
    n = np.cross(x_phi, x_th)
    if n @ x_r < 0:
        n = -n
    a_n = n / np.linalg.norm(n)
    t1 = x_phi / np.linalg.norm(x_phi)
    t2 = np.cross(a_n, t1)
    alpha = math.radians(-60.0 + 120.0 * (1.0 - r))
    a_l = math.cos(alpha) * t1 + math.sin(alpha) * t2
    a_t = np.cross(a_n, a_l)
    return a_l, a_t, a_n


def conductivity(sig, frame):
    """D = sum_k sig_k a_k a_k^T."""
    return sum(s * np.outer(a, a) for s, a in zip(sig, frame))


def q1_stiffness_gauss(h, D):
    """8x8 Q1 element matrix of the form grad(phi)^T D grad(phi), 2x2x2 Gauss.

    Local node a = ax + 2 ay + 4 az sits at (ax hx, ay hy, az hz).
    """
    hx, hy, hz = h
    gp = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))
    wq = hx * hy * hz / 8.0
    K = np.zeros((8, 8))
    for xi in gp:
        for eta in gp:
            for zeta in gp:
                G = np.zeros((8, 3))
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    lx = xi if ax else 1.0 - xi
                    ly = eta if ay else 1.0 - eta
                    lz = zeta if az else 1.0 - zeta
                    dx = (1.0 if ax else -1.0) / hx
                    dy = (1.0 if ay else -1.0) / hy
                    dz = (1.0 if az else -1.0) / hz
                    G[a] = (dx * ly * lz, lx * dy * lz, lx * ly * dz)
                K += wq * G @ D @ G.T
    return K


def q1_element_iso(X, D):
    """Isoparametric Q1 element on the hexahedron with corners X (8x3).

    Returns the 8x8 stiffness (grad phi_a)^T D grad phi_b and the 8 lumped
    masses int phi_a, by 2x2x2 Gauss on [0,1]^3 with the map x = sum_a X_a phi_a;
    physical gradients are J^-T times the reference gradients.
    """
    gp = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))
    K = np.zeros((8, 8))
    m = np.zeros(8)
    for xi in gp:
        for eta in gp:
            for zeta in gp:
                N = np.zeros(8)
                dN = np.zeros((8, 3))
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    lx = xi if ax else 1.0 - xi
                    ly = eta if ay else 1.0 - eta
                    lz = zeta if az else 1.0 - zeta
                    sx, sy, sz = (1.0 if ax else -1.0), (1.0 if ay else -1.0), (1.0 if az else -1.0)
                    N[a] = lx * ly * lz
                    dN[a] = (sx * ly * lz, lx * sy * lz, lx * ly * sz)
                J = X.T @ dN  # J[p, q] = d x_p / d xi_q
                det = np.linalg.det(J)
                G = dN @ np.linalg.inv(J)
                K += (det / 8.0) * G @ D @ G.T
                m += (det / 8.0) * N
    return K, m


class FEM:
    """Global and per-subdomain (subassembled) Q1 matrices for one partition."""

    def __init__(self, mesh, sigma_i, sigma_e):
        self.sigma_i, self.sigma_e = tuple(sigma_i), tuple(sigma_e)  # (l, t, n) per medium
        import scipy.sparse as sp
        self.mesh = mesh
        m = mesh
        vol = m.h[0] * m.h[1] * m.h[2]
        lz = m.l[2]
        self.Ke_i = np.empty((m.n_elem, 8, 8))
        self.Ke_e = np.empty((m.n_elem, 8, 8))
        self.Me = np.full((m.n_elem, 8), vol / 8.0)  # lumped element masses
        for e in range(m.n_elem):
            if m.ellipsoid is None:
                zc = (m.elem_ijk[e, 2] + 0.5) * m.h[2]
                fr = fibre_frame_slab(zc, lz)
                self.Ke_i[e] = q1_stiffness_gauss(m.h, conductivity(sigma_i, fr))
                self.Ke_e[e] = q1_stiffness_gauss(m.h, conductivity(sigma_e, fr))
            else:
                pc = np.array(m.origin) + (m.elem_ijk[e] + 0.5) * np.array(m.h)
                fr = fibre_frame_ellipsoid(pc, m.ellipsoid["axes"])
                X = m.coords[m.conn[e]]
                self.Ke_i[e], self.Me[e] = q1_element_iso(X, conductivity(sigma_i, fr))
                self.Ke_e[e], _ = q1_element_iso(X, conductivity(sigma_e, fr))
        rows = np.repeat(m.conn, 8, axis=1).ravel()
        cols = np.tile(m.conn, (1, 8)).ravel()
        n = m.n_node
        self.A_i = sp.csr_matrix((self.Ke_i.ravel(), (rows, cols)), shape=(n, n))
        self.A_e = sp.csr_matrix((self.Ke_e.ravel(), (rows, cols)), shape=(n, n))
        self.M = np.zeros(n)
        np.add.at(self.M, m.conn.ravel(), self.Me.ravel())

    def local(self, elems, nodes):
        """Subassembled dense A_i^(j), A_e^(j), M^(j) over ``elems`` on ``nodes``."""
        m = self.mesh
        pos = {int(x): k for k, x in enumerate(nodes)}
        n = len(nodes)
        Ai = np.zeros((n, n))
        Ae = np.zeros((n, n))
        Ml = np.zeros(n)
        for e in elems:
            loc = [pos[int(x)] for x in m.conn[e]]
            Ai[np.ix_(loc, loc)] += self.Ke_i[e]
            Ae[np.ix_(loc, loc)] += self.Ke_e[e]
            Ml[loc] += self.Me[e]
        return Ai, Ae, Ml
