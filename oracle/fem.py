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

Pinned by: the tensor-product closed form of the box-element stiffness (tests),
zero row sums, symmetry, and total lumped mass = volume.
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
        for e in range(m.n_elem):
            zc = (m.elem_ijk[e, 2] + 0.5) * m.h[2]
            fr = fibre_frame_slab(zc, lz)
            self.Ke_i[e] = q1_stiffness_gauss(m.h, conductivity(sigma_i, fr))
            self.Ke_e[e] = q1_stiffness_gauss(m.h, conductivity(sigma_e, fr))
        rows = np.repeat(m.conn, 8, axis=1).ravel()
        cols = np.tile(m.conn, (1, 8)).ravel()
        n = m.n_node
        self.A_i = sp.csr_matrix((self.Ke_i.ravel(), (rows, cols)), shape=(n, n))
        self.A_e = sp.csr_matrix((self.Ke_e.ravel(), (rows, cols)), shape=(n, n))
        self.M = np.zeros(n)
        np.add.at(self.M, m.conn.ravel(), vol / 8.0)
        self.vol_e = vol

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
            Ml[loc] += self.vol_e / 8.0
        return Ai, Ae, Ml
