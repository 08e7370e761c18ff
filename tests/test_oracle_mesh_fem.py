"""Pins for the oracle's index sets (Section 4.1) and Q1 matrices (Section 3a)."""
import itertools

import numpy as np
import pytest

from conftest import oracle_problem
from oracle.fem import conductivity, fibre_frame_slab, q1_stiffness_gauss
from oracle.mesh import EDGE, FACE, VERTEX, Mesh, Partition


def _counts(part):
    return [int((part.cls_type == t).sum()) for t in (VERTEX, EDGE, FACE)]


def test_cube8_hand_counts():
    # 2x2x2 subdomains of 4^3 elements: one centre vertex, six half-lines of
    # 4-subdomain edges (3 interior nodes each + 1 boundary node), twelve faces
    # of 4x4 nodes -> 1 + 6*4 + 12*16 = 217 interface nodes.
    part = oracle_problem("cube8").part
    assert _counts(part) == [1, 6, 12]
    assert len(part.iface_nodes) == 217
    assert [len(part.cls_nodes[c]) for c in range(part.n_cls) if part.cls_type[c] == EDGE] == [4] * 6
    assert [len(part.cls_nodes[c]) for c in range(part.n_cls) if part.cls_type[c] == FACE] == [16] * 12
    for j in range(8):
        assert len(part.interior_nodes(j)) == 64
    assert part.gauge_node == 4 + 9 * (4 + 9 * 4)


@pytest.mark.parametrize("name,counts,nprimal", [
    ("slab32", [9, 42, 64], 102),
    ("opt4", [27, 108, 144], 270),
])
def test_class_counts(name, counts, nprimal):
    import synth
    w = synth.workload(name)
    part = Partition(Mesh(w["n"], w["l"]), w["s"], w["primal"])
    assert _counts(part) == counts
    assert part.n_primal == nprimal


def test_nx_brute_force():
    """N_x from the definition (closure of each box block) on a ragged grid."""
    import synth
    w = synth.workload("ragged")
    m = Mesh(w["n"], w["l"])
    part = Partition(m, w["s"], w["primal"])
    s = w["s"]
    nb = [-(-w["n"][d] // s[d]) for d in range(3)]
    for x in range(m.n_node):
        i = m.node_ijk[x]
        owners = []
        for b in itertools.product(*[range(k) for k in nb]):
            if all(b[d] * s[d] <= i[d] <= min((b[d] + 1) * s[d], w["n"][d]) for d in range(3)):
                owners.append(b[0] + nb[0] * (b[1] + nb[1] * b[2]))
        assert tuple(sorted(owners)) == part.N[x]


def test_classes_partition_interface():
    part = oracle_problem("ragged").part
    allnodes = np.sort(np.concatenate(part.cls_nodes))
    assert np.array_equal(allnodes, part.iface_nodes)
    for c in range(part.n_cls):
        nodes = part.cls_nodes[c]
        assert all(part.N[x] == part.cls_subs[c] for x in nodes)
        if part.cls_type[c] == VERTEX:
            assert len(nodes) == 1 and len(part.cls_subs[c]) >= 3


def test_transform_average_and_deviation():
    """Columns of T: edge averages are all-ones on the edge, deviations sum to 0."""
    prob = oracle_problem("cube8ve")
    d, part = prob.dofs, prob.part
    T = d.T
    for c in range(part.n_cls):
        if part.cls_type[c] != EDGE:
            continue
        rows = 2 * d.gnode_to_iface[part.cls_nodes[c]]
        for f in range(2):
            col = d.n_dual + 2 * part.primal_index[c] + f
            assert np.all(T[rows + f, col] == 1.0)
            for k in range(len(part.cls_nodes[c]) - 1):
                colk = d.cls_dual_start[c] + 2 * k + f
                assert T[rows + f, colk].sum() == 0.0
    assert np.linalg.matrix_rank(T) == T.shape[0] == T.shape[1]


def _tensor_closed_form(h, D):
    """Box-element stiffness from exact 1D integrals (independent of quadrature).

    With phi_a = l_ax(x) l_ay(y) l_az(z), the entry sum_{p,q} D_pq int d_p phi_a d_q phi_b
    factorises into 1D integrals: int l_i l_j = h/6 (2 if i == j else 1),
    int l_i' l_j = s_i / 2, int l_i l_j' = s_j / 2, int l_i' l_j' = s_i s_j / h, s_0 = -1, s_1 = 1.
    """
    def one(i, j, di, dj, hh):
        si, sj = (1.0 if i else -1.0), (1.0 if j else -1.0)
        if not di and not dj:
            return hh / 6.0 * (2.0 if i == j else 1.0)
        if di and not dj:
            return si / 2.0
        if dj and not di:
            return sj / 2.0
        return si * sj / hh

    K = np.zeros((8, 8))
    for a in range(8):
        ia = (a & 1, (a >> 1) & 1, (a >> 2) & 1)
        for b in range(8):
            ib = (b & 1, (b >> 1) & 1, (b >> 2) & 1)
            for p in range(3):
                for q in range(3):
                    v = 1.0
                    for d in range(3):
                        v *= one(ia[d], ib[d], d == p, d == q, h[d])
                    K[a, b] += D[p, q] * v
    return K


def test_q1_stiffness_closed_form():
    rng = np.random.default_rng(3)
    h = (0.05, 0.04, 0.07)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    D = Q @ np.diag([3e-3, 3.1525e-4, 3.1525e-5]) @ Q.T
    K = q1_stiffness_gauss(h, D)
    np.testing.assert_allclose(K, _tensor_closed_form(h, D), rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(K, K.T, atol=1e-18)
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-18)
    # textbook 1D stiffness K1 = (1/h)[[1,-1],[-1,1]] and mass M1 = (h/6)[[2,1],[1,2]]
    Kd = q1_stiffness_gauss(h, np.diag([1.0, 0.0, 0.0]))
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h[0]
    M1y = np.array([[2.0, 1.0], [1.0, 2.0]]) * h[1] / 6.0
    M1z = np.array([[2.0, 1.0], [1.0, 2.0]]) * h[2] / 6.0
    np.testing.assert_allclose(Kd, np.kron(M1z, np.kron(M1y, K1)), rtol=1e-12)


def test_fibres_and_mass():
    a_l, a_t, a_n = fibre_frame_slab(0.0, 1.0)
    assert np.isclose(np.degrees(np.arctan2(a_l[1], a_l[0])), 60.0)
    a_l2, _, _ = fibre_frame_slab(1.0, 1.0)
    assert np.isclose(np.degrees(np.arctan2(a_l2[1], a_l2[0])), -60.0)
    D = conductivity((3.0, 2.0, 1.0), (a_l, a_t, a_n))
    np.testing.assert_allclose(np.linalg.eigvalsh(D), [1.0, 2.0, 3.0])
    prob = oracle_problem("ragged")
    assert np.isclose(prob.fem.M.sum(), 0.5 * 0.45 * 0.35)
    A = prob.fem.A_i
    assert abs(A - A.T).max() < 1e-18
    np.testing.assert_allclose(np.asarray(A.sum(axis=1)).ravel(), 0.0, atol=1e-17)
    assert A.getnnz(axis=1).max() == 27
