"""Oracle: structured Q1 grid, non-overlapping subdomains and interface classes.

Follows Section 4.1 of the paper: subdomains are unions of elements; the
interface Gamma is the set of nodes in at least two subdomains; N_x is the set
of subdomains whose closure holds node x, and it induces the face / edge /
vertex equivalence classes (Section 4.2, after the rho-scaling formula).

Readings (the paper leaves these open):

* node ids are lexicographic over the used grid nodes, x fastest;
* a class is a maximal set of interface nodes with the same N_x that is
  connected through element edges; |N_x| = 2 -> face; |N_x| >= 3 -> edge when
  the class has more than one node, vertex when it has one node;
* nodes on the outer boundary belong to the class of their N_x (the paper
  counts Neumann-boundary nodes as ordinary, not special);
* classes are ordered by (type, smallest node id) with vertex < edge < face;
* a subdomain fragment with no vertex on its interface (masked grids) promotes the
  lowest-id node of each of its edge classes (of its face classes if it has no
  edge) to a vertex, the rest of the class being split again into classes;
* primal sets: "V" = vertex classes, "VE" = vertices and edges, "VEF" =
  vertices, edges and faces (Section 6, Test 3 and Table 7); an edge or face
  class holds its average as the primal dof and n - 1 deviations as dual dofs.

Pinned by hand counts (a 2x2x2 partition of an 8^3 grid has one vertex, six
edges and twelve faces holding 217 interface nodes) and by a brute-force
recount of N_x in the tests.
"""
from __future__ import annotations

import numpy as np

VERTEX, EDGE, FACE = 0, 1, 2

# the 12 edges of a hexahedron in the local numbering a = ax + 2 ay + 4 az
HEX_EDGES = [(0, 1), (2, 3), (4, 5), (6, 7),
             (0, 2), (1, 3), (4, 6), (5, 7),
             (0, 4), (1, 5), (2, 6), (3, 7)]


def ellipsoid_map(p, axes):
    """Truncated ellipsoid of Section 6: parametric (phi, theta, r) -> (x, y, z) cm.

    x = a(r) cos(theta) cos(phi), y = b(r) cos(theta) sin(phi), z = c(r) sin(theta),
    with a(r) = a1 + r (a2 - a1) and likewise b, c; r = 0 is the endocardium, r = 1
    the epicardium.  The printed z component reads sin(phi); with it the surfaces
    r = const would not be ellipsoids, so sin(theta) (the standard ellipsoidal
    coordinates) is taken.  ``axes`` = (a1, a2, b1, b2, c1, c2).
    """
    a1, a2, b1, b2, c1, c2 = axes
    p = np.asarray(p, float)
    phi, th, r = p[..., 0], p[..., 1], p[..., 2]
    a, b, c = a1 + r * (a2 - a1), b1 + r * (b2 - b1), c1 + r * (c2 - c1)
    return np.stack([a * np.cos(th) * np.cos(phi), b * np.cos(th) * np.sin(phi), c * np.sin(th)], axis=-1)


class Mesh:
    """Structured grid of nx*ny*nz Q1 elements with an optional element mask.

    Box geometry: the grid spans [0, l0] x [0, l1] x [0, l2] cm.  Ellipsoid
    geometry (``ellipsoid`` = dict(axes, phi, theta), Section 6): the grid is
    uniform in the parametric coordinates (phi, theta, r) over
    [phi0, phi1] x [theta0, theta1] x [0, 1] and the nodes are mapped by
    ``ellipsoid_map`` (isoparametric Q1 elements).  ``pcoords`` holds the
    parametric coordinates origin + ijk h (equal to ``coords`` for a box).
    """

    def __init__(self, n, l=None, elem_mask=None, ellipsoid=None):
        self.n = tuple(int(v) for v in n)
        self.ellipsoid = None if ellipsoid is None else dict(ellipsoid)
        if self.ellipsoid is None:
            self.l = tuple(float(v) for v in l)
            self.origin = (0.0, 0.0, 0.0)
        else:
            (p0, p1), (t0, t1) = self.ellipsoid["phi"], self.ellipsoid["theta"]
            self.l = (float(p1) - float(p0), float(t1) - float(t0), 1.0)
            self.origin = (float(p0), float(t0), 0.0)
        nx, ny, nz = self.n
        self.h = (self.l[0] / nx, self.l[1] / ny, self.l[2] / nz)
        ne_full = nx * ny * nz
        keep = np.ones(ne_full, bool) if elem_mask is None else np.asarray(elem_mask, bool).ravel()
        assert keep.size == ne_full
        ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        # element id lexicographic with x fastest
        order = np.argsort((ex + nx * (ey + ny * ez)).ravel(), kind="stable")
        ex, ey, ez = ex.ravel()[order], ey.ravel()[order], ez.ravel()[order]
        gx, gy = nx + 1, ny + 1
        conn_full = np.empty((ne_full, 8), np.int64)
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            conn_full[:, a] = (ex + ax) + gx * ((ey + ay) + gy * (ez + az))
        nfull = gx * gy * (nz + 1)
        used = np.zeros(nfull, bool)
        used[conn_full[keep].ravel()] = True
        node_of_full = -np.ones(nfull, np.int64)
        node_of_full[used] = np.arange(int(used.sum()))
        self.grid_index = np.nonzero(used)[0]           # full-grid index of each node
        self.conn = node_of_full[conn_full[keep]]        # (ne, 8) node ids
        self.elem_ijk = np.stack([ex[keep], ey[keep], ez[keep]], axis=1)
        self.n_elem = self.conn.shape[0]
        self.n_node = int(used.sum())
        gi = self.grid_index
        ijk = np.stack([gi % gx, (gi // gx) % gy, gi // (gx * gy)], axis=1)
        self.node_ijk = ijk
        if self.ellipsoid is None:
            self.pcoords = ijk * np.array(self.h)[None, :]
            self.coords = self.pcoords
        else:
            self.pcoords = np.array(self.origin)[None, :] + ijk * np.array(self.h)[None, :]
            self.coords = ellipsoid_map(self.pcoords, self.ellipsoid["axes"])


class Partition:
    """Subdomains, the sets N_x, interface classes and primal set (Section 4.1).

    ``s`` is the number of elements per subdomain along x, y, z (H/h).  Each
    box block of elements is split into node-connected components; the
    components are the subdomains, ordered by block and then by smallest node.
    """

    def __init__(self, mesh: Mesh, s, primal: str = "V"):
        self.mesh = mesh
        self.s = tuple(int(v) for v in s)
        self.primal_kind = primal
        m = mesh
        bx = -(-m.n[0] // self.s[0])
        by = -(-m.n[1] // self.s[1])
        block = (m.elem_ijk[:, 0] // self.s[0]) + bx * (
            (m.elem_ijk[:, 1] // self.s[1]) + by * (m.elem_ijk[:, 2] // self.s[2]))
        # split blocks into connected components (elements sharing a node)
        elem_sub = -np.ones(m.n_elem, np.int64)
        subs = []
        for b in np.unique(block):
            elems = np.nonzero(block == b)[0]
            comps = _components_of_elements(m.conn, elems)
            comps.sort(key=lambda es: int(m.conn[es].min()))
            subs.extend(comps)
        for j, es in enumerate(subs):
            elem_sub[es] = j
        self.elem_sub = elem_sub
        self.n_sub = len(subs)
        self.sub_elems = [np.sort(np.asarray(es)) for es in subs]
        self.sub_nodes = [np.unique(m.conn[es].ravel()) for es in self.sub_elems]
        # N_x: sorted tuple of subdomains whose closure contains x
        nsets = [set() for _ in range(m.n_node)]
        for j, nodes in enumerate(self.sub_nodes):
            for x in nodes:
                nsets[x].add(j)
        self.N = [tuple(sorted(t)) for t in nsets]
        self.mult = np.array([len(t) for t in self.N], np.int64)
        self.iface_nodes = np.nonzero(self.mult >= 2)[0]
        self._classes()
        self._primal()

    # -- equivalence classes -------------------------------------------------
    def _classes(self):
        m = self.mesh
        is_iface = self.mult >= 2
        adj = [[] for _ in range(m.n_node)]
        for el in m.conn:
            for a, b in HEX_EDGES:
                x, y = int(el[a]), int(el[b])
                if is_iface[x] and is_iface[y] and self.N[x] == self.N[y]:
                    adj[x].append(y)
                    adj[y].append(x)
        seen = np.zeros(m.n_node, bool)
        classes = []
        for x in self.iface_nodes:
            if seen[x]:
                continue
            stack, comp = [int(x)], []
            seen[x] = True
            while stack:
                y = stack.pop()
                comp.append(y)
                for z in adj[y]:
                    if not seen[z]:
                        seen[z] = True
                        stack.append(z)
            comp = sorted(comp)
            classes.append(_make_class(comp, self.N[x]))
        classes.sort(key=lambda c: (c[0], c[1]))
        classes = self._promote_vertices(classes, adj)
        self.cls_type = np.array([c[0] for c in classes], np.int64)
        self.cls_nodes = [c[2] for c in classes]
        self.cls_subs = [c[3] for c in classes]
        self.n_cls = len(classes)
        self.node_cls = -np.ones(m.n_node, np.int64)
        for c, nodes in enumerate(self.cls_nodes):
            self.node_cls[nodes] = c

    def _promote_vertices(self, classes, adj):
        """A subdomain fragment of a masked grid may have no vertex on its interface (reading
        of Section 4.2 for non-box subdomains): for subdomains j = 0, 1, ... in order, one
        without a vertex class promotes the lowest-id node of each of its edge classes (of
        its face classes if it has no edge) to a vertex class of its own; the rest of each
        such class is split again into connected classes by the usual rule; the classes
        are re-sorted by (type, smallest node) after every subdomain."""
        for j in range(self.n_sub):
            mine = [c for c in classes if j in c[3]]
            if any(c[0] == VERTEX for c in mine):
                continue
            cand = [c for c in mine if c[0] == EDGE] or [c for c in mine if c[0] == FACE]
            if not cand:
                continue
            drop = {id(c) for c in cand}
            out = [c for c in classes if id(c) not in drop]
            for c in cand:
                nodes = [int(v) for v in c[2]]
                out.append((VERTEX, nodes[0], np.array(nodes[:1], np.int64), c[3]))
                rest = set(nodes[1:])
                seen = set()
                for x in sorted(rest):
                    if x in seen:
                        continue
                    stack, comp = [x], []
                    seen.add(x)
                    while stack:
                        y = stack.pop()
                        comp.append(y)
                        for z in adj[y]:
                            if z in rest and z not in seen:
                                seen.add(z)
                                stack.append(z)
                    out.append(_make_class(sorted(comp), c[3]))
            classes = sorted(out, key=lambda c: (c[0], c[1]))
        return classes

    def _primal(self):
        kinds = {"V": (VERTEX,), "VE": (VERTEX, EDGE), "VEF": (VERTEX, EDGE, FACE)}[self.primal_kind]
        self.cls_primal = np.array([t in kinds for t in self.cls_type], bool)
        self.primal_cls = np.nonzero(self.cls_primal)[0]
        # global primal dofs: per primal class, field i then field e
        self.primal_index = -np.ones(self.n_cls, np.int64)
        self.primal_index[self.primal_cls] = np.arange(len(self.primal_cls))
        self.n_primal = 2 * len(self.primal_cls)
        verts = np.nonzero(self.cls_type == VERTEX)[0]
        if len(verts) == 0:
            raise ValueError("partition has no vertex class: no gauge vertex")
        # gauge: u_e correction fixed to zero at the lowest-id vertex (first vertex class)
        self.gauge_node = int(self.cls_nodes[verts[0]][0])
        self.gauge_primal = 2 * int(self.primal_index[verts[0]]) + 1
        for j in range(self.n_sub):
            if not any(self.cls_primal[c] for c in self.sub_classes(j)):
                raise ValueError(f"subdomain {j} has no primal constraint")

    def sub_classes(self, j):
        """Classes on Gamma^(j), in class order."""
        return [c for c in range(self.n_cls) if j in self.cls_subs[c]]

    # -- dof bookkeeping -----------------------------------------------------
    def interior_nodes(self, j):
        nodes = self.sub_nodes[j]
        return nodes[self.mult[nodes] == 1]

    def iface_nodes_of(self, j):
        nodes = self.sub_nodes[j]
        return nodes[self.mult[nodes] >= 2]


def _make_class(comp, subs):
    """(type, smallest node, nodes, N_x) of a connected set of interface nodes with the
    same N_x: a face when two subdomains share it, else an edge (several nodes) or a
    vertex (one node)."""
    t = FACE if len(subs) == 2 else (EDGE if len(comp) > 1 else VERTEX)
    return (t, comp[0], np.array(comp, np.int64), subs)


def _components_of_elements(conn, elems):
    """Split a set of elements into groups connected through shared nodes."""
    elems = list(int(e) for e in elems)
    node_to_elems = {}
    for e in elems:
        for x in conn[e]:
            node_to_elems.setdefault(int(x), []).append(e)
    seen = set()
    comps = []
    for e in elems:
        if e in seen:
            continue
        stack, comp = [e], []
        seen.add(e)
        while stack:
            f = stack.pop()
            comp.append(f)
            for x in conn[f]:
                for g in node_to_elems[int(x)]:
                    if g not in seen:
                        seen.add(g)
                        stack.append(g)
        comps.append(comp)
    return comps


class DofMaps:
    """Interface and local dof numbering shared by BDDC and FETI-DP.

    Global interface vector (original nodal basis): interface nodes sorted by
    id, two dofs per node (u_i then u_e).

    Transformed basis (change of basis for edge averages, standard for a
    primal space that contains averages): for every primal edge E with nodes
    e_0 < ... < e_{n-1} and each field, the n nodal dofs are replaced by the
    average a and the deviations d_k (k < n-1), with
    u(e_k) = a + d_k (k < n-1) and u(e_{n-1}) = a - sum_k d_k.
    Every other interface dof keeps its nodal meaning.

    Global transformed dual dofs: dual classes in class order; inside a class,
    its nodes by id (without the last node for a primal edge), fields i, e.
    Global primal dofs: primal classes in class order, fields i, e.
    Local dofs of subdomain j: interior nodes by id (fields i, e), then the
    dual dofs of its classes in global order, then its primal dofs.
    """

    def __init__(self, part: Partition):
        self.part = part
        p = part
        self.gnode_to_iface = -np.ones(p.mesh.n_node, np.int64)
        self.gnode_to_iface[p.iface_nodes] = np.arange(len(p.iface_nodes))
        self.n_iface = 2 * len(p.iface_nodes)
        # global transformed dual dofs, grouped per class
        self.cls_dual_nodes = []
        start = 0
        self.cls_dual_start = -np.ones(p.n_cls, np.int64)
        for c in range(p.n_cls):
            nodes = p.cls_nodes[c]
            if p.cls_primal[c]:
                dn = nodes[:0] if p.cls_type[c] == VERTEX else nodes[:-1]  # averaged class: n - 1 deviations
            else:
                dn = nodes
            self.cls_dual_nodes.append(dn)
            self.cls_dual_start[c] = start
            start += 2 * len(dn)
        self.n_dual = start
        # T_glob: (n_iface x (n_dual + n_primal)) maps transformed -> nodal
        self.T = self._build_T()

    def _build_T(self):
        p = self.part
        T = np.zeros((self.n_iface, self.n_dual + p.n_primal))
        for c in range(p.n_cls):
            nodes = p.cls_nodes[c]
            for f in range(2):
                if p.cls_primal[c]:
                    col_a = self.n_dual + 2 * p.primal_index[c] + f
                    for x in nodes:
                        T[2 * self.gnode_to_iface[x] + f, col_a] = 1.0
                    if p.cls_type[c] != VERTEX:  # edge or face average: u(x_k) = a + d_k, u(x_last) = a - sum d_k
                        last = nodes[-1]
                        for k, x in enumerate(nodes[:-1]):
                            col = self.cls_dual_start[c] + 2 * k + f
                            T[2 * self.gnode_to_iface[x] + f, col] += 1.0
                            T[2 * self.gnode_to_iface[last] + f, col] -= 1.0
                else:
                    for k, x in enumerate(nodes):
                        col = self.cls_dual_start[c] + 2 * k + f
                        T[2 * self.gnode_to_iface[x] + f, col] = 1.0
        return T

    def local(self, j):
        """Local index lists of subdomain j.

        Returns a dict with
          interior_nodes  global node ids of the interior
          iface_nodes     global node ids of Gamma^(j), sorted
          R               global interface dof of each local nodal interface dof
          dual            global transformed dual dof of each local dual dof
          primal          global primal dof of each local primal dof
          classes         classes of Gamma^(j)
          Tloc            local (2|Gamma^(j)| x (n_dual_j + n_primal_j)) basis change
        """
        p = self.part
        inodes = p.interior_nodes(j)
        gnodes = p.iface_nodes_of(j)
        R = np.empty(2 * len(gnodes), np.int64)
        R[0::2] = 2 * self.gnode_to_iface[gnodes]
        R[1::2] = 2 * self.gnode_to_iface[gnodes] + 1
        classes = p.sub_classes(j)
        dual = []
        for c in classes:
            dual.extend(range(self.cls_dual_start[c], self.cls_dual_start[c] + 2 * len(self.cls_dual_nodes[c])))
        primal = []
        for c in classes:
            if p.cls_primal[c]:
                primal.extend([2 * p.primal_index[c], 2 * p.primal_index[c] + 1])
        dual = np.array(dual, np.int64)
        primal = np.array(primal, np.int64)
        cols = np.concatenate([dual, self.n_dual + primal])
        Tloc = self.T[np.ix_(R, cols)]
        return dict(interior_nodes=inodes, iface_nodes=gnodes, R=R, dual=dual,
                    primal=primal, classes=classes, Tloc=Tloc)
