// Host-side setup plan (see plan.h).  Integer work only; runs once per setup.
#include "plan.h"

#include <algorithm>
#include <map>
#include <set>
#include <numeric>

namespace bd {

namespace {

// hexahedron edges in the corner numbering a = ax + 2 ay + 4 az
const int kHexEdges[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                              {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

struct DSU {
  std::vector<int> p;
  explicit DSU(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int find(int x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
  }
  void join(int a, int b) { a = find(a); b = find(b); if (a != b) p[std::max(a, b)] = std::min(a, b); }
};

}  // namespace

std::string build_plan(Plan &p, const int n[3], const double l[3], const int s[3],
                       const unsigned char *elem_mask, int primal_kind, const Geometry &geo) {
  double ext[3] = {l[0], l[1], l[2]};
  p.geo = geo;
  p.origin[0] = p.origin[1] = p.origin[2] = 0.0;
  if (geo.kind == GEOM_ELLIPSOID) {
    const double half_pi = 1.5707963267948966;
    for (int k = 0; k < 6; ++k)
      if (!(geo.axes[k] > 0)) return "ellipsoid axes must be positive";
    if (!(geo.phi[1] > geo.phi[0]) || !(geo.theta[1] > geo.theta[0]) || !(geo.theta[0] > -half_pi) ||
        !(geo.theta[1] < half_pi))
      return "ellipsoid ranges need phi0 < phi1 and -pi/2 < theta0 < theta1 < pi/2";
    ext[0] = geo.phi[1] - geo.phi[0];
    ext[1] = geo.theta[1] - geo.theta[0];
    ext[2] = 1.0;
    p.origin[0] = geo.phi[0];
    p.origin[1] = geo.theta[0];
  } else if (geo.kind != GEOM_BOX) {
    return "unknown geometry";
  }
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1 || s[d] < 1 || !(ext[d] > 0)) return "mesh sizes, lengths and subdomain sizes must be positive";
    p.n[d] = n[d]; p.l[d] = ext[d]; p.s[d] = s[d]; p.h[d] = ext[d] / n[d];
  }
  if (primal_kind != PRIMAL_V && primal_kind != PRIMAL_VE && primal_kind != PRIMAL_VEF) return "unknown primal space";
  p.primal_kind = primal_kind;
  const int nx = n[0], ny = n[1], nz = n[2];
  const int gx = nx + 1, gy = ny + 1, gz = nz + 1;
  const long ne_full = (long)nx * ny * nz;
  const long nn_full = (long)gx * gy * gz;
  if (nn_full > (1L << 30)) return "mesh too large";
  // elements (x fastest) and used nodes
  std::vector<int> node_of_full(nn_full, -1);
  std::vector<char> used(nn_full, 0);
  p.elem_grid.assign(ne_full, -1);
  for (long e = 0; e < ne_full; ++e) {
    if (elem_mask && !elem_mask[e]) continue;
    int ex = e % nx, ey = (e / nx) % ny, ez = e / ((long)nx * ny);
    for (int a = 0; a < 8; ++a) {
      long g = (ex + (a & 1)) + gx * ((long)(ey + ((a >> 1) & 1)) + gy * (long)(ez + ((a >> 2) & 1)));
      used[g] = 1;
    }
  }
  int nn = 0;
  for (long g = 0; g < nn_full; ++g) if (used[g]) node_of_full[g] = nn++;
  p.n_node = nn;
  p.node_ijk.resize(3 * nn);
  p.coords.resize(3 * nn);
  for (long g = 0; g < nn_full; ++g) if (used[g]) {
    int x = node_of_full[g];
    int i = g % gx, j = (g / gx) % gy, k = g / ((long)gx * gy);
    p.node_ijk[3 * x] = i; p.node_ijk[3 * x + 1] = j; p.node_ijk[3 * x + 2] = k;
    p.coords[3 * x] = p.origin[0] + i * p.h[0];
    p.coords[3 * x + 1] = p.origin[1] + j * p.h[1];
    p.coords[3 * x + 2] = p.origin[2] + k * p.h[2];
  }
  p.conn.clear(); p.elem_ijk.clear();
  int ne = 0;
  for (long e = 0; e < ne_full; ++e) {
    if (elem_mask && !elem_mask[e]) continue;
    int ex = e % nx, ey = (e / nx) % ny, ez = e / ((long)nx * ny);
    p.elem_grid[e] = ne++;
    p.elem_ijk.push_back(ex); p.elem_ijk.push_back(ey); p.elem_ijk.push_back(ez);
    for (int a = 0; a < 8; ++a) {
      long g = (ex + (a & 1)) + gx * ((long)(ey + ((a >> 1) & 1)) + gy * (long)(ez + ((a >> 2) & 1)));
      p.conn.push_back(node_of_full[g]);
    }
  }
  p.n_elem = ne;
  if (ne == 0) return "mask removes every element";
  // global 27-point neighbour table (slot = (dx+1) + 3 (dy+1) + 9 (dz+1))
  p.nbr27.assign(27L * nn, -1);
  for (int x = 0; x < nn; ++x) {
    int i = p.node_ijk[3 * x], j = p.node_ijk[3 * x + 1], k = p.node_ijk[3 * x + 2];
    for (int sl = 0; sl < 27; ++sl) {
      int ii = i + sl % 3 - 1, jj = j + (sl / 3) % 3 - 1, kk = k + sl / 9 - 1;
      if (ii < 0 || jj < 0 || kk < 0 || ii >= gx || jj >= gy || kk >= gz) continue;
      p.nbr27[27L * x + sl] = node_of_full[ii + gx * ((long)jj + gy * (long)kk)];
    }
  }
  // box blocks split into node-connected components
  const int bx = (nx + s[0] - 1) / s[0], by = (ny + s[1] - 1) / s[1];
  std::vector<long> block(ne);
  for (int e = 0; e < ne; ++e)
    block[e] = p.elem_ijk[3 * e] / s[0] + (long)bx * (p.elem_ijk[3 * e + 1] / s[1] + (long)by * (p.elem_ijk[3 * e + 2] / s[2]));
  std::map<long, std::vector<int>> block_elems;
  for (int e = 0; e < ne; ++e) block_elems[block[e]].push_back(e);
  p.elem_sub.assign(ne, -1);
  int nsub = 0;
  std::vector<std::vector<int>> sub_elems;
  for (auto &kv : block_elems) {
    const std::vector<int> &es = kv.second;
    // union elements sharing a node
    std::map<int, int> first_elem_of_node;
    DSU dsu((int)es.size());
    for (int q = 0; q < (int)es.size(); ++q)
      for (int a = 0; a < 8; ++a) {
        int x = p.conn[8 * es[q] + a];
        auto it = first_elem_of_node.find(x);
        if (it == first_elem_of_node.end()) first_elem_of_node[x] = q;
        else dsu.join(q, it->second);
      }
    std::map<int, std::vector<int>> comps;
    for (int q = 0; q < (int)es.size(); ++q) comps[dsu.find(q)].push_back(es[q]);
    std::vector<std::pair<int, std::vector<int>>> ordered;
    for (auto &c : comps) {
      int mn = 1 << 30;
      for (int e : c.second) for (int a = 0; a < 8; ++a) mn = std::min(mn, p.conn[8 * e + a]);
      ordered.push_back({mn, c.second});
    }
    std::sort(ordered.begin(), ordered.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    for (auto &c : ordered) {
      std::vector<int> v = c.second;
      std::sort(v.begin(), v.end());
      for (int e : v) p.elem_sub[e] = nsub;
      sub_elems.push_back(v);
      ++nsub;
    }
  }
  p.n_sub = nsub;
  // N_x
  std::vector<std::vector<int>> nsets(nn);
  for (int j = 0; j < nsub; ++j) {
    std::vector<int> nodes;
    for (int e : sub_elems[j]) for (int a = 0; a < 8; ++a) nodes.push_back(p.conn[8 * e + a]);
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    for (int x : nodes) nsets[x].push_back(j);
  }
  p.nx_ptr.assign(nn + 1, 0); p.nx_idx.clear(); p.mult.assign(nn, 0);
  for (int x = 0; x < nn; ++x) {
    p.mult[x] = (int)nsets[x].size();
    for (int j : nsets[x]) p.nx_idx.push_back(j);
    p.nx_ptr[x + 1] = (int)p.nx_idx.size();
  }
  p.iface_nodes.clear();
  p.node_to_iface.assign(nn, -1);
  for (int x = 0; x < nn; ++x) if (p.mult[x] >= 2) { p.node_to_iface[x] = (int)p.iface_nodes.size(); p.iface_nodes.push_back(x); }
  // classes: same N_x, connected through element edges
  DSU cd(nn);
  for (int e = 0; e < ne; ++e)
    for (auto &ed : kHexEdges) {
      int x = p.conn[8 * e + ed[0]], y = p.conn[8 * e + ed[1]];
      if (p.mult[x] >= 2 && p.mult[y] >= 2 && nsets[x] == nsets[y]) cd.join(x, y);
    }
  std::map<int, std::vector<int>> groups;
  for (int x : p.iface_nodes) groups[cd.find(x)].push_back(x);
  struct Cls { int type, first; std::vector<int> nodes; std::vector<int> subs; };
  std::vector<Cls> cls;
  for (auto &g : groups) {
    Cls c;
    c.nodes = g.second;
    std::sort(c.nodes.begin(), c.nodes.end());
    c.first = c.nodes[0];
    c.subs = nsets[c.first];
    int k = (int)c.subs.size();
    c.type = (k == 2) ? CLS_FACE : ((int)c.nodes.size() > 1 ? CLS_EDGE : CLS_VERTEX);
    cls.push_back(c);
  }
  auto by_type_first = [](const Cls &a, const Cls &b) {
    return a.type != b.type ? a.type < b.type : a.first < b.first; };
  std::sort(cls.begin(), cls.end(), by_type_first);
  // A subdomain fragment of a masked grid may have no vertex on its interface: for
  // subdomains j = 0, 1, ... in order, one without a vertex class promotes the lowest-id
  // node of each of its edge classes (of its face classes if it has no edge) to a vertex
  // class of its own, the rest of each such class is split again into connected classes
  // by the usual rule, and the classes are re-sorted after every subdomain.
  {
    std::vector<std::vector<int>> adj(nn);
    for (int e = 0; e < ne; ++e)
      for (auto &ed : kHexEdges) {
        int x = p.conn[8 * e + ed[0]], y = p.conn[8 * e + ed[1]];
        if (p.mult[x] >= 2 && p.mult[y] >= 2 && nsets[x] == nsets[y]) {
          adj[x].push_back(y);
          adj[y].push_back(x);
        }
      }
    auto make = [&](std::vector<int> nodes, const std::vector<int> &subs) {
      Cls c;
      std::sort(nodes.begin(), nodes.end());
      c.nodes = nodes;
      c.first = nodes[0];
      c.subs = subs;
      c.type = ((int)subs.size() == 2) ? CLS_FACE : ((int)nodes.size() > 1 ? CLS_EDGE : CLS_VERTEX);
      return c;
    };
    for (int j = 0; j < nsub; ++j) {
      bool has_vertex = false;
      std::vector<int> edges, faces;
      for (int c = 0; c < (int)cls.size(); ++c) {
        if (!std::binary_search(cls[c].subs.begin(), cls[c].subs.end(), j)) continue;
        if (cls[c].type == CLS_VERTEX) has_vertex = true;
        else if (cls[c].type == CLS_EDGE) edges.push_back(c);
        else faces.push_back(c);
      }
      if (has_vertex) continue;
      const std::vector<int> &cand = edges.empty() ? faces : edges;
      if (cand.empty()) continue;
      std::vector<char> drop(cls.size(), 0);
      std::vector<Cls> out;
      for (int c : cand) drop[c] = 1;
      for (int c = 0; c < (int)cls.size(); ++c)
        if (!drop[c]) out.push_back(cls[c]);
      for (int c : cand) {
        const Cls &old = cls[c];
        Cls v = make({old.nodes[0]}, old.subs);
        v.type = CLS_VERTEX;  // promoted, whatever |N_x|
        out.push_back(v);
        std::set<int> rest(old.nodes.begin() + 1, old.nodes.end()), seen;
        for (int x : rest) {
          if (seen.count(x)) continue;
          std::vector<int> stack{x}, comp;
          seen.insert(x);
          while (!stack.empty()) {
            int y = stack.back();
            stack.pop_back();
            comp.push_back(y);
            for (int z : adj[y])
              if (rest.count(z) && !seen.count(z)) {
                seen.insert(z);
                stack.push_back(z);
              }
          }
          out.push_back(make(comp, old.subs));
        }
      }
      std::sort(out.begin(), out.end(), by_type_first);
      cls.swap(out);
    }
  }
  p.n_cls = (int)cls.size();
  p.cls_type.resize(p.n_cls);
  p.cls_ptr.assign(1, 0); p.cls_nodes.clear(); p.cls_sub_ptr.assign(1, 0); p.cls_subs.clear();
  p.node_cls.assign(nn, -1);
  for (int c = 0; c < p.n_cls; ++c) {
    p.cls_type[c] = cls[c].type;
    for (int x : cls[c].nodes) { p.cls_nodes.push_back(x); p.node_cls[x] = c; }
    p.cls_ptr.push_back((int)p.cls_nodes.size());
    for (int j : cls[c].subs) p.cls_subs.push_back(j);
    p.cls_sub_ptr.push_back((int)p.cls_subs.size());
  }
  // primal set and gauge
  p.cls_primal.assign(p.n_cls, 0);
  p.primal_index.assign(p.n_cls, -1);
  int np = 0;
  for (int c = 0; c < p.n_cls; ++c) {
    bool pr = p.cls_type[c] == CLS_VERTEX || (primal_kind != PRIMAL_V && p.cls_type[c] == CLS_EDGE) ||
              (primal_kind == PRIMAL_VEF && p.cls_type[c] == CLS_FACE);
    if (pr) { p.cls_primal[c] = 1; p.primal_index[c] = np++; }
  }
  p.n_primal = 2 * np;
  int first_vertex = -1;
  for (int c = 0; c < p.n_cls; ++c) if (p.cls_type[c] == CLS_VERTEX) { first_vertex = c; break; }
  if (first_vertex < 0) return "partition has no vertex class: no gauge vertex";
  p.gauge_node = p.cls_nodes[p.cls_ptr[first_vertex]];
  p.gauge_primal = 2 * p.primal_index[first_vertex] + 1;
  // dual layout
  p.cls_dual_start.assign(p.n_cls, 0);
  p.cls_dual_nodes.assign(p.n_cls, 0);
  int nd = 0;
  for (int c = 0; c < p.n_cls; ++c) {
    int cnt = p.cls_ptr[c + 1] - p.cls_ptr[c];
    // a primal edge or face keeps its average as the primal dof and cnt - 1 deviations as dual dofs
    int dn = p.cls_primal[c] ? (p.cls_type[c] == CLS_VERTEX ? 0 : cnt - 1) : cnt;
    p.cls_dual_start[c] = nd;
    p.cls_dual_nodes[c] = dn;
    nd += 2 * dn;
  }
  p.n_dual = nd;
  // per-subdomain lists
  p.subs.assign(nsub, SubPlan());
  std::vector<std::vector<int>> sub_cls(nsub);
  for (int c = 0; c < p.n_cls; ++c)
    for (int q = p.cls_sub_ptr[c]; q < p.cls_sub_ptr[c + 1]; ++q) sub_cls[p.cls_subs[q]].push_back(c);
  for (int j = 0; j < nsub; ++j) {
    SubPlan &sp = p.subs[j];
    sp.elems = sub_elems[j];
    std::vector<int> nodes;
    for (int e : sp.elems) for (int a = 0; a < 8; ++a) nodes.push_back(p.conn[8 * e + a]);
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    sp.nodes.clear();
    for (int x : nodes) if (p.mult[x] == 1) sp.nodes.push_back(x);
    sp.n_interior = (int)sp.nodes.size();
    for (int x : nodes) if (p.mult[x] >= 2) sp.nodes.push_back(x);
    sp.classes = sub_cls[j];
    bool has_primal = false;
    for (int c : sp.classes) {
      for (int q = 0; q < 2 * p.cls_dual_nodes[c]; ++q) sp.dual.push_back(p.cls_dual_start[c] + q);
      if (p.cls_primal[c]) has_primal = true;
    }
    for (int c : sp.classes)
      if (p.cls_primal[c]) { sp.primal.push_back(2 * p.primal_index[c]); sp.primal.push_back(2 * p.primal_index[c] + 1); }
    if (!has_primal) return "subdomain " + std::to_string(j) + " has no primal constraint";
    // local neighbour table
    std::map<int, int> loc;
    for (int q = 0; q < (int)sp.nodes.size(); ++q) loc[sp.nodes[q]] = q;
    sp.nbr.assign(27 * sp.nodes.size(), -1);
    for (int q = 0; q < (int)sp.nodes.size(); ++q) {
      int x = sp.nodes[q];
      for (int sl = 0; sl < 27; ++sl) {
        int y = p.nbr27[27L * x + sl];
        if (y < 0) continue;
        auto it = loc.find(y);
        if (it != loc.end()) sp.nbr[27 * q + sl] = it->second;
      }
    }
  }
  // global change of basis T: nodal interface dof <- transformed dof
  const int nif = p.n_iface();
  std::vector<std::vector<std::pair<int, double>>> rows(nif);
  for (int c = 0; c < p.n_cls; ++c) {
    const int *nodes = &p.cls_nodes[p.cls_ptr[c]];
    int cnt = p.cls_ptr[c + 1] - p.cls_ptr[c];
    for (int f = 0; f < 2; ++f) {
      if (p.cls_primal[c]) {
        int col_a = p.n_dual + 2 * p.primal_index[c] + f;
        for (int k = 0; k < cnt; ++k) rows[2 * p.node_to_iface[nodes[k]] + f].push_back({col_a, 1.0});
        if (p.cls_type[c] != CLS_VERTEX) {  // average: u(x_k) = a + d_k, u(x_last) = a - sum_k d_k
          int last = nodes[cnt - 1];
          for (int k = 0; k < cnt - 1; ++k) {
            int col = p.cls_dual_start[c] + 2 * k + f;
            rows[2 * p.node_to_iface[nodes[k]] + f].push_back({col, 1.0});
            rows[2 * p.node_to_iface[last] + f].push_back({col, -1.0});
          }
        }
      } else {
        for (int k = 0; k < cnt; ++k) rows[2 * p.node_to_iface[nodes[k]] + f].push_back({p.cls_dual_start[c] + 2 * k + f, 1.0});
      }
    }
  }
  const int nt = p.n_dual + p.n_primal;
  std::vector<std::vector<std::pair<int, double>>> cols(nt);
  p.T_ptr.assign(1, 0); p.T_col.clear(); p.T_val.clear();
  for (int r = 0; r < nif; ++r) {
    std::sort(rows[r].begin(), rows[r].end());
    for (auto &e : rows[r]) { p.T_col.push_back(e.first); p.T_val.push_back(e.second); cols[e.first].push_back({r, e.second}); }
    p.T_ptr.push_back((int)p.T_col.size());
  }
  p.Tt_ptr.assign(1, 0); p.Tt_col.clear(); p.Tt_val.clear();
  for (int c = 0; c < nt; ++c) {
    std::sort(cols[c].begin(), cols[c].end());
    for (auto &e : cols[c]) { p.Tt_col.push_back(e.first); p.Tt_val.push_back(e.second); }
    p.Tt_ptr.push_back((int)p.Tt_col.size());
  }
  return "";
}

void local_T(const Plan &p, int j, std::vector<int> &ptr, std::vector<int> &row, std::vector<double> &val) {
  const SubPlan &sp = p.subs[j];
  // local nodal interface dof of each global interface dof present in Gamma^(j)
  std::map<int, int> gl;
  for (int q = sp.n_interior; q < (int)sp.nodes.size(); ++q) {
    int gi = p.node_to_iface[sp.nodes[q]];
    gl[2 * gi] = 2 * (q - sp.n_interior);
    gl[2 * gi + 1] = 2 * (q - sp.n_interior) + 1;
  }
  ptr.assign(1, 0); row.clear(); val.clear();
  auto emit = [&](int tcol) {
    for (int q = p.Tt_ptr[tcol]; q < p.Tt_ptr[tcol + 1]; ++q) {
      auto it = gl.find(p.Tt_col[q]);
      if (it != gl.end()) { row.push_back(it->second); val.push_back(p.Tt_val[q]); }
    }
    ptr.push_back((int)row.size());
  };
  for (int d : sp.dual) emit(d);
  for (int q : sp.primal) emit(p.n_dual + q);
}

}  // namespace bd
