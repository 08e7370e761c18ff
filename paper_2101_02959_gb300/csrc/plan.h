// Host-side setup plan: grid, subdomains, interface classes, dof maps.
//
// Section 4.1 of the paper: non-overlapping subdomains made of whole
// elements, interface Gamma = nodes in at least two subdomains, the sets N_x
// (subdomains whose closure holds node x) and the face / edge / vertex
// equivalence classes they induce; primal constraints V (vertex values) or
// V+E (vertex values and edge averages, Section 6, Test 3).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace bd {

enum { CLS_VERTEX = 0, CLS_EDGE = 1, CLS_FACE = 2 };
enum { PRIMAL_V = 0, PRIMAL_VE = 1, PRIMAL_VEF = 2 };
enum { GEOM_BOX = 0, GEOM_ELLIPSOID = 1 };

// Domain geometry (Section 6).  A box grid spans [0,l0]x[0,l1]x[0,l2]; the
// truncated ellipsoid is a grid uniform in the parametric coordinates
// (phi, theta, r) over [phi0,phi1]x[theta0,theta1]x[0,1], mapped by
// x = a(r) cos(theta) cos(phi), y = b(r) cos(theta) sin(phi), z = c(r) sin(theta)
// with a(r) = a1 + r (a2 - a1) and likewise b, c (axes = a1, a2, b1, b2, c1, c2).
struct Geometry {
  int kind = GEOM_BOX;
  double axes[6] = {0, 0, 0, 0, 0, 0};
  double phi[2] = {0, 0}, theta[2] = {0, 0};
};

struct SubPlan {
  std::vector<int> nodes;     // local node order: interior (sorted) then interface (sorted)
  int n_interior = 0;         // number of interior nodes
  std::vector<int> elems;     // own elements (sorted)
  std::vector<int> classes;   // classes on Gamma^(j), in class order
  std::vector<int> dual;      // global transformed dual dof of each local dual dof
  std::vector<int> primal;    // global primal dof of each local primal dof
  std::vector<int> nbr;       // 27 local neighbour indices per local node (-1 = none)
  int nI() const { return 2 * n_interior; }
  int nG() const { return 2 * ((int)nodes.size() - n_interior); }
  int nD() const { return (int)dual.size(); }
  int nP() const { return (int)primal.size(); }
};

struct Plan {
  // grid
  int n[3] = {0, 0, 0};
  Geometry geo;
  // grid extent, spacing and origin in the parametric coordinates (cm for a box)
  double l[3] = {0, 0, 0}, h[3] = {0, 0, 0}, origin[3] = {0, 0, 0};
  int s[3] = {0, 0, 0};
  int n_node = 0, n_elem = 0;
  std::vector<int> conn;        // 8 node ids per element, corner a = ax + 2 ay + 4 az
  std::vector<int> elem_ijk;    // 3 per element
  std::vector<int> node_ijk;    // 3 per node
  std::vector<int> elem_grid;   // full element grid -> element id or -1
  std::vector<int> nbr27;       // 27 neighbour node ids per node (-1 = none)
  std::vector<double> coords;   // 3 parametric coordinates per node: origin + ijk h
  // partition
  int n_sub = 0;
  std::vector<int> elem_sub;
  std::vector<int> nx_ptr, nx_idx;  // N_x as CSR over nodes
  std::vector<int> mult;            // |N_x|
  std::vector<int> iface_nodes;     // sorted
  std::vector<int> node_to_iface;   // -1 for interior nodes
  // classes
  int n_cls = 0;
  std::vector<int> cls_type, cls_ptr, cls_nodes, cls_sub_ptr, cls_subs;
  std::vector<int> node_cls;
  int primal_kind = PRIMAL_V;
  std::vector<int> cls_primal;      // 0/1
  std::vector<int> primal_index;    // class -> primal class index or -1
  int n_primal = 0;                 // 2 per primal class
  int gauge_node = -1, gauge_primal = -1;
  std::vector<int> cls_dual_start, cls_dual_nodes;  // per class: first global dual dof, # dual nodes
  int n_dual = 0;
  std::vector<SubPlan> subs;
  // global change of basis T (nodal interface dofs <- transformed dofs), CSR by nodal row
  std::vector<int> T_ptr, T_col;
  std::vector<double> T_val;
  // its transpose, CSR by transformed row (dual dofs first, then primal)
  std::vector<int> Tt_ptr, Tt_col;
  std::vector<double> Tt_val;
  int n_iface() const { return 2 * (int)iface_nodes.size(); }
};

// Builds the plan; returns "" on success or an error message.
std::string build_plan(Plan &p, const int n[3], const double l[3], const int s[3],
                       const unsigned char *elem_mask, int primal_kind, const Geometry &geo = Geometry());

// Local change of basis of subdomain j, CSC by transformed local dof
// ([dual; primal]): entries (local nodal interface dof, coefficient).
void local_T(const Plan &p, int j, std::vector<int> &ptr, std::vector<int> &row,
             std::vector<double> &val);

}  // namespace bd
