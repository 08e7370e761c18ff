// Q1 assembly, gating, residual and reductions (Sections 2, 3a, 3b).
#include "kernels.cuh"

namespace bd {

// ---------------------------------------------------------------------------
// Element matrices (Section 3a).  For a box element of sides (hx, hy, hz) and
// a constant tensor D, the entry for corners a, b is
//   sum_{p,q} D_pq  prod_d  I_d(a_d, b_d, p == d, q == d)
// with the exact 1D integrals of the linear shape functions l_0 = 1 - t/h,
// l_1 = t/h:  int l_i l_j = h (2 if i == j else 1) / 6,  int l_i' l_j = s_i/2,
// int l_i l_j' = s_j/2,  int l_i' l_j' = s_i s_j / h  (s_0 = -1, s_1 = +1).
// ---------------------------------------------------------------------------
__device__ inline double int1d(int i, int j, bool di, bool dj, double hh) {
  const double si = i ? 1.0 : -1.0, sj = j ? 1.0 : -1.0;
  if (!di && !dj) return hh * (i == j ? 2.0 : 1.0) / 6.0;
  if (di && !dj) return 0.5 * si;
  if (!di && dj) return 0.5 * sj;
  return si * sj / hh;
}

// Fibre frame of the slab (Section 6): angle -60 + 120 (1 - z/lz) degrees in
// the x-y plane, sheet normal e_z; D = sum_k sigma_k a_k a_k^T.
__device__ inline void slab_tensor(const double sig[3], double z, double lz, double D[3][3]) {
  const double alpha = (-60.0 + 120.0 * (1.0 - z / lz)) * (M_PI / 180.0);
  double c, s;
  sincos(alpha, &s, &c);
  const double al[3] = {c, s, 0.0}, at[3] = {-s, c, 0.0}, an[3] = {0.0, 0.0, 1.0};
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) D[p][q] = sig[0] * al[p] * al[q] + sig[1] * at[p] * at[q] + sig[2] * an[p] * an[q];
}

__global__ void k_element_matrices(int ne, const int *__restrict__ elem_ijk, double hx, double hy, double hz,
                                   double lz, FemParams fp, double *__restrict__ Ke, double *__restrict__ Me) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double vol8 = hx * hy * hz / 8.0;
  for (int a = 0; a < 8; ++a) Me[8LL * e + a] = vol8;
  const double zc = (elem_ijk[3 * e + 2] + 0.5) * hz;
  const double h[3] = {hx, hy, hz};
  for (int f = 0; f < 2; ++f) {
    double D[3][3];
    slab_tensor(f == 0 ? fp.sigma_i : fp.sigma_e, zc, lz, D);
    double *K = Ke + ((long long)e * 2 + f) * 64;
    for (int a = 0; a < 8; ++a) {
      const int ia[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
      for (int b = 0; b < 8; ++b) {
        const int ib[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
        double acc = 0.0;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) {
            double v = D[p][q];
            for (int d = 0; d < 3; ++d) v *= int1d(ia[d], ib[d], p == d, q == d, h[d]);
            acc += v;
          }
        K[a * 8 + b] = acc;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Truncated ellipsoid (Section 6).  Parametric (phi, theta, r) maps to
// (a cos(theta) cos(phi), b cos(theta) sin(phi), c sin(theta)) with a, b, c
// linear in the wall depth r.  The fibre frame at a point: a_n the outward unit
// normal of the surface r = const, t1 the unit tangent along phi, t2 = a_n x t1,
// a_l = cos(alpha) t1 + sin(alpha) t2 with alpha = -60 + 120 (1 - r) degrees,
// a_t = a_n x a_l.
// ---------------------------------------------------------------------------
__device__ inline void ell_radii(const double ax[6], double r, double &a, double &b, double &c) {
  a = ax[0] + r * (ax[1] - ax[0]);
  b = ax[2] + r * (ax[3] - ax[2]);
  c = ax[4] + r * (ax[5] - ax[4]);
}

__device__ inline void ell_point(const double ax[6], double phi, double th, double r, double X[3]) {
  double a, b, c, sp, cp, st, ct;
  ell_radii(ax, r, a, b, c);
  sincos(phi, &sp, &cp);
  sincos(th, &st, &ct);
  X[0] = a * ct * cp;
  X[1] = b * ct * sp;
  X[2] = c * st;
}

__device__ inline void cross3(const double u[3], const double v[3], double w[3]) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

__device__ inline void ell_tensor(const double sig[3], const double ax[6], double phi, double th, double r,
                                  double D[3][3]) {
  double a, b, c, sp, cp, st, ct;
  ell_radii(ax, r, a, b, c);
  sincos(phi, &sp, &cp);
  sincos(th, &st, &ct);
  const double x_phi[3] = {-a * ct * sp, b * ct * cp, 0.0};
  const double x_th[3] = {-a * st * cp, -b * st * sp, c * ct};
  const double x_r[3] = {(ax[1] - ax[0]) * ct * cp, (ax[3] - ax[2]) * ct * sp, (ax[5] - ax[4]) * st};
  double n[3];
  cross3(x_phi, x_th, n);
  const double sgn = (n[0] * x_r[0] + n[1] * x_r[1] + n[2] * x_r[2]) < 0.0 ? -1.0 : 1.0;
  const double nn = sgn / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const double tn = 1.0 / sqrt(x_phi[0] * x_phi[0] + x_phi[1] * x_phi[1]);
  double an[3], t1[3], t2[3], al[3], at[3];
  for (int p = 0; p < 3; ++p) { an[p] = n[p] * nn; t1[p] = x_phi[p] * tn; }
  cross3(an, t1, t2);
  double sa, ca;
  sincos((-60.0 + 120.0 * (1.0 - r)) * (M_PI / 180.0), &sa, &ca);
  for (int p = 0; p < 3; ++p) al[p] = ca * t1[p] + sa * t2[p];
  cross3(an, al, at);
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) D[p][q] = sig[0] * al[p] * al[q] + sig[1] * at[p] * at[q] + sig[2] * an[p] * an[q];
}

// Isoparametric Q1 element (Section 3a) on the mapped hexahedron: stiffness
// int grad(phi_a)^T D grad(phi_b) and lumped masses int phi_a by 2x2x2 Gauss on
// the reference cube, physical gradients J^-T times the reference ones; D is
// taken at the element's parametric centroid.  One thread per element
// (setup only).
__global__ void k_element_matrices_iso(int ne, const int *__restrict__ elem_ijk, GeoParams g, FemParams fp,
                                       double *__restrict__ Ke, double *__restrict__ Me) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int ie[3] = {elem_ijk[3 * e], elem_ijk[3 * e + 1], elem_ijk[3 * e + 2]};
  double X[8][3];
  for (int a = 0; a < 8; ++a) {
    const int c[3] = {ie[0] + (a & 1), ie[1] + ((a >> 1) & 1), ie[2] + ((a >> 2) & 1)};
    ell_point(g.axes, g.o[0] + c[0] * g.h[0], g.o[1] + c[1] * g.h[1], g.o[2] + c[2] * g.h[2], X[a]);
  }
  double D[2][3][3];
  const double pc[3] = {g.o[0] + (ie[0] + 0.5) * g.h[0], g.o[1] + (ie[1] + 0.5) * g.h[1],
                        g.o[2] + (ie[2] + 0.5) * g.h[2]};
  ell_tensor(fp.sigma_i, g.axes, pc[0], pc[1], pc[2], D[0]);
  ell_tensor(fp.sigma_e, g.axes, pc[0], pc[1], pc[2], D[1]);
  double *K = Ke + (long long)e * 128;
  double *M = Me + 8LL * e;
  for (int t = 0; t < 128; ++t) K[t] = 0.0;
  for (int a = 0; a < 8; ++a) M[a] = 0.0;
  const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  for (int q = 0; q < 8; ++q) {
    const double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], gp[(q >> 2) & 1]};
    double N[8], dN[8][3];
    for (int a = 0; a < 8; ++a) {
      const int b[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
      double l[3], sd[3];
      for (int d = 0; d < 3; ++d) { l[d] = b[d] ? xi[d] : 1.0 - xi[d]; sd[d] = b[d] ? 1.0 : -1.0; }
      N[a] = l[0] * l[1] * l[2];
      dN[a][0] = sd[0] * l[1] * l[2];
      dN[a][1] = l[0] * sd[1] * l[2];
      dN[a][2] = l[0] * l[1] * sd[2];
    }
    double J[3][3];  // J[p][d] = d x_p / d xi_d
    for (int p = 0; p < 3; ++p)
      for (int d = 0; d < 3; ++d) {
        double v = 0.0;
        for (int a = 0; a < 8; ++a) v += X[a][p] * dN[a][d];
        J[p][d] = v;
      }
    double C[3][3];  // cofactors: J^-1[d][p] = C[p][d] / det
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    const double w = det / 8.0, inv = 1.0 / det;
    double G[8][3];  // physical gradients: G[a][p] = sum_d dN[a][d] J^-1[d][p]
    for (int a = 0; a < 8; ++a)
      for (int p = 0; p < 3; ++p) G[a][p] = (dN[a][0] * C[p][0] + dN[a][1] * C[p][1] + dN[a][2] * C[p][2]) * inv;
    for (int a = 0; a < 8; ++a) M[a] += w * N[a];
    for (int f = 0; f < 2; ++f) {
      double DG[8][3];
      for (int b = 0; b < 8; ++b)
        for (int p = 0; p < 3; ++p) DG[b][p] = D[f][p][0] * G[b][0] + D[f][p][1] * G[b][1] + D[f][p][2] * G[b][2];
      for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
          K[f * 64 + a * 8 + b] += w * (G[a][0] * DG[b][0] + G[a][1] * DG[b][1] + G[a][2] * DG[b][2]);
    }
  }
}

// Lumped node masses: the sum over the elements around x (those of one
// subdomain, when given) of their corner mass at x, in the stencil's element order.
__global__ void k_mass_gather(int nrows, const int *__restrict__ row_node, const int *__restrict__ row_sub,
                              const int *__restrict__ node_ijk, const int *__restrict__ elem_grid,
                              const int *__restrict__ elem_sub, int nx, int ny, int nz, const double *__restrict__ Me,
                              double *__restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int x = row_node ? row_node[r] : r;
  const int sub = row_sub ? row_sub[r] : -1;
  const int i = node_ijk[3 * x], j = node_ijk[3 * x + 1], k = node_ijk[3 * x + 2];
  double acc = 0.0;
  for (int ez = 0; ez < 2; ++ez)
    for (int ey = 0; ey < 2; ++ey)
      for (int ex = 0; ex < 2; ++ex) {
        const int gi = i - 1 + ex, gj = j - 1 + ey, gk = k - 1 + ez;
        if (gi < 0 || gj < 0 || gk < 0 || gi >= nx || gj >= ny || gk >= nz) continue;
        const int e = elem_grid[gi + nx * (gj + ny * gk)];
        if (e < 0) continue;
        if (sub >= 0 && elem_sub[e] != sub) continue;
        acc += Me[8LL * e + (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez)];
      }
  out[r] = acc;
}

// Stencil rows: for node x (optionally restricted to the elements of one
// subdomain) and each of the 27 neighbour slots, the sum over the elements
// around x that hold both x and the neighbour of their matrix entries.
// Summation order is fixed (elements by grid position), so it is deterministic.
__global__ void k_stencil_gather(int nrows, const int *__restrict__ row_node, const int *__restrict__ row_sub,
                                 const int *__restrict__ node_ijk, const int *__restrict__ elem_grid,
                                 const int *__restrict__ elem_sub, int nx, int ny, int nz,
                                 const double *__restrict__ Ke, double *__restrict__ out, int soa_stride) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nrows * 27) return;
  const int r = (int)(t / 27), sl = (int)(t % 27);
  const int x = row_node[r];
  const int sub = row_sub ? row_sub[r] : -1;
  const int dx = sl % 3 - 1, dy = (sl / 3) % 3 - 1, dz = sl / 9 - 1;
  const int i = node_ijk[3 * x], j = node_ijk[3 * x + 1], k = node_ijk[3 * x + 2];
  double acc[2] = {0.0, 0.0};
  for (int ez = 0; ez < 2; ++ez)
    for (int ey = 0; ey < 2; ++ey)
      for (int ex = 0; ex < 2; ++ex) {
        // element whose corner (1-ex, 1-ey, 1-ez) is x
        const int gi = i - 1 + ex, gj = j - 1 + ey, gk = k - 1 + ez;
        if (gi < 0 || gj < 0 || gk < 0 || gi >= nx || gj >= ny || gk >= nz) continue;
        const int e = elem_grid[gi + nx * (gj + ny * gk)];
        if (e < 0) continue;
        if (sub >= 0 && elem_sub[e] != sub) continue;
        const int ax = 1 - ex, ay = 1 - ey, az = 1 - ez;
        const int bx = ax + dx, by = ay + dy, bz = az + dz;
        if (bx < 0 || by < 0 || bz < 0 || bx > 1 || by > 1 || bz > 1) continue;
        const int a = ax + 2 * ay + 4 * az, b = bx + 2 * by + 4 * bz;
        acc[0] += Ke[((long long)e * 2 + 0) * 64 + a * 8 + b];
        acc[1] += Ke[((long long)e * 2 + 1) * 64 + a * 8 + b];
      }
  if (soa_stride > 0) {  // global stencil: SoA [f][slot][node]
    out[(long long)(0 * 27 + sl) * soa_stride + r] = acc[0];
    out[(long long)(1 * 27 + sl) * soa_stride + r] = acc[1];
  } else {  // local stencil: [row][slot][f]
    out[((long long)r * 27 + sl) * 2 + 0] = acc[0];
    out[((long long)r * 27 + sl) * 2 + 1] = acc[1];
  }
}

// ---------------------------------------------------------------------------
// Rogers-McCulloch model (Section 2) and Step 1 (Section 3b).
// ---------------------------------------------------------------------------
__device__ inline double rmc_iion(double v, double w, const FemParams &p) {
  return p.G * v * (1.0 - v / p.vth) * (1.0 - v / p.vp) + p.eta1 * v * w;
}
__device__ inline double rmc_diion(double v, double w, const FemParams &p) {
  // derivative of G v (1 - v a)(1 - v b) + eta1 v w with a = 1/vth, b = 1/vp
  const double a = 1.0 / p.vth, b = 1.0 / p.vp;
  return p.G * (1.0 - 2.0 * (a + b) * v + 3.0 * a * b * v * v) + p.eta1 * w;
}

__global__ void k_gating(int n, const double *__restrict__ ui, const double *__restrict__ ue,
                         const double *__restrict__ w, double *__restrict__ wn, FemParams p) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const double v = ui[x] - ue[x];
  const double te = p.tau * p.eta2;
  wn[x] = (w[x] + te * v / p.vp) / (1.0 + te);
}

// F(u) - G (Step 2) with the Jacobian factor chi Cm + tau dI/dv, and per-block
// partial sums of ||F - G||^2.  u = x + lam * s when s != nullptr (line search).
__global__ void k_residual(int n, const double *__restrict__ stencil, const int *__restrict__ nbr,
                           const double *__restrict__ mass, const int *__restrict__ node_ijk,
                           const double *__restrict__ ui0, const double *__restrict__ ue0,
                           const double *__restrict__ si, const double *__restrict__ se, double lam,
                           const double *__restrict__ wn, const double *__restrict__ uin,
                           const double *__restrict__ uen, FemParams p, StimParams st,
                           double *__restrict__ ri, double *__restrict__ re, double *__restrict__ factor,
                           double *__restrict__ ui_out, double *__restrict__ ue_out, double *__restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    double Au_i = 0.0, Au_e = 0.0;
#pragma unroll 3
    for (int sl = 0; sl < 27; ++sl) {
      const int y = nbr[(long long)sl * n + x];
      if (y < 0) continue;
      double yi = ui0[y], ye = ue0[y];
      if (si) { yi += lam * si[y]; ye += lam * se[y]; }
      Au_i += stencil[(long long)sl * n + x] * yi;
      Au_e += stencil[(long long)(27 + sl) * n + x] * ye;
    }
    double xi = ui0[x], xe = ue0[x];
    if (si) { xi += lam * si[x]; xe += lam * se[x]; }
    const double v = xi - xe, vn = uin[x] - uen[x];
    const double M = mass[x];
    const double cap = p.chi_cm * M * (v - vn);
    const double ion = p.tau * M * rmc_iion(v, wn[x], p);
    double app = 0.0;
    if (st.active) {
      const double cx = st.o[0] + node_ijk[3 * x] * st.h[0], cy = st.o[1] + node_ijk[3 * x + 1] * st.h[1],
                   cz = st.o[2] + node_ijk[3 * x + 2] * st.h[2];
      const double eps = 1e-12;
      if (cx >= st.box[0] - eps && cx <= st.box[1] + eps && cy >= st.box[2] - eps && cy <= st.box[3] + eps &&
          cz >= st.box[4] - eps && cz <= st.box[5] + eps)
        app = p.tau * M * st.amp;
    }
    const double a = cap + p.tau * Au_i + ion - app;
    const double b = -cap + p.tau * Au_e - ion + app;
    ri[x] = a;
    re[x] = b;
    if (factor) factor[x] = p.chi_cm + p.tau * rmc_diion(v, wn[x], p);
    if (ui_out) { ui_out[x] = xi; ue_out[x] = xe; }
    acc += a * a + b * b;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0 && partial) partial[blockIdx.x] = acc;
}

// Partial sums of up to three dot products over the same index range.
__global__ void k_dot3(int n, const double *__restrict__ a0, const double *__restrict__ b0,
                       const double *__restrict__ a1, const double *__restrict__ b1,
                       const double *__restrict__ a2, const double *__restrict__ b2, double *__restrict__ partial) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    s0 += a0[x] * b0[x];
    if (a1) s1 += a1[x] * b1[x];
    if (a2) s2 += a2[x] * b2[x];
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x] = s0;
    partial[3 * blockIdx.x + 1] = s1;
    partial[3 * blockIdx.x + 2] = s2;
  }
}

// Sums `width` interleaved partial series of length nblk (fixed order).
__global__ void k_finalize(int nblk, int width, const double *__restrict__ partial, double *__restrict__ out) {
  __shared__ double sh[32];
  for (int c = 0; c < width; ++c) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += partial[(long long)b * width + c];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[c] = v;
  }
}

// u += c * (1, 1) shift to the zero lumped-mass mean of u_e (scal[0] = sum M u_e, scal[1] = sum M).
__global__ void k_gauge_shift(int n, double *__restrict__ ui, double *__restrict__ ue, const double *__restrict__ scal) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const double c = scal[0] / scal[1];
  ui[x] -= c;
  ue[x] -= c;
}

// ---- host launchers --------------------------------------------------------
void launch_element_matrices(int ne, const int *elem_ijk, const GeoParams &g, const FemParams &fp, double *Ke,
                             double *Me, cudaStream_t s) {
  if (ne <= 0) return;
  if (g.kind == 1)
    k_element_matrices_iso<<<ceil_div(ne, 64), 64, 0, s>>>(ne, elem_ijk, g, fp, Ke, Me);
  else
    k_element_matrices<<<ceil_div(ne, 128), 128, 0, s>>>(ne, elem_ijk, g.h[0], g.h[1], g.h[2], g.lz, fp, Ke, Me);
  count_launch();
}

void launch_mass_gather(int nrows, const int *row_node, const int *row_sub, const int *node_ijk,
                        const int *elem_grid, const int *elem_sub, const int n[3], const double *Me, double *out,
                        cudaStream_t s) {
  if (nrows <= 0) return;
  k_mass_gather<<<ceil_div(nrows, 256), 256, 0, s>>>(nrows, row_node, row_sub, node_ijk, elem_grid, elem_sub, n[0],
                                                      n[1], n[2], Me, out);
  count_launch();
}

void launch_stencil_gather(int nrows, const int *row_node, const int *row_sub, const int *node_ijk,
                           const int *elem_grid, const int *elem_sub, const int n[3], const double *Ke,
                           double *out, int soa_stride, cudaStream_t s) {
  const long long tot = (long long)nrows * 27;
  k_stencil_gather<<<(int)((tot + 255) / 256), 256, 0, s>>>(nrows, row_node, row_sub, node_ijk, elem_grid, elem_sub,
                                                          n[0], n[1], n[2], Ke, out, soa_stride);
  count_launch();
}

void launch_gating(int n, const double *ui, const double *ue, const double *w, double *wn, const FemParams &p,
                   cudaStream_t s) {
  k_gating<<<ceil_div(n, 256), 256, 0, s>>>(n, ui, ue, w, wn, p);
  count_launch();
}

void launch_residual(int n, const double *stencil, const int *nbr, const double *mass, const int *node_ijk,
                     const double *ui0, const double *ue0, const double *si, const double *se, double lam,
                     const double *wn, const double *uin, const double *uen, const FemParams &p,
                     const StimParams &st, double *ri, double *re, double *factor, double *ui_out,
                     double *ue_out, double *partial, double *norm2, cudaStream_t s) {
  k_residual<<<kRedBlocks, 256, 0, s>>>(n, stencil, nbr, mass, node_ijk, ui0, ue0, si, se, lam, wn, uin, uen, p, st,
                                        ri, re, factor, ui_out, ue_out, partial);
  count_launch();
  if (norm2) {
    k_finalize<<<1, 256, 0, s>>>(kRedBlocks, 1, partial, norm2);
    count_launch();
  }
}

void launch_dot3(int n, const double *a0, const double *b0, const double *a1, const double *b1, const double *a2,
                 const double *b2, double *partial, double *out, cudaStream_t s) {
  k_dot3<<<kRedBlocks, 256, 0, s>>>(n, a0, b0, a1, b1, a2, b2, partial);
  count_launch();
  k_finalize<<<1, 256, 0, s>>>(kRedBlocks, 3, partial, out);
  count_launch();
}

void launch_sum_partials(int nblk, const double *partial, double *out, cudaStream_t s) {
  k_finalize<<<1, 256, 0, s>>>(nblk, 1, partial, out);
  count_launch();
}

void launch_gauge_shift(int n, double *ui, double *ue, const double *scal, cudaStream_t s) {
  k_gauge_shift<<<ceil_div(n, 256), 256, 0, s>>>(n, ui, ue, scal);
  count_launch();
}

}  // namespace bd
