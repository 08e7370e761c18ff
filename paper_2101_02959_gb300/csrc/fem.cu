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
                                   double lz, FemParams fp, double *__restrict__ Ke) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
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
      const double cx = node_ijk[3 * x] * st.h[0], cy = node_ijk[3 * x + 1] * st.h[1], cz = node_ijk[3 * x + 2] * st.h[2];
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
void launch_element_matrices(int ne, const int *elem_ijk, const double h[3], double lz, const FemParams &fp,
                             double *Ke, cudaStream_t s) {
  k_element_matrices<<<ceil_div(ne, 128), 128, 0, s>>>(ne, elem_ijk, h[0], h[1], h[2], lz, fp, Ke);
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
