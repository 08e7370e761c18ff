// Domain-decomposition kernels: local assembly, Schur blocks, deluxe scaling,
// coarse problem, BDDC / FETI-DP application and the PCG recurrences
// (Sections 4.1-4.4 of the paper).
#include <algorithm>

#include "dd_kernels.cuh"

namespace bd {

// ---- local matrices K^(j) (Section 4.1, local forms a^(j)) -------------------
// One thread per (local node q, stencil slot).  Local dofs are 2a + field in the
// order [interior nodes; interface nodes].  The self slot also writes the
// coupling Kc = M^(j) (chi Cm + tau dI/dv): +Kc on both diagonals, -Kc across.
template <typename T>
__global__ void k_assemble_local(int nq, const int *__restrict__ q_sub, const int *__restrict__ q_loc,
                                 const int *__restrict__ q_node, const int *__restrict__ nbr,
                                 const double *__restrict__ stencil, const double *__restrict__ mass,
                                 const double *__restrict__ factor, double tau, const MatDesc *__restrict__ desc,
                                 T *__restrict__ base) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nq * 27) return;
  const int q = (int)(t / 27), sl = (int)(t % 27);
  const int b = nbr[(long long)q * 27 + sl];
  if (b < 0) return;
  const MatDesc d = desc[q_sub[q]];
  const int a = q_loc[q];
  T *K = base + d.off;
  double vi = tau * stencil[((long long)q * 27 + sl) * 2 + 0];
  double ve = tau * stencil[((long long)q * 27 + sl) * 2 + 1];
  if (sl == 13) {
    const double kc = mass[q] * factor[q_node[q]];
    vi += kc;
    ve += kc;
    K[(long long)(2 * a) * d.ld + 2 * a + 1] = (T)(-kc);
    K[(long long)(2 * a + 1) * d.ld + 2 * a] = (T)(-kc);
  }
  K[(long long)(2 * a) * d.ld + 2 * b] = (T)vi;
  K[(long long)(2 * a + 1) * d.ld + 2 * b + 1] = (T)ve;
}

// ---- block copies ------------------------------------------------------------
template <typename TS, typename TD>
__global__ void __launch_bounds__(256) k_copy(const CopyTask *__restrict__ tasks, const TS *__restrict__ src,
                                              TD *__restrict__ dst) {
  // 32 x 32 tiles through shared memory, so reads and writes stay coalesced however
  // the tile is transposed.  mode 0: dst(i, k) = src(r0 + i, c0 + k); mode 1:
  // dst(i, k) = src(r0 + k, c0 + i); modes 2 and 3: the full symmetric matrix from
  // the lower triangle, dst(i, k) = src(r0 + max, c0 + min).  sign is +1 or -1.
  const CopyTask c = tasks[blockIdx.y];
  __shared__ TS tD[32][33], tT[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int ntr = (c.rows + 31) / 32, ntc = (c.cols + 31) / 32;
  const bool sym = c.mode >= 2;
  const bool neg = c.sign < 0.0;
  for (int tile = blockIdx.x; tile < ntr * ntc; tile += gridDim.x) {
    const int i0 = (tile / ntc) * 32, k0 = (tile % ntc) * 32;
    const bool need_d = c.mode == 0 || (sym && i0 + 31 >= k0);
    const bool need_t = c.mode == 1 || (sym && k0 + 31 > i0);
    __syncthreads();
    if (need_d) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, k = k0 + tx;
        if (i < c.rows && k < c.cols && (!sym || i >= k))
          tD[ty + 8 * q][tx] = src[c.src_off + (long long)(c.r0 + i) * c.src_ld + c.c0 + k];
      }
    }
    if (need_t) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kk = k0 + ty + 8 * q, ii = i0 + tx;  // element (ii, kk) of dst
        if (ii < c.rows && kk < c.cols && (!sym || kk > ii))
          tT[ty + 8 * q][tx] = src[c.src_off + (long long)(c.r0 + kk) * c.src_ld + c.c0 + ii];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ty + 8 * q, k = k0 + tx;
      if (i < c.rows && k < c.cols) {
        const bool direct = c.mode == 0 || (sym && i >= k);
        const TS v = direct ? tD[ty + 8 * q][tx] : tT[tx][ty + 8 * q];
        dst[c.dst_off + (long long)i * c.dst_ld + k] = (TD)(neg ? -v : v);
      }
    }
  }
}

// ---- augmented matrix of the constrained local problem ------------------------
// Aug = [[Sb_DD, Sb_DP, I], [Sb_PD, Sb_PP, 0], [I, 0, 0]] with Sb = T^T S T
// (change of basis for the primal averages), S read from the full symmetric
// copy of S_Gamma.  T_loc is CSC by transformed dof.  One warp per row a, lanes
// over the columns b <= a (the factorisation and the copies read the lower
// triangle only); sums in the matrix precision.
template <typename T>
__global__ void __launch_bounds__(256) k_build_aug(const MatDesc *__restrict__ sdesc, const T *__restrict__ sbase,
                                                   const MatDesc *__restrict__ adesc, T *__restrict__ abase,
                                                   const int *__restrict__ nD, const int *__restrict__ tptr_off,
                                                   const int *__restrict__ tptr, const int *__restrict__ trow,
                                                   const T *__restrict__ tval) {
  const int j = blockIdx.y;
  const MatDesc ad = adesc[j];
  const int a = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= ad.m) return;
  const MatDesc sd = sdesc[j];
  const int nd = nD[j];
  const int nt = ad.m - nd;  // nD + nP
  const int *P = tptr + tptr_off[j];
  const T *S = sbase + sd.off;
  T *arow = abase + ad.off + (long long)a * ad.ld;
  const int pa0 = a < nt ? P[a] : 0, pa1 = a < nt ? P[a + 1] : 0;
  for (int b = lane; b <= a; b += 32) {
    T v = T(0);
    if (a < nt && b < nt) {
      const int pb0 = P[b], pb1 = P[b + 1];
      for (int p = pa0; p < pa1; ++p) {
        const T *srow = S + (long long)trow[p] * sd.ld;
        T acc = T(0);
        for (int q = pb0; q < pb1; ++q) acc += tval[q] * srow[trow[q]];
        v += tval[p] * acc;
      }
    } else if (a >= nt && b < nd) {
      v = (a - nt == b) ? T(1) : T(0);
    }
    arow[b] = v;
  }
}

// ---- deluxe class inverses: AugC = [[sum_j S_C^(j), I], [I, 0]] ---------------
template <typename T>
__global__ void k_class_aug(const ClassTask *__restrict__ cls, const PairTask *__restrict__ pairs,
                            const T *__restrict__ blk, const MatDesc *__restrict__ cdesc, T *__restrict__ cbase) {
  const ClassTask c = cls[blockIdx.y];
  const MatDesc d = cdesc[blockIdx.y];
  const int n = c.n, m = 2 * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * m; t += gridDim.x * blockDim.x) {
    const int a = t / m, b = t % m;
    T v = T(0);
    if (a < n && b < n) {
      for (int p = c.pair_beg; p < c.pair_end; ++p) v += blk[pairs[p].blk_off + (long long)a * n + b];
    } else if (a >= n && b < n) {
      v = (a - n == b) ? T(1) : T(0);
    } else if (b >= n && a < n) {
      v = (b - n == a) ? T(1) : T(0);
    }
    cbase[d.off + (long long)a * d.ld + b] = v;
  }
}

// ---- coarse matrix S_PP = sum_j R_P^T S_PP^(j) R_P (Section 4.4) ---------------
// One thread per stored entry e of the sparse pattern of S_PP (CSR, row crow[e],
// column ccol[e]): the listed local entries are summed in FP64 in a fixed order
// into val64[e]; the gauge row and column become a unit row and column.  The same
// value goes into the dense augmented matrix AugCo = [[S_PP, I], [I, 0]] (in the
// local precision, zeroed beforehand) whose partial Cholesky gives the explicit
// inverse; threads e >= nnz write the two identity blocks.
template <typename T>
__global__ void k_coarse_assemble(int nnz, int np, int gauge, const int *__restrict__ crow,
                                  const int *__restrict__ ccol, const int *__restrict__ sptr,
                                  const long long *__restrict__ src, const T *__restrict__ abase,
                                  double *__restrict__ val64, T *__restrict__ co, int ld, double *__restrict__ dense64) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnz) {
    const int a = crow[e], b = ccol[e];
    double v = 0.0;
    if (a == gauge || b == gauge) v = (a == b) ? 1.0 : 0.0;
    else
      for (int k = sptr[e]; k < sptr[e + 1]; ++k) v += (double)abase[src[k]];
    val64[e] = v;
    co[(long long)a * ld + b] = (T)v;
    if (dense64) dense64[(long long)a * np + b] = v;
  } else if (e < nnz + np) {
    const int q = e - nnz;
    co[(long long)(np + q) * ld + q] = T(1);
    co[(long long)q * ld + np + q] = T(1);
  }
}

// ---- coarse right-hand side c = rP - sum_j (Psi^T r_D)_j, c[gauge] = 0 ------------
// rP is a vector, a sparse product (rPc.ptr set) or absent; yprim holds the local
// products Psi^T r_D, assembled through the lists (pl_ptr, pl_idx) in a fixed order.
__device__ __forceinline__ double coarse_rhs_row(int q, int gauge, const int *__restrict__ pl_ptr,
                                                 const int *__restrict__ pl_idx, const double *__restrict__ yprim,
                                                 const double *__restrict__ rP, const CsrIn &rPc) {
  double acc = 0.0;
  for (int k = pl_ptr[q]; k < pl_ptr[q + 1]; ++k) acc += yprim[pl_idx[k]];
  double v = -acc;
  if (rP) v += rP[q];
  else if (rPc.ptr) v += csr_row(rPc, q);
  return q == gauge ? 0.0 : v;
}

__global__ void k_coarse_rhs(int np, int gauge, const int *__restrict__ pl_ptr, const int *__restrict__ pl_idx,
                             const double *__restrict__ yprim, const double *__restrict__ rP, const CsrIn rPc,
                             double *__restrict__ c, const int *__restrict__ done) {
  if (done && *done) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < np) c[q] = coarse_rhs_row(q, gauge, pl_ptr, pl_idx, yprim, rP, rPc);
}

// rho = c - S_PP z (FP64 CSR), one warp per row (coarse rows hold a few hundred entries)
__global__ void k_coarse_resid(int np, const int *__restrict__ ptr, const int *__restrict__ col,
                               const double *__restrict__ val, const double *__restrict__ c,
                               const double *__restrict__ z, double *__restrict__ rho, const int *__restrict__ done) {
  if (done && *done) return;
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (q >= np) return;
  double acc = 0.0;
  for (int k = ptr[q] + lane; k < ptr[q + 1]; k += 32) acc += val[k] * z[col[k]];
  acc = warp_sum(acc);
  if (lane == 0) rho[q] = c[q] - acc;
}

// C = alpha A B + beta D for n x n FP64 matrices (row-major, leading dimension n): the
// Newton-Schulz refinement of small coarse inverses.  16 x 16 output tiles in shared memory.
__global__ void __launch_bounds__(256) k_gemm64(int n, const double *__restrict__ A, const double *__restrict__ B,
                                                const double *__restrict__ D, double alpha, double beta,
                                                double *__restrict__ C) {
  __shared__ double As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 16) {
    As[ty][tx] = (i < n && k0 + tx < n) ? A[(long long)i * n + k0 + tx] : 0.0;
    Bs[ty][tx] = (k0 + ty < n && j < n) ? B[(long long)(k0 + ty) * n + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc += As[ty][k] * Bs[k][tx];
    __syncthreads();
  }
  if (i < n && j < n) C[(long long)i * n + j] = alpha * acc + (D ? beta * D[(long long)i * n + j] : 0.0);
}

// y (np x np, leading dimension np) = (double) x (leading dimension ldx)
template <typename T>
__global__ void k_widen(int np, int ldx, const T *__restrict__ x, double *__restrict__ y) {
  const long long n = (long long)np * np;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = (double)x[(t / np) * ldx + t % np];
}

// Small coarse problems (np <= kCoarseSmall), once per Jacobian: the inverse in the local
// precision widened to FP64 and brought to FP64 accuracy by two Newton-Schulz steps
// X <- 2X - X C X (the error squares at each step), C the dense FP64 S_PP.
template <typename T>
void coarse_refine64(int np, const T *x0, int ld0, const double *C, double *X, double *W, double *Y, cudaStream_t s) {
  if (np == 0) return;
  const long long nn = (long long)np * np;
  k_widen<T><<<(int)std::min<long long>((nn + 255) / 256, 4096), 256, 0, s>>>(np, ld0, x0, X);
  const dim3 g(ceil_div(np, 16), ceil_div(np, 16));
  for (int it = 0; it < 2; ++it) {
    k_gemm64<<<g, 256, 0, s>>>(np, C, X, nullptr, 1.0, 0.0, W);  // W = C X
    k_gemm64<<<g, 256, 0, s>>>(np, X, W, X, -1.0, 2.0, Y);       // Y = 2X - X W
    cudaMemcpyAsync(X, Y, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s);
  }
  count_launch(5);
}

// The whole coarse solve of a small coarse problem in one CTA: c (as k_coarse_rhs),
// z = X c with the FP64 explicit inverse X, then nref steps of iterative refinement
// z += X (c - S_PP z) with the FP64 sparse S_PP.  The refinement makes the solve
// backward stable (the explicit inverse alone is not: its error grows with cond(S_PP)
// times the size of X, and the (u_i, u_e) constant mode that the gauge alone holds is
// where it shows).
__global__ void __launch_bounds__(1024) k_coarse_solve_small(
    int np, int gauge, const int *__restrict__ pl_ptr, const int *__restrict__ pl_idx,
    const double *__restrict__ yprim, const double *__restrict__ rP, const CsrIn rPc, const double *__restrict__ X,
    const int *__restrict__ sptr, const int *__restrict__ scol, const double *__restrict__ sval, int nref,
    double *__restrict__ z_out, const int *__restrict__ done) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *c = reinterpret_cast<double *>(smem_raw);
  double *z = c + np;
  double *r = z + np;
  for (int q = threadIdx.x; q < np; q += blockDim.x) {
    c[q] = coarse_rhs_row(q, gauge, pl_ptr, pl_idx, yprim, rP, rPc);
    r[q] = c[q];
    z[q] = 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int pass = 0; pass <= nref; ++pass) {
    // z += X r (r = c on the first pass)
    for (int q = wid; q < np; q += nw) {
      const double *row = X + (long long)q * np;
      double a0 = 0.0, a1 = 0.0;
      int k = lane;
      for (; k + 32 < np; k += 64) {
        a0 += row[k] * r[k];
        a1 += row[k + 32] * r[k + 32];
      }
      if (k < np) a0 += row[k] * r[k];
      const double v = warp_sum(a0 + a1);
      if (lane == 0) z[q] += v;
    }
    __syncthreads();
    if (pass == nref) break;
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
      double acc = 0.0;
      for (int k = sptr[q]; k < sptr[q + 1]; ++k) acc += sval[k] * z[scol[k]];
      r[q] = c[q] - acc;
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < np; q += blockDim.x) z_out[q] = z[q];
}

// ---- rho-scaling (Section 4.2) --------------------------------------------------
// The deluxe kernels form D_C^(j) = Sinv_C Blk_C^(j); writing Sinv_C = diag(1 / sum_k
// sigma_M^(k)) and Blk_C^(j) = diag(sigma_M^(j)) (field i on even, e on odd dual dofs)
// turns every one of them into the rho-scaling weights, with no other change.  The
// conductivities are equal in every subdomain, so the weights are 1 / |N_C|.  One CTA
// per class.
template <typename T>
__global__ void k_rho_blocks(const ClassTask *__restrict__ cls, const PairTask *__restrict__ pairs, double sig_i,
                             double sig_e, T *__restrict__ sinv, T *__restrict__ blk) {
  const ClassTask c = cls[blockIdx.x];
  const int n = c.n, k = c.pair_end - c.pair_beg;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int a = t / n, b = t % n;
    const double sm = (a % 2 == 0) ? sig_i : sig_e;
    sinv[c.sinv_off + t] = (a == b) ? (T)(1.0 / (k * sm)) : T(0);
    for (int q = c.pair_beg; q < c.pair_end; ++q) blk[pairs[q].blk_off + t] = (a == b) ? (T)sm : T(0);
  }
}
template <typename T>
void launch_rho_blocks(int ncls, const ClassTask *cls, const PairTask *pairs, double sig_i, double sig_e, T *sinv,
                       T *blk, cudaStream_t s) {
  if (ncls == 0) return;
  k_rho_blocks<T><<<ncls, 256, 0, s>>>(cls, pairs, sig_i, sig_e, sinv, blk);
  count_launch();
}

// ---- sparse (CSR) matrix-vector product y = A x, y[zero] = 0 --------------------
__global__ void k_spmv(int n, const int *__restrict__ ptr, const int *__restrict__ col, const double *__restrict__ val,
                       const double *__restrict__ x, double *__restrict__ y, int zero, const int *__restrict__ done) {
  if (done && *done) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double acc = 0.0;
  for (int k = ptr[r]; k < ptr[r + 1]; ++k) acc += val[k] * x[col[k]];
  y[r] = (r == zero) ? 0.0 : acc;
}

// y[g] = sum of the listed local values (interface assembly R^T), y[zero] = 0.
// The addend may instead be a sparse product evaluated on the fly (add_csr.ptr set).
__global__ void k_gather_sum(int n, const int *__restrict__ ptr, const int *__restrict__ idx,
                             const double *__restrict__ src, double *__restrict__ y, int zero, double alpha,
                             const double *__restrict__ addend, const int *__restrict__ done, const CsrIn add_csr) {
  if (done && *done) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double acc = 0.0;
  for (int k = ptr[r]; k < ptr[r + 1]; ++k) acc += src[idx[k]];
  double v = alpha * acc;
  if (addend) v += addend[r];
  else if (add_csr.ptr) v += csr_row(add_csr, r);
  y[r] = (r == zero) ? 0.0 : v;
}

// ---- batched small GEMM C = A B (deluxe D_C^(j) = (sum S)^-1 S_C^(j)) ----------
// 32x32 output tiles, 256 threads (2x2 per thread), K in chunks of 32.
template <typename T>
__global__ void __launch_bounds__(256) k_small_gemm(const GemmTask *__restrict__ tasks, const T *__restrict__ A,
                                                    const T *__restrict__ B, T *__restrict__ C) {
  const GemmTask t = tasks[blockIdx.y];
  const int nt = ceil_div(t.n, 32);
  if ((int)blockIdx.x >= nt * nt) return;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  __shared__ T As[32][33], Bs[32][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
  for (int k0 = 0; k0 < t.n; k0 += 32) {
    for (int q = threadIdx.x; q < 32 * 32; q += 256) {
      const int i = q >> 5, k = q & 31;
      const int ra = ti * 32 + i, ca = k0 + k;
      As[i][k] = (ra < t.n && ca < t.n) ? A[t.a_off + (long long)ra * t.n + ca] : T(0);
      const int rb = k0 + i, cb = tj * 32 + k;
      Bs[i][k] = (rb < t.n && cb < t.n) ? B[t.b_off + (long long)rb * t.n + cb] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const T a0 = As[ty][k], a1 = As[ty + 16][k];
      const T b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
      acc[0][0] += a0 * b0; acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int r = ti * 32 + ty + 16 * i, c = tj * 32 + tx + 16 * j;
      if (r < t.n && c < t.n) C[t.c_off + (long long)r * t.ldc + c] = acc[i][j];
    }
}

// ---- small dense matvec in shared memory (FETI-DP scaled jumps) --------------
template <typename T>
__device__ inline void smem_gemv(const T *__restrict__ A, int n, const T *__restrict__ x, T *__restrict__ y) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int u = wid; u < n; u += nw) {
    T acc = T(0);
    for (int v = lane; v < n; v += 32) acc += A[(long long)u * n + v] * x[v];
    acc = warp_sum(acc);
    if (lane == 0) y[u] = acc;
  }
}

// ---- FETI-DP jump operators (Section 4.3) ---------------------------------------
// B w: lambda_ab = w_a - w_b on the class block.
__global__ void k_jump(const LamTask *__restrict__ lt, const PairTask *__restrict__ pairs, const double *__restrict__ w,
                       double *__restrict__ lam, const int *__restrict__ done) {
  if (done && *done) return;
  const LamTask t = lt[blockIdx.y];
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= t.n) return;
  lam[t.lam_off + u] = w[pairs[t.pa].ldual_off + u] - w[pairs[t.pb].ldual_off + u];
}

// B^T lambda: w_(j,C) = sum of +-lambda over the multipliers touching (j, C).
__global__ void k_jump_t(const WTask *__restrict__ wt, const WEnt *__restrict__ ent, const double *__restrict__ lam,
                         double *__restrict__ w, const int *__restrict__ done) {
  if (done && *done) return;
  const WTask t = wt[blockIdx.y];
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= t.n) return;
  double acc = 0.0;
  for (int k = t.ent_beg; k < t.ent_end; ++k) acc += ent[k].sign * lam[ent[k].lam_off + u];
  w[t.ldual_off + u] = acc;
}

// B_D^T mu: w_(j,C) = (sum S)^-1 sum_{pairs} +-S_C^(partner) mu_pair.
template <typename T>
__global__ void k_jump_dt(const WTask *__restrict__ wt, const WEnt *__restrict__ ent, const T *__restrict__ blk,
                          const T *__restrict__ sinv, const double *__restrict__ mu, double *__restrict__ w,
                          const int *__restrict__ done) {
  if (done && *done) return;
  const WTask t = wt[blockIdx.x];
  extern __shared__ unsigned char smem_raw[];
  T *acc = reinterpret_cast<T *>(smem_raw);
  T *mm = acc + t.n;
  T *tmp = mm + t.n;
  for (int u = threadIdx.x; u < t.n; u += blockDim.x) acc[u] = T(0);
  __syncthreads();
  for (int k = t.ent_beg; k < t.ent_end; ++k) {
    const WEnt e = ent[k];
    for (int u = threadIdx.x; u < t.n; u += blockDim.x) mm[u] = (T)mu[e.lam_off + u];
    __syncthreads();
    smem_gemv(blk + e.partner_blk_off, t.n, mm, tmp);
    __syncthreads();
    for (int u = threadIdx.x; u < t.n; u += blockDim.x) acc[u] += (e.sign > 0 ? tmp[u] : -tmp[u]);
    __syncthreads();
  }
  smem_gemv(sinv + t.sinv_off, t.n, acc, tmp);
  __syncthreads();
  for (int u = threadIdx.x; u < t.n; u += blockDim.x) w[t.ldual_off + u] = (double)tmp[u];
}

// B_D y: mu_ab = S_C^(b) (sum S)^-1 y_a - S_C^(a) (sum S)^-1 y_b.
template <typename T>
__global__ void k_jump_d(const LamTask *__restrict__ lt, const PairTask *__restrict__ pairs, const T *__restrict__ blk,
                         const T *__restrict__ sinv, const double *__restrict__ y, double *__restrict__ mu,
                         const int *__restrict__ done) {
  if (done && *done) return;
  const LamTask t = lt[blockIdx.x];
  extern __shared__ unsigned char smem_raw[];
  T *ya = reinterpret_cast<T *>(smem_raw);
  T *yb = ya + t.n;
  T *ta = yb + t.n;
  T *tb = ta + t.n;
  T *oa = tb + t.n;
  T *ob = oa + t.n;
  const PairTask pa = pairs[t.pa], pb = pairs[t.pb];
  for (int u = threadIdx.x; u < t.n; u += blockDim.x) {
    ya[u] = (T)y[pa.ldual_off + u];
    yb[u] = (T)y[pb.ldual_off + u];
  }
  __syncthreads();
  smem_gemv(sinv + t.sinv_off, t.n, ya, ta);
  smem_gemv(sinv + t.sinv_off, t.n, yb, tb);
  __syncthreads();
  smem_gemv(blk + pb.blk_off, t.n, ta, oa);
  smem_gemv(blk + pa.blk_off, t.n, tb, ob);
  __syncthreads();
  for (int u = threadIdx.x; u < t.n; u += blockDim.x) mu[t.lam_off + u] = (double)oa[u] - (double)ob[u];
}

// Mean over the subdomains sharing each global dual dof (FETI-DP recovery).
__global__ void k_dual_mean(const ClassTask *__restrict__ cls, const PairTask *__restrict__ pairs,
                            const double *__restrict__ zD, double *__restrict__ zbar) {
  const ClassTask c = cls[blockIdx.y];
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= c.n) return;
  double acc = 0.0;
  for (int p = c.pair_beg; p < c.pair_end; ++p) acc += zD[pairs[p].ldual_off + u];
  zbar[c.dual_start + u] = acc / (double)(c.pair_end - c.pair_beg);
}

// ---- vector helpers ------------------------------------------------------------
// Local interior vector of every subdomain from a global SoA pair (f_i, f_e):
// v[off_j + 2a + f] = f_f[node of interior node a].
__global__ void k_gather_pairs(int n, const int *__restrict__ node, const double *__restrict__ fi,
                               const double *__restrict__ fe, double *__restrict__ v, double scale,
                               const double *__restrict__ mult) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int x = node[t];
  const double sc = mult ? scale / mult[t] : scale;
  v[2 * t] = sc * fi[x];
  v[2 * t + 1] = sc * fe[x];
}

// Global SoA pair from a nodal-interleaved vector: s_f[node[t]] = v[2t + f].
__global__ void k_scatter_pairs(int n, const int *__restrict__ node, const double *__restrict__ v,
                                double *__restrict__ si, double *__restrict__ se) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int x = node[t];
  si[x] = v[2 * t];
  se[x] = v[2 * t + 1];
}

// Local transformed vector gbar_j = T_loc^T g_j (CSC of T_loc by transformed
// dof, flattened over subdomains); dual entries go to outD (local dual layout),
// primal entries to outP (local primal layout).
__global__ void k_tloc_t(int nt_total, const int *__restrict__ t_sub, const int *__restrict__ t_loc,
                         const int *__restrict__ t_ptr, const int *__restrict__ t_row, const double *__restrict__ t_val,
                         const int *__restrict__ g_off, const double *__restrict__ g, const int *__restrict__ nD,
                         const int *__restrict__ ldual_off, const int *__restrict__ lprim_off,
                         double *__restrict__ outD, double *__restrict__ outP) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt_total) return;
  const int j = t_sub[t], a = t_loc[t];
  double acc = 0.0;
  for (int k = t_ptr[t]; k < t_ptr[t + 1]; ++k) acc += t_val[k] * g[g_off[j] + t_row[k]];
  if (a < nD[j]) outD[ldual_off[j] + a] = acc;
  else outP[lprim_off[j] + a - nD[j]] = acc;
}

// y[t] = x[idx[t]] * w[idx[t]] - y[t]
__global__ void k_gather_scale_sub(int n, const int *__restrict__ idx, const double *__restrict__ x,
                                   const double *__restrict__ w, double *__restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int g = idx[t];
  y[t] = x[g] * w[g] - y[t];
}

__global__ void k_fill(int n, double *__restrict__ y, double v) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = v;
}

__global__ void k_copy_vec(int n, const double *__restrict__ x, double *__restrict__ y, const int *__restrict__ done) {
  if (done && *done) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = x[t];
}

// y = a x + b y with scalars a, b (device doubles, optional)
__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b, double *__restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = a * x[t] + b * y[t];
}

// ---- PCG recurrences (device scalars, early exit once converged) ---------------
__global__ void k_pcg_start(KrylovState *__restrict__ ks, const double *__restrict__ dots) {
  ks->rz = dots[0];
  ks->zn0 = sqrt(fmax(dots[1], 0.0));
  ks->zn = ks->zn0;
  ks->tol = fmax(ks->rtol * ks->zn0, ks->atol);
  ks->it = 0;
  ks->reason = 0;
  ks->done = (ks->zn0 <= ks->atol) ? 1 : 0;
  if (!isfinite(ks->zn0)) { ks->done = 1; ks->reason = -6; }
}

__global__ void k_pcg_alpha(KrylovState *__restrict__ ks, const double *__restrict__ dots, double *__restrict__ hist_a) {
  if (ks->done) return;
  const double pq = dots[0];
  ks->alpha = ks->rz / pq;
  if (ks->it < ks->hist_cap) hist_a[ks->it] = ks->alpha;
}

__global__ void k_pcg_xr(int n, const KrylovState *__restrict__ ks, const double *__restrict__ p,
                         const double *__restrict__ q, double *__restrict__ x, double *__restrict__ r) {
  if (ks->done) return;
  const double a = ks->alpha;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    x[t] += a * p[t];
    r[t] -= a * q[t];
  }
}

__global__ void k_pcg_beta(KrylovState *__restrict__ ks, const double *__restrict__ dots, double *__restrict__ hist_b) {
  if (ks->done) return;
  ks->it += 1;
  const double zn = sqrt(fmax(dots[1], 0.0));
  ks->zn = zn;
  if (!isfinite(zn)) { ks->done = 1; ks->reason = -6; return; }
  if (zn <= ks->tol) { ks->done = 1; ks->reason = 0; return; }
  if (zn > ks->dtol * ks->zn0) { ks->done = 1; ks->reason = -4; return; }
  if (ks->it >= ks->maxit) { ks->done = 1; ks->reason = -3; return; }
  ks->beta = dots[0] / ks->rz;
  if (ks->it - 1 < ks->hist_cap) hist_b[ks->it - 1] = ks->beta;
  ks->rz = dots[0];
}

__global__ void k_pcg_p(int n, const KrylovState *__restrict__ ks, const double *__restrict__ z, double *__restrict__ p) {
  if (ks->done) return;
  const double b = ks->beta;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) p[t] = z[t] + b * p[t];
}

// Fused PCG reductions: every block writes its partial sums; the last block to
// finish (counter) adds the partials in block order (deterministic) and applies
// the scalar recurrence.  which = 0: s0 = p.q -> alpha; which = 1: s0 = r.z,
// s1 = z.z -> beta and the convergence test.  Every thread of the block calls it.
__device__ void pcg_dot_tail(int which, double s0, double s1, double *__restrict__ partial,
                             unsigned int *__restrict__ counter, KrylovState *__restrict__ ks,
                             double *__restrict__ hist) {
  __shared__ double sh[32];
  __shared__ bool last;
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t0 = 0.0, t1 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    t0 += ((volatile double *)partial)[2 * b];
    t1 += ((volatile double *)partial)[2 * b + 1];
  }
  t0 = block_sum(t0, sh);
  t1 = block_sum(t1, sh);
  if (threadIdx.x != 0) return;
  *counter = 0u;
  if (which == 0) {
    ks->alpha = ks->rz / t0;
    if (ks->it < ks->hist_cap) hist[ks->it] = ks->alpha;
    return;
  }
  ks->it += 1;
  const double zn = sqrt(fmax(t1, 0.0));
  ks->zn = zn;
  if (!isfinite(zn)) { ks->done = 1; ks->reason = -6; return; }
  if (zn <= ks->tol) { ks->done = 1; ks->reason = 0; return; }
  if (zn > ks->dtol * ks->zn0) { ks->done = 1; ks->reason = -4; return; }
  if (ks->it >= ks->maxit) { ks->done = 1; ks->reason = -3; return; }
  ks->beta = t0 / ks->rz;
  if (ks->it - 1 < ks->hist_cap) hist[ks->hist_cap + ks->it - 1] = ks->beta;
  ks->rz = t0;
}

__global__ void k_pcg_dot_step(int n, int which, const double *__restrict__ a0, const double *__restrict__ b0,
                               const double *__restrict__ a1, const double *__restrict__ b1,
                               double *__restrict__ partial, unsigned int *__restrict__ counter,
                               KrylovState *__restrict__ ks, double *__restrict__ hist) {
  if (ks->done) return;
  double s0 = 0.0, s1 = 0.0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    s0 += a0[x] * b0[x];
    if (a1) s1 += a1[x] * b1[x];
  }
  pcg_dot_tail(which, s0, s1, partial, counter, ks, hist);
}

// y = interface assembly (as k_gather_sum, alpha = 1, no addend) fused with the PCG
// reduction of the operator output: s0 = a.y (and s1 = y.y when which = 1).
__global__ void k_gather_sum_dot(int n, const int *__restrict__ ptr, const int *__restrict__ idx,
                                 const double *__restrict__ src, double *__restrict__ y, int zero, DotFuse f) {
  if (f.ks->done) return;
  double s0 = 0.0, s1 = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = ptr[r]; k < ptr[r + 1]; ++k) acc += src[idx[k]];
    const double v = (r == zero) ? 0.0 : acc;
    y[r] = v;
    s0 += f.a[r] * v;
    s1 += v * v;
  }
  pcg_dot_tail(f.which, s0, f.which ? s1 : 0.0, f.partial, f.counter, f.ks, f.hist);
}

// y = A x (CSR, as k_spmv) fused with the PCG reduction of the output.
__global__ void k_spmv_dot(int n, const int *__restrict__ ptr, const int *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
                           int zero, DotFuse f) {
  if (f.ks->done) return;
  double s0 = 0.0, s1 = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = ptr[r]; k < ptr[r + 1]; ++k) acc += val[k] * x[col[k]];
    const double v = (r == zero) ? 0.0 : acc;
    y[r] = v;
    s0 += f.a[r] * v;
    s1 += v * v;
  }
  pcg_dot_tail(f.which, s0, f.which ? s1 : 0.0, f.partial, f.counter, f.ks, f.hist);
}

// dots with an early exit (Krylov loop): partial sums then a fixed-order finalize
__global__ void k_dot2_done(int n, const double *__restrict__ a0, const double *__restrict__ b0,
                            const double *__restrict__ a1, const double *__restrict__ b1,
                            double *__restrict__ partial, const int *__restrict__ done) {
  if (done && *done) return;
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    s0 += a0[x] * b0[x];
    if (a1) s1 += a1[x] * b1[x];
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

__global__ void k_finalize2_done(int nblk, const double *__restrict__ partial, double *__restrict__ out,
                                 const int *__restrict__ done) {
  if (done && *done) return;
  __shared__ double sh[32];
  for (int c = 0; c < 2; ++c) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += partial[2 * b + c];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[c] = v;
  }
}

// ---- launchers -------------------------------------------------------------------
#define GRID1(n) ceil_div((n), 256), 256, 0, s

template <typename T>
void launch_assemble_local(int nq, const int *q_sub, const int *q_loc, const int *q_node, const int *nbr,
                           const double *stencil, const double *mass, const double *factor, double tau,
                           const MatDesc *desc, T *base, cudaStream_t s) {
  const long long tot = (long long)nq * 27;
  k_assemble_local<T><<<(int)((tot + 255) / 256), 256, 0, s>>>(nq, q_sub, q_loc, q_node, nbr, stencil, mass, factor,
                                                             tau, desc, base);
  count_launch();
}

template <typename TS, typename TD>
void launch_copy(int ntasks, long long max_elems, const CopyTask *tasks, const TS *src, TD *dst, cudaStream_t s) {
  if (ntasks == 0 || max_elems == 0) return;
  const int gx = (int)std::min<long long>((max_elems + 1023) / 1024, 4096);
  k_copy<TS, TD><<<dim3(gx, ntasks), 256, 0, s>>>(tasks, src, dst);
  count_launch();
}

template <typename T>
void launch_build_aug(int nsub, int max_m, const MatDesc *sdesc, const T *sbase, const MatDesc *adesc,
                      T *abase, const int *nD, const int *tptr_off, const int *tptr, const int *trow,
                      const T *tval, cudaStream_t s) {
  const int gx = ceil_div(max_m, 8);
  k_build_aug<T><<<dim3(gx, nsub), 256, 0, s>>>(sdesc, sbase, adesc, abase, nD, tptr_off, tptr, trow, tval);
  count_launch();
}

template <typename T>
void launch_class_aug(int ncls, int max_n, const ClassTask *cls, const PairTask *pairs, const T *blk,
                      const MatDesc *cdesc, T *cbase, cudaStream_t s) {
  if (ncls == 0) return;
  const int gx = std::max(1, std::min(ceil_div(4 * max_n * max_n, 256), 1024));
  k_class_aug<T><<<dim3(gx, ncls), 256, 0, s>>>(cls, pairs, blk, cdesc, cbase);
  count_launch();
}

template <typename T>
void launch_coarse_assemble(int nnz, int np, int gauge, const int *crow, const int *ccol, const int *sptr,
                            const long long *src, const T *abase, double *val64, T *co, int ld, double *dense64,
                            cudaStream_t s) {
  const int tot = nnz + np;
  if (tot == 0) return;
  k_coarse_assemble<T><<<ceil_div(tot, 256), 256, 0, s>>>(nnz, np, gauge, crow, ccol, sptr, src, abase, val64, co,
                                                          ld, dense64);
  count_launch();
}

template <typename T>
void launch_coarse_solve(const CoarseSolve &cs, const T *X, const double *yprim, const double *rP, const CsrIn *rPc,
                         double *z, double *c, double *rho, const int *done, cudaStream_t s) {
  if (cs.np == 0) return;
  const CsrIn rc = rPc ? *rPc : CsrIn{};
  if (cs.X64) {
    k_coarse_solve_small<<<1, 1024, 3 * sizeof(double) * cs.np, s>>>(
        cs.np, cs.gauge, cs.pl_ptr, cs.pl_idx, yprim, rP, rc, cs.X64, cs.sptr, cs.scol, cs.sval, cs.nref, z, done);
    count_launch();
    return;
  }
  k_coarse_rhs<<<ceil_div(cs.np, 256), 256, 0, s>>>(cs.np, cs.gauge, cs.pl_ptr, cs.pl_idx, yprim, rP, rc, c, done);
  count_launch();
  launch_symv_rows<T>(cs.np, X, cs.ld_x, c, z, 0, done, s);
  for (int it = 0; it < cs.nref; ++it) {
    k_coarse_resid<<<ceil_div(cs.np, 8), 256, 0, s>>>(cs.np, cs.sptr, cs.scol, cs.sval, c, z, rho, done);
    count_launch();
    launch_symv_rows<T>(cs.np, X, cs.ld_x, rho, z, 1, done, s);
  }
}

template <typename T>
void launch_small_gemm(int ntasks, int max_n, const GemmTask *tasks, const T *A, const T *B, T *C, cudaStream_t s) {
  if (ntasks == 0) return;
  const int nt = ceil_div(max_n, 32);
  k_small_gemm<T><<<dim3(nt * nt, ntasks), 256, 0, s>>>(tasks, A, B, C);
  count_launch();
}

void launch_gather_sum_dot(int n, const int *ptr, const int *idx, const double *src, double *y, int zero,
                           const DotFuse &f, cudaStream_t s) {
  if (n == 0) return;
  k_gather_sum_dot<<<std::min(ceil_div(n, 256), kRedBlocks), 256, 0, s>>>(n, ptr, idx, src, y, zero, f);
  count_launch();
}
void launch_spmv_dot(int n, const int *ptr, const int *col, const double *val, const double *x, double *y, int zero,
                     const DotFuse &f, cudaStream_t s) {
  if (n == 0) return;
  k_spmv_dot<<<std::min(ceil_div(n, 256), kRedBlocks), 256, 0, s>>>(n, ptr, col, val, x, y, zero, f);
  count_launch();
}
void launch_spmv(int n, const int *ptr, const int *col, const double *val, const double *x, double *y, int zero,
                 const int *done, cudaStream_t s) {
  if (n == 0) return;
  k_spmv<<<GRID1(n)>>>(n, ptr, col, val, x, y, zero, done);
  count_launch();
}

void launch_gather_sum(int n, const int *ptr, const int *idx, const double *src, double *y, int zero, double alpha,
                       const double *addend, const int *done, cudaStream_t s, const CsrIn *add_csr) {
  if (n == 0) return;
  k_gather_sum<<<GRID1(n)>>>(n, ptr, idx, src, y, zero, alpha, addend, done, add_csr ? *add_csr : CsrIn{});
  count_launch();
}

void launch_jump(int nlt, int max_n, const LamTask *lt, const PairTask *pairs, const double *w, double *lam,
                 const int *done, cudaStream_t s) {
  if (nlt == 0) return;
  k_jump<<<dim3(ceil_div(max_n, 128), nlt), 128, 0, s>>>(lt, pairs, w, lam, done);
  count_launch();
}

void launch_jump_t(int nwt, int max_n, const WTask *wt, const WEnt *ent, const double *lam, double *w,
                   const int *done, cudaStream_t s) {
  if (nwt == 0) return;
  k_jump_t<<<dim3(ceil_div(max_n, 128), nwt), 128, 0, s>>>(wt, ent, lam, w, done);
  count_launch();
}

template <typename T>
void launch_jump_dt(int nwt, int max_n, const WTask *wt, const WEnt *ent, const T *blk, const T *sinv,
                    const double *mu, double *w, const int *done, cudaStream_t s) {
  if (nwt == 0) return;
  k_jump_dt<T><<<nwt, 256, 3 * sizeof(T) * max_n, s>>>(wt, ent, blk, sinv, mu, w, done);
  count_launch();
}

template <typename T>
void launch_jump_d(int nlt, int max_n, const LamTask *lt, const PairTask *pairs, const T *blk, const T *sinv,
                   const double *y, double *mu, const int *done, cudaStream_t s) {
  if (nlt == 0) return;
  k_jump_d<T><<<nlt, 256, 6 * sizeof(T) * max_n, s>>>(lt, pairs, blk, sinv, y, mu, done);
  count_launch();
}

void launch_dual_mean(int ncls, int max_n, const ClassTask *cls, const PairTask *pairs, const double *zD,
                      double *zbar, cudaStream_t s) {
  if (ncls == 0) return;
  k_dual_mean<<<dim3(ceil_div(max_n, 128), ncls), 128, 0, s>>>(cls, pairs, zD, zbar);
  count_launch();
}

void launch_gather_pairs(int n, const int *node, const double *fi, const double *fe, double *v, double scale,
                         const double *mult, cudaStream_t s) {
  if (n == 0) return;
  k_gather_pairs<<<GRID1(n)>>>(n, node, fi, fe, v, scale, mult);
  count_launch();
}

void launch_scatter_pairs(int n, const int *node, const double *v, double *si, double *se, cudaStream_t s) {
  if (n == 0) return;
  k_scatter_pairs<<<GRID1(n)>>>(n, node, v, si, se);
  count_launch();
}

void launch_tloc_t(int nt, const int *t_sub, const int *t_loc, const int *t_ptr, const int *t_row,
                   const double *t_val, const int *g_off, const double *g, const int *nD, const int *ldual_off,
                   const int *lprim_off, double *outD, double *outP, cudaStream_t s) {
  if (nt == 0) return;
  k_tloc_t<<<GRID1(nt)>>>(nt, t_sub, t_loc, t_ptr, t_row, t_val, g_off, g, nD, ldual_off, lprim_off, outD, outP);
  count_launch();
}

void launch_gather_scale_sub(int n, const int *idx, const double *x, const double *w, double *y, cudaStream_t s) {
  if (n == 0) return;
  k_gather_scale_sub<<<GRID1(n)>>>(n, idx, x, w, y);
  count_launch();
}

void launch_fill(int n, double *y, double v, cudaStream_t s) {
  if (n == 0) return;
  k_fill<<<GRID1(n)>>>(n, y, v);
  count_launch();
}

void launch_copy_vec(int n, const double *x, double *y, const int *done, cudaStream_t s) {
  if (n == 0) return;
  k_copy_vec<<<GRID1(n)>>>(n, x, y, done);
  count_launch();
}

void launch_axpby(int n, double a, const double *x, double b, double *y, cudaStream_t s) {
  if (n == 0) return;
  k_axpby<<<GRID1(n)>>>(n, a, x, b, y);
  count_launch();
}

void launch_pcg_start(KrylovState *ks, const double *dots, cudaStream_t s) {
  k_pcg_start<<<1, 1, 0, s>>>(ks, dots);
  count_launch();
}
void launch_pcg_alpha(KrylovState *ks, const double *dots, double *ha, cudaStream_t s) {
  k_pcg_alpha<<<1, 1, 0, s>>>(ks, dots, ha);
  count_launch();
}
void launch_pcg_beta(KrylovState *ks, const double *dots, double *hb, cudaStream_t s) {
  k_pcg_beta<<<1, 1, 0, s>>>(ks, dots, hb);
  count_launch();
}
void launch_pcg_xr(int n, const KrylovState *ks, const double *p, const double *q, double *x, double *r,
                   cudaStream_t s) {
  k_pcg_xr<<<std::max(1, std::min(ceil_div(n, 256), kRedBlocks)), 256, 0, s>>>(n, ks, p, q, x, r);
  count_launch();
}
void launch_pcg_p(int n, const KrylovState *ks, const double *z, double *p, cudaStream_t s) {
  k_pcg_p<<<std::max(1, std::min(ceil_div(n, 256), kRedBlocks)), 256, 0, s>>>(n, ks, z, p);
  count_launch();
}
void launch_pcg_dot_step(int n, int which, const double *a0, const double *b0, const double *a1, const double *b1,
                        double *partial, unsigned int *counter, KrylovState *ks, double *hist, cudaStream_t s) {
  k_pcg_dot_step<<<kRedBlocks, 256, 0, s>>>(n, which, a0, b0, a1, b1, partial, counter, ks, hist);
  count_launch();
}

void launch_dot2(int n, const double *a0, const double *b0, const double *a1, const double *b1, double *partial,
                 double *out, const int *done, cudaStream_t s) {
  k_dot2_done<<<kRedBlocks, 256, 0, s>>>(n, a0, b0, a1, b1, partial, done);
  count_launch();
  k_finalize2_done<<<1, 256, 0, s>>>(kRedBlocks, partial, out, done);
  count_launch();
}

#define BD_DD_INST(T)                                                                                           \
  template void launch_assemble_local<T>(int, const int *, const int *, const int *, const int *, const double *, \
                                         const double *, const double *, double, const MatDesc *, T *,         \
                                         cudaStream_t);                                                        \
  template void launch_build_aug<T>(int, int, const MatDesc *, const T *, const MatDesc *, T *, const int *,    \
                                    const int *, const int *, const int *, const T *, cudaStream_t);                                                             \
  template void launch_small_gemm<T>(int, int, const GemmTask *, const T *, const T *, T *, cudaStream_t);      \
  template void launch_class_aug<T>(int, int, const ClassTask *, const PairTask *, const T *, const MatDesc *,  \
                                    T *, cudaStream_t);                                                        \
  template void launch_coarse_assemble<T>(int, int, int, const int *, const int *, const int *,                 \
                                          const long long *, const T *, double *, T *, int, double *,         \
                                          cudaStream_t);                                                      \
  template void coarse_refine64<T>(int, const T *, int, const double *, double *, double *, double *,           \
                                   cudaStream_t);                                                              \
  template void launch_coarse_solve<T>(const CoarseSolve &, const T *, const double *, const double *,         \
                                       const CsrIn *, double *, double *, double *, const int *, cudaStream_t); \
  template void launch_jump_dt<T>(int, int, const WTask *, const WEnt *, const T *, const T *, const double *,  \
                                  double *, const int *, cudaStream_t);                                        \
  template void launch_jump_d<T>(int, int, const LamTask *, const PairTask *, const T *, const T *,             \
                                 const double *, double *, const int *, cudaStream_t);                         \
  template void launch_copy<T, T>(int, long long, const CopyTask *, const T *, T *, cudaStream_t);            \
  template void launch_rho_blocks<T>(int, const ClassTask *, const PairTask *, double, double, T *, T *,        \
                                     cudaStream_t);
BD_DD_INST(float)
BD_DD_INST(double)
template void launch_copy<float, double>(int, long long, const CopyTask *, const float *, double *, cudaStream_t);
template void launch_copy<double, float>(int, long long, const CopyTask *, const double *, float *, cudaStream_t);


// ---- GMRES(m), left preconditioned, CGS2 orthogonalisation ---------------------
// V holds m+1 basis vectors of length n (column q at V + q n).  All kernels of a
// step return at once when `stop` is set (converged, diverged or at maxit).
__global__ void k_multidot(int n, int k, const double *__restrict__ V, const double *__restrict__ z,
                           double *__restrict__ partial, const GmresState *__restrict__ gs) {
  if (gs->stop) return;
  __shared__ double sh[32];
  const int q = blockIdx.y;
  const double *v = V + (long long)q * n;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += v[i] * z[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[q * gridDim.x + blockIdx.x] = acc;
}

// h[q] (+)= sum of the partials of dot q, q < k (fixed order)
__global__ void k_multidot_fin(int k, int nblk, const double *__restrict__ partial, double *__restrict__ h, int add,
                               const GmresState *__restrict__ gs) {
  if (gs->stop) return;
  const int q = threadIdx.x;
  if (q >= k) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += partial[q * nblk + b];
  h[q] = add ? h[q] + acc : acc;
}

// z -= sum_q c[q] V_q  (c = the projections just computed)
__global__ void k_orth_sub(int n, int k, const double *__restrict__ V, const double *__restrict__ c,
                           double *__restrict__ z, const GmresState *__restrict__ gs) {
  if (gs->stop) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = z[i];
    for (int q = 0; q < k; ++q) acc -= c[q] * V[(long long)q * n + i];
    z[i] = acc;
  }
}

// column j of H from (h1 + h2, ||z||), Givens rotations, residual estimate, stop test
__global__ void k_gmres_rot(GmresState *__restrict__ gs, const double *__restrict__ h1, const double *__restrict__ h2,
                            const double *__restrict__ zz, int j) {
  if (gs->stop) return;
  const int m = gs->restart;
  double *H = gs->H;
  for (int i = 0; i <= j; ++i) H[i * m + j] = h1[i] + h2[i];
  const double hn = sqrt(fmax(zz[0], 0.0));
  H[(j + 1) * m + j] = hn;
  gs->hn = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], b = H[(i + 1) * m + j];
    H[i * m + j] = gs->cs[i] * a + gs->sn[i] * b;
    H[(i + 1) * m + j] = -gs->sn[i] * a + gs->cs[i] * b;
  }
  const double a = H[j * m + j], b = H[(j + 1) * m + j];
  const double den = hypot(a, b);
  gs->cs[j] = a / den;
  gs->sn[j] = b / den;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  gs->g[j + 1] = -gs->sn[j] * gs->g[j];
  gs->g[j] = gs->cs[j] * gs->g[j];
  gs->its += 1;
  gs->j = j + 1;
  const double res = fabs(gs->g[j + 1]);
  gs->res = res;
  if (!isfinite(res)) { gs->stop = 1; gs->reason = -6; return; }
  if (res <= gs->tol) { gs->stop = 1; gs->converged = 1; gs->reason = 0; return; }
  if (res > gs->dtol * gs->res0) { gs->stop = 1; gs->reason = -4; return; }
  if (gs->its >= gs->maxit) { gs->stop = 1; gs->reason = -3; return; }
  if (gs->j >= m) gs->stop = 1;  // end of the cycle
}

// V_{j+1} = z / ||z|| (also V_0 = r / beta at a cycle start).  Vectors written after a
// stop are never read: the update uses only the first gs->j basis vectors.
__global__ void k_gmres_scale(int n, const double *__restrict__ z, double *__restrict__ vout,
                              const GmresState *__restrict__ gs) {
  const double inv = gs->hn > 0.0 ? 1.0 / gs->hn : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) vout[i] = z[i] * inv;
}

// end of a cycle: y = H^-1 g over the steps done, x += V y
__global__ void k_gmres_solve_y(GmresState *__restrict__ gs) {
  const int m = gs->restart, k = gs->j;
  for (int i = k - 1; i >= 0; --i) {
    double v = gs->g[i];
    for (int q = i + 1; q < k; ++q) v -= gs->H[i * m + q] * gs->y[q];
    gs->y[i] = v / gs->H[i * m + i];
  }
}

__global__ void k_gmres_update_x(int n, const double *__restrict__ V, double *__restrict__ x,
                                 const GmresState *__restrict__ gs) {
  const int k = gs->j;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int q = 0; q < k; ++q) acc += gs->y[q] * V[(long long)q * n + i];
    x[i] = acc;
  }
}

// start of a cycle from r (= M^-1 (b - A x)) with ||r||^2 in rr: V_0 = r / beta, g = beta e_1
__global__ void k_gmres_begin(GmresState *__restrict__ gs, const double *__restrict__ rr, int first) {
  const double beta = sqrt(fmax(rr[0], 0.0));
  if (first) {
    gs->res0 = beta;
    gs->tol = fmax(gs->rtol * beta, gs->atol);
    gs->its = 0;
    gs->reason = 0;
    gs->converged = 0;
  }
  for (int i = 0; i <= gs->restart; ++i) gs->g[i] = 0.0;
  gs->g[0] = beta;
  gs->hn = beta;
  gs->j = 0;
  gs->res = beta;
  gs->stop = 0;
  if (first && beta <= gs->atol) { gs->stop = 1; gs->converged = 1; }
  if (!isfinite(beta)) { gs->stop = 1; gs->reason = -6; }
}

void launch_gmres_step(int n, int j, double *V, double *z, double *partial, double *h1, double *h2, double *zz,
                       GmresState *gs, cudaStream_t s) {
  const int nblk = 32;
  k_multidot<<<dim3(nblk, j + 1), 256, 0, s>>>(n, j + 1, V, z, partial, gs);
  k_multidot_fin<<<1, 64, 0, s>>>(j + 1, nblk, partial, h1, 0, gs);
  k_orth_sub<<<std::max(1, std::min(ceil_div(n, 256), kRedBlocks)), 256, 0, s>>>(n, j + 1, V, h1, z, gs);
  k_multidot<<<dim3(nblk, j + 1), 256, 0, s>>>(n, j + 1, V, z, partial, gs);
  k_multidot_fin<<<1, 64, 0, s>>>(j + 1, nblk, partial, h2, 0, gs);
  k_orth_sub<<<std::max(1, std::min(ceil_div(n, 256), kRedBlocks)), 256, 0, s>>>(n, j + 1, V, h2, z, gs);
  k_multidot<<<dim3(nblk, 1), 256, 0, s>>>(n, 1, z, z, partial, gs);
  k_multidot_fin<<<1, 64, 0, s>>>(1, nblk, partial, zz, 0, gs);
  k_gmres_rot<<<1, 1, 0, s>>>(gs, h1, h2, zz, j);
  k_gmres_scale<<<std::max(1, std::min(ceil_div(n, 256), kRedBlocks)), 256, 0, s>>>(n, z, V + (long long)(j + 1) * n,
                                                                                   gs);
  count_launch(10);
}

void launch_gmres_begin(int n, const double *r, double *v0, GmresState *gs, const double *rr, int first,
                        cudaStream_t s) {
  k_gmres_begin<<<1, 1, 0, s>>>(gs, rr, first);
  k_gmres_scale<<<std::max(1, std::min(ceil_div(n, 256), kRedBlocks)), 256, 0, s>>>(n, r, v0, gs);
  count_launch(2);
}

void launch_gmres_end(int n, const double *V, double *x, GmresState *gs, cudaStream_t s) {
  k_gmres_solve_y<<<1, 1, 0, s>>>(gs);
  k_gmres_update_x<<<std::max(1, std::min(ceil_div(n, 256), kRedBlocks)), 256, 0, s>>>(n, V, x, gs);
  count_launch(2);
}

}  // namespace bd
