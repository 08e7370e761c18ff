// Launchers of the domain-decomposition kernels (dd.cu).
#pragma once
#include "kernels.cuh"
#include "tasks.h"

namespace bd {

// Device-resident Krylov scalars; every kernel of an iteration returns at once
// when `done` is set, so iterations can be enqueued ahead of the convergence test.
struct KrylovState {
  double rz, alpha, beta, zn, zn0, tol;
  double rtol, atol, dtol;
  int it, done, reason, maxit, hist_cap, pad;
};

// A PCG reduction fused into the kernel that produces its second operand y:
// which = 0: a.y -> alpha; which = 1: (a.y, y.y) -> beta and the convergence test.
struct DotFuse {
  int which;
  const double *a;
  double *partial;
  unsigned int *counter;
  KrylovState *ks;
  double *hist;
};

// Device-resident GMRES(m) state (m <= kMaxRestart).
constexpr int kMaxRestart = 64;
struct GmresState {
  double H[(kMaxRestart + 1) * kMaxRestart];
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
  double rtol, atol, dtol, tol, res0, res, hn;
  int restart, maxit, its, j, stop, converged, reason, pad;
};
void launch_gmres_step(int n, int j, double *V, double *z, double *partial, double *h1, double *h2, double *zz,
                       GmresState *gs, cudaStream_t s);
void launch_gmres_begin(int n, const double *r, double *v0, GmresState *gs, const double *rr, int first,
                        cudaStream_t s);
void launch_gmres_end(int n, const double *V, double *x, GmresState *gs, cudaStream_t s);

template <typename T>
void launch_assemble_local(int nq, const int *q_sub, const int *q_loc, const int *q_node, const int *nbr,
                           const double *stencil, const double *mass, const double *factor, double tau,
                           const MatDesc *desc, T *base, cudaStream_t s);
template <typename TS, typename TD>
void launch_copy(int ntasks, long long max_elems, const CopyTask *tasks, const TS *src, TD *dst, cudaStream_t s);
template <typename T>
void launch_build_aug(int nsub, int max_m, const MatDesc *sdesc, const T *sbase, const MatDesc *adesc,
                      T *abase, const int *nD, const int *tptr_off, const int *tptr, const int *trow,
                      const T *tval, cudaStream_t s);
template <typename T>
void launch_small_gemm(int ntasks, int max_n, const GemmTask *tasks, const T *A, const T *B, T *C, cudaStream_t s);
template <typename T>
void launch_class_aug(int ncls, int max_n, const ClassTask *cls, const PairTask *pairs, const T *blk,
                      const MatDesc *cdesc, T *cbase, cudaStream_t s);
// ---- coarse problem (Section 4.4) ------------------------------------------------
// S_PP is kept as an FP64 CSR matrix (pattern of the local primal couplings, gauge row
// and column pinned to the unit vector) and, in the local precision, as the dense
// augmented matrix [[S_PP, I], [I, 0]] whose partial Cholesky leaves -S_PP^-1.
// Entry e of the CSR sums the local entries src[sptr[e] .. sptr[e + 1]) of the
// augmented local matrices.
// dense64 (nullable): also the dense FP64 S_PP, np x np (small problems)
template <typename T>
void launch_coarse_assemble(int nnz, int np, int gauge, const int *crow, const int *ccol, const int *sptr,
                            const long long *src, const T *abase, double *val64, T *co, int ld, double *dense64,
                            cudaStream_t s);
// small problems: X = (double) x0 (leading dimension ld0), then two Newton-Schulz steps
// X <- 2X - X C X against the dense FP64 S_PP (C); W, Y scratch (np x np each)
template <typename T>
void coarse_refine64(int np, const T *x0, int ld0, const double *C, double *X, double *W, double *Y, cudaStream_t s);

// The coarse solve z = S_PP^-1 c with c = rP - sum_j (Psi^T r_D)_j: an explicit
// inverse followed by nref steps of iterative refinement z += X (c - S_PP z) against the
// FP64 CSR, so the result is the FP64 solution.  np <= kCoarseSmall: the inverse refined
// to FP64 once per Jacobian (X64) and one CTA per solve; otherwise the inverse in the
// local precision and one GEMV per pass over the whole grid.
constexpr int kCoarseSmall = 320;
struct CoarseSolve {
  int np = 0, gauge = -1, nref = 1;
  const double *X64 = nullptr;                      // small problems: the FP64 inverse
  const int *pl_ptr = nullptr, *pl_idx = nullptr;  // assembly lists of the local primal products
  const int *sptr = nullptr, *scol = nullptr;      // S_PP (CSR, FP64)
  const double *sval = nullptr;
  int ld_x = 0;                                     // row stride of the explicit inverse X (multiple of 8)
};
// c and rho: np-long scratch (large problems only); z: np-long output
template <typename T>
void launch_coarse_solve(const CoarseSolve &cs, const T *X, const double *yprim, const double *rP, const CsrIn *rPc,
                         double *z, double *c, double *rho, const int *done, cudaStream_t s);
void launch_spmv(int n, const int *ptr, const int *col, const double *val, const double *x, double *y, int zero,
                 const int *done, cudaStream_t s);
void launch_gather_sum(int n, const int *ptr, const int *idx, const double *src, double *y, int zero, double alpha,
                       const double *addend, const int *done, cudaStream_t s, const CsrIn *add_csr = nullptr);
// rho-scaling: Sinv_C = diag(1 / sum sigma_M), Blk_C^(j) = diag(sigma_M) for every class
template <typename T>
void launch_rho_blocks(int ncls, const ClassTask *cls, const PairTask *pairs, double sig_i, double sig_e, T *sinv,
                       T *blk, cudaStream_t s);
// fused with the PCG reduction f (alpha = 1, no addend; y[zero] = 0)
void launch_gather_sum_dot(int n, const int *ptr, const int *idx, const double *src, double *y, int zero,
                           const DotFuse &f, cudaStream_t s);
void launch_spmv_dot(int n, const int *ptr, const int *col, const double *val, const double *x, double *y, int zero,
                     const DotFuse &f, cudaStream_t s);
void launch_jump(int nlt, int max_n, const LamTask *lt, const PairTask *pairs, const double *w, double *lam,
                 const int *done, cudaStream_t s);
void launch_jump_t(int nwt, int max_n, const WTask *wt, const WEnt *ent, const double *lam, double *w,
                   const int *done, cudaStream_t s);
template <typename T>
void launch_jump_dt(int nwt, int max_n, const WTask *wt, const WEnt *ent, const T *blk, const T *sinv,
                    const double *mu, double *w, const int *done, cudaStream_t s);
template <typename T>
void launch_jump_d(int nlt, int max_n, const LamTask *lt, const PairTask *pairs, const T *blk, const T *sinv,
                   const double *y, double *mu, const int *done, cudaStream_t s);
void launch_dual_mean(int ncls, int max_n, const ClassTask *cls, const PairTask *pairs, const double *zD,
                      double *zbar, cudaStream_t s);
void launch_gather_pairs(int n, const int *node, const double *fi, const double *fe, double *v, double scale,
                         const double *mult, cudaStream_t s);
void launch_scatter_pairs(int n, const int *node, const double *v, double *si, double *se, cudaStream_t s);
void launch_tloc_t(int nt, const int *t_sub, const int *t_loc, const int *t_ptr, const int *t_row,
                   const double *t_val, const int *g_off, const double *g, const int *nD, const int *ldual_off,
                   const int *lprim_off, double *outD, double *outP, cudaStream_t s);
void launch_gather_scale_sub(int n, const int *idx, const double *x, const double *w, double *y, cudaStream_t s);
void launch_fill(int n, double *y, double v, cudaStream_t s);
void launch_copy_vec(int n, const double *x, double *y, const int *done, cudaStream_t s);
void launch_axpby(int n, double a, const double *x, double b, double *y, cudaStream_t s);
void launch_pcg_start(KrylovState *ks, const double *dots, cudaStream_t s);
void launch_pcg_alpha(KrylovState *ks, const double *dots, double *ha, cudaStream_t s);
void launch_pcg_beta(KrylovState *ks, const double *dots, double *hb, cudaStream_t s);
void launch_pcg_xr(int n, const KrylovState *ks, const double *p, const double *q, double *x, double *r,
                   cudaStream_t s);
void launch_pcg_p(int n, const KrylovState *ks, const double *z, double *p, cudaStream_t s);
// hist: alphas at [0, cap), betas at [cap, 2 cap)
void launch_pcg_dot_step(int n, int which, const double *a0, const double *b0, const double *a1, const double *b1,
                         double *partial, unsigned int *counter, KrylovState *ks, double *hist, cudaStream_t s);
void launch_dot2(int n, const double *a0, const double *b0, const double *a1, const double *b1, double *partial,
                 double *out, const int *done, cudaStream_t s);

}  // namespace bd
