// Kernel launchers of the Bidomain GB300 library (host-callable).
#pragma once
#include <vector>

#include "common.cuh"

namespace bd {

constexpr int kRedBlocks = 304;  // fixed reduction grid (2 x 152 SMs): deterministic sums
constexpr int kNB = 32;          // panel width of the partial Cholesky

// Per-launch timing hook (CUDA events recorded on the launch stream) and
// the library-wide kernel launch counter.
// Kernel classes (timed per launch) and regions of a step (timed as a whole, also
// while the Krylov iterations replay as CUDA graphs).
enum {
  PROF_RANKK = 0, PROF_PANEL = 1, PROF_GEMV = 2, PROF_RESID = 3,
  PROF_LINEARIZE = 4, PROF_KRYLOV = 5, PROF_TRSV = 6, PROF_MLP = 7, PROF_STEP = 8,
  PROF_NCLASS = 9, PROF_FIRST_REGION = 4
};
struct ProfHook {
  virtual void begin(int id, cudaStream_t s) = 0;
  virtual void end(int id, cudaStream_t s, double flops, double bytes) = 0;
  virtual ~ProfHook() {}
};
void count_launch(int n = 1);
long long launch_count();

struct FemParams {
  double sigma_i[3], sigma_e[3];
  double G, eta1, eta2, vth, vp, chi_cm, tau;
};

struct StimParams {
  int active;
  double amp;
  double box[6];
  double h[3];
  double o[3];  // grid origin in the parametric coordinates
};

// Element geometry: kind 0 = box (spacing h, slab depth lz), 1 = truncated
// ellipsoid (Section 6) over the parametric grid origin + ijk h with
// axes a1, a2, b1, b2, c1, c2.
struct GeoParams {
  int kind;
  double h[3], o[3], lz;
  double axes[6];
};

// fem.cu
// Ke: 2 x 64 per element (intra, extra); Me: 8 lumped masses per element.
void launch_element_matrices(int ne, const int *elem_ijk, const GeoParams &g, const FemParams &fp, double *Ke,
                             double *Me, cudaStream_t s);
// out[r] = lumped mass of node row_node[r] (r itself when row_node is null),
// summed over its elements (those of subdomain row_sub[r] when row_sub is given).
void launch_mass_gather(int nrows, const int *row_node, const int *row_sub, const int *node_ijk,
                        const int *elem_grid, const int *elem_sub, const int n[3], const double *Me, double *out,
                        cudaStream_t s);
void launch_stencil_gather(int nrows, const int *row_node, const int *row_sub, const int *node_ijk,
                           const int *elem_grid, const int *elem_sub, const int n[3], const double *Ke,
                           double *out, int soa_stride, cudaStream_t s);
void launch_gating(int n, const double *ui, const double *ue, const double *w, double *wn, const FemParams &p,
                   cudaStream_t s);
void launch_residual(int n, const double *stencil, const int *nbr, const double *mass, const int *node_ijk,
                     const double *ui0, const double *ue0, const double *si, const double *se, double lam,
                     const double *wn, const double *uin, const double *uen, const FemParams &p,
                     const StimParams &st, double *ri, double *re, double *factor, double *ui_out,
                     double *ue_out, double *partial, double *norm2, cudaStream_t s);
void launch_dot3(int n, const double *a0, const double *b0, const double *a1, const double *b1, const double *a2,
                 const double *b2, double *partial, double *out, cudaStream_t s);
void launch_gauge_shift(int n, double *ui, double *ue, const double *scal, cudaStream_t s);
void launch_sum_partials(int nblk, const double *partial, double *out, cudaStream_t s);

// dense.cu -- batched partial Cholesky: eliminates the first e columns of every
// matrix; afterwards the trailing (m-e) x (m-e) lower triangle holds the Schur
// complement A22 - A21 A11^-1 A12 and the first e columns hold L11 and L21.
struct EngineShape {
  int count;
  int max_e, max_m;
  std::vector<int> m, e;  // host copies for per-step grid sizes
  int ob = 256;           // outer block: columns per long-K trailing update (multiple of 128)
  std::vector<int> band;  // host copies of MatDesc::band (empty: every matrix dense)
  std::vector<int> id0;   // host copies of MatDesc::id0 (empty: no identity block)
  std::vector<const int *> ifirst;  // host copies of MatDesc::ifirst (empty or nullptr: dense)
};
// The engine works through outer blocks of sh.ob columns: panels of kEnginePanel
// columns (k_bigpanel), each followed by an update of the rest of its block, then
// one long-K (K = ob) update of the trailing columns.  store: block store
// receiving the factored kNB x kNB diagonal blocks L_kk; matrix b uses slots
// [desc[b].dblk, desc[b].dblk + ceil(e_b / kNB)) (row-major, identity outside the last
// block's width).  tc: FP32 only, run the long-K updates on the tensor cores (tc.cu).
constexpr int kEnginePanel = 128;
// pinv (FP32 with tc only): 128 x 128 floats per matrix of scratch; with it, the rows below
// every panel are solved as one tensor-core product with the inverse of the diagonal block.
template <typename T>
void engine_partial_cholesky(const EngineShape &sh, const MatDesc *d_desc, T *base, int *d_err, cudaStream_t s,
                             T *store, ProfHook *prof = nullptr, bool tc = false, float *pinv = nullptr);

bool dense_configure();
size_t dense_smem_limit();  // bytes of shared memory the dense kernels may stage per CTA

// tc.cu
bool tc_configure();
void launch_rankk_tc(const MatDesc *d_desc, float *base, int mode, int K0, int K1, int max_rows, int max_cols,
                     int count, int *err, cudaStream_t s, const float *pinv = nullptr);

// The same products for many small matrices: one CTA per task over all its rows (columns)
template <typename T>
void launch_gemv_task(int ntasks, int max_rows, int max_cols, const GemvDesc *d_tasks, const T *A, const double *x,
                      const int *xidx, double *y, double alpha, const int *done, cudaStream_t s);
template <typename T>
void launch_gemv_t_task(int ntasks, int max_rows, int max_cols, const GemvDesc *d_tasks, const T *A,
                        const double *x, const int *xidx, double *y, double alpha, const int *done, cudaStream_t s,
                        const CsrIn *csr = nullptr);
// Batched symmetric GEMV over SymvTask (split CTAs per task, lower block triangle read once);
// symv_smem: its shared memory for matrices up to max_n (above dense_smem_limit: not usable);
// symv_occupancy: resident CTAs per SM at that size; symv_split: CTAs per task for a number of
// resident slots.  With split > 1, scratch holds ntasks x split rows of ld_scr >= max_n values
// and counter ntasks zeroed ints (left zeroed by every launch).
template <typename T>
size_t symv_smem(int max_n);
template <typename T>
int symv_occupancy(int max_n);
int symv_split(int ntasks, int max_n, int slots);
template <typename T>
void launch_symv_batched(int ntasks, int max_n, int split, const SymvTask *d_tasks, const T *A, const double *x,
                         const int *xidx, double *y, double alpha, const int *done, T *scratch, int *counter,
                         int ld_scr, cudaStream_t s);
// y (+)= A x for one large symmetric n x n row-major matrix (ld a multiple of 8, zero padding
// columns), reading only its lower block triangle
template <typename T>
void launch_symv_rows(int n, const T *A, int ld, const double *x, double *y, int accumulate, const int *done,
                      cudaStream_t s);
// y = alpha * A x (+ y): tasks in d_tasks (GemvDesc); x gathered through xidx when flagged.
template <typename T>
void launch_gemv(int ntasks, int max_rows, int max_cols, const GemvDesc *d_tasks, const T *A, const double *x,
                 const int *xidx, double *y, double alpha, const int *done, cudaStream_t s);
// y[a] = (accumulate ? y[a] : 0) + alpha * sum_p A[p][a] x[p]  (x gathered through xidx when flagged)
template <typename T>
void launch_gemv_t(int ntasks, int max_rows, int max_cols, const GemvDesc *d_tasks, const T *A, const double *x,
                   const int *xidx, double *y, double alpha, const int *done, cudaStream_t s,
                   const CsrIn *csr = nullptr);
// Batched triangular solves with the leading n x n lower triangles (MatDesc.e = n) left
// by the engine (off-diagonal blocks in base, diagonal blocks in the engine's store):
// y = L^-1 b (lower) or y = L^-T b (upper); b and y are concatenated vectors at vec_off[b].
template <typename T>
void launch_trsv(int count, int max_n, const MatDesc *d_desc, const int *vec_off, const T *base, const T *store,
                 const double *b, double *y, bool transpose, cudaStream_t s);

}  // namespace bd
