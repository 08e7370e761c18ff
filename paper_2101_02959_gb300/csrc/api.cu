// Host orchestration and the C-ABI (include/bidomain.h).
//
// Per Newton step (Section 3c) the Jacobian is rebuilt from its only varying
// part, the diagonal coupling Kc = M (chi Cm + tau dI/dv); every local
// matrix is factorised and condensed on the GPU (Sections 4.1-4.4) and the
// interface (BDDC) or multiplier (FETI-DP) system is solved by a device-side
// Krylov loop whose scalars never leave the GPU until convergence is tested.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "bidomain.h"
#include "dd_kernels.cuh"
#include "mlp.cuh"
#include "plan.h"

using namespace bd;

namespace {

struct Status : std::runtime_error {
  int code;
  Status(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

void ck(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) throw Status(BD_ERR_NOMEM, what);
  if (e != cudaSuccess) throw Status(BD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DevMem {
  std::vector<void *> ptrs;
  template <class X>
  X *alloc(size_t n) {
    void *p = nullptr;
    ck(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(X)), "cudaMalloc");
    ptrs.push_back(p);
    return static_cast<X *>(p);
  }
  template <class X>
  X *upload(const std::vector<X> &v, cudaStream_t s) {
    X *p = alloc<X>(v.size());
    if (!v.empty()) ck(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, s), "upload");
    return p;
  }
  ~DevMem() {
    for (void *p : ptrs) cudaFree(p);
  }
};

inline int pad8(int n) { return (n + 7) & ~7; }
inline long long pad32(long long n) { return (n + 31) & ~31LL; }

template <class T>
struct Dense {
  T *K = nullptr, *Aug = nullptr, *Sorig = nullptr, *Z = nullptr, *SDD = nullptr, *Blk = nullptr, *CA = nullptr,
    *Sinv = nullptr, *Dd = nullptr, *Linv = nullptr, *LdK = nullptr;  // Linv: block store scratch; LdK: K's
  // coarse problem in the local precision: augmented matrix, its block store, S_PiPi^-1
  T *Co = nullptr, *LdCo = nullptr, *CoInv = nullptr;
};

struct GemvSet {
  GemvDesc *d = nullptr;
  int n = 0, max_rows = 0, max_cols = 0;
};
// entries of the lower block triangle of 32 x 32 tiles of an n x n matrix, clipped to n
static inline long long sym_tile_entries(int n) {
  const long long nb = (n + 31) / 32;
  long long tot = 0;
  for (long long I = 0; I < nb; ++I) {
    const long long rows = std::min<long long>(32, n - 32 * I);
    tot += rows * std::min<long long>(n, 32 * (I + 1));
  }
  return tot;
}
struct SymvSet {  // batched symmetric GEMV tasks; n = 0 when their shared memory does not fit
  SymvTask *d = nullptr;
  int n = 0, max_n = 0;
  int split = 1, ld_scr = 0;  // CTAs per task; partial-sum rows (split > 1)
  void *scratch = nullptr;    // n x split x ld_scr values of the local precision
  int *counter = nullptr;     // n zeroed ints
};
template <class T>
void launch_symv(const SymvSet &g, const T *A, const double *x, const int *xidx, double *y, const int *done,
                 cudaStream_t s) {
  launch_symv_batched<T>(g.n, g.max_n, g.split, g.d, A, x, xidx, y, 1.0, done, static_cast<T *>(g.scratch),
                         g.counter, g.ld_scr, s);
}
struct CopySet {
  CopyTask *d = nullptr;
  int n = 0;
  long long max_elems = 0;
};

// Extreme eigenvalues of the symmetric tridiagonal matrix (d, e) by Sturm bisection.
double tridiag_cond(const std::vector<double> &d, const std::vector<double> &e) {
  const int k = (int)d.size();
  if (k == 0) return 1.0;
  double lo = d[0], hi = d[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = d[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < k; ++i) {
      if (q == 0.0) q = 1e-300;
      q = d[i] - x - e[i - 1] * e[i - 1] / q;
      if (q < 0) ++c;
    }
    return c;
  };
  auto kth = [&](int idx) {  // idx-th smallest eigenvalue, 0-based
    double a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      const double m = 0.5 * (a + b);
      if (count_below(m) > idx) b = m;
      else a = m;
      if (b - a <= 1e-15 * std::max(std::fabs(a), std::fabs(b))) break;
    }
    return 0.5 * (a + b);
  };
  const double lmin = kth(0), lmax = kth(k - 1);
  return lmax / lmin;
}

// Per-launch CUDA-event timing of selected kernel classes.
struct Profiler : ProfHook {
  int on = 0;  // 0 off, 1 kernel classes and regions, 2 regions only
  struct Rec {
    int id;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  std::vector<Rec> recs;
  std::vector<size_t> open;  // records begun and not yet ended (regions nest)
  bool wants(int id) const { return on == 1 || (on == 2 && id >= PROF_FIRST_REGION); }
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  double tot[PROF_NCLASS][4] = {};
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      ck(cudaEventCreate(&e), "event");
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(int id, cudaStream_t s) override {
    if (!wants(id)) return;
    cudaEvent_t a = get();
    ck(cudaEventRecord(a, s), "event");
    open.push_back(recs.size());
    recs.push_back(Rec{id, a, nullptr, 0.0, 0.0});
  }
  void end(int id, cudaStream_t s, double flops, double bytes) override {
    if (!wants(id) || open.empty()) return;
    cudaEvent_t b = get();
    ck(cudaEventRecord(b, s), "event");
    Rec &r = recs[open.back()];
    open.pop_back();
    r.b = b;
    r.flops = flops;
    r.bytes = bytes;
  }
  void harvest() {
    if (!open.empty()) return;  // only between regions
    for (auto &r : recs) {
      float ms = 0.f;
      ck(cudaEventSynchronize(r.b), "event sync");
      ck(cudaEventElapsedTime(&ms, r.a, r.b), "event time");
      tot[r.id][0] += 1.0;
      tot[r.id][1] += ms;
      tot[r.id][2] += r.flops;
      tot[r.id][3] += r.bytes;
    }
    recs.clear();
    used = 0;
  }
  void reset() {
    harvest();
    open.clear();
    recs.clear();
    used = 0;
    for (auto &t : tot) for (double &v : t) v = 0.0;
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

struct bd_plan {
  Plan p;
};

struct bd_handle {
  Plan plan;
  bd_options opt;
  FemParams fp;
  double tau = 0.0;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  // a second stream for the coarse solve of a preconditioner application, which runs beside
  // the local constrained solve (fork / join events; captured into the Krylov graphs too)
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int device = -1;  // the device current at bidomain_setup: every buffer of the handle lives there
  long step_n = 0;
  DevMem mem;
  int N = 0, NE = 0, nsub = 0, nif = 0, nd = 0, np = 0, nlam = 0;
  int gauge_iface = -1, gauge_primal = -1;
  double sum_mass = 0.0;
  // global FEM data
  int *d_node_ijk, *d_elem_ijk, *d_elem_grid, *d_elem_sub, *d_nbr;
  double *d_mass, *d_Ke, *d_stencil;
  // state and Newton work vectors
  double *d_ui, *d_ue, *d_w, *d_uin, *d_uen, *d_wn, *d_factor, *d_ri, *d_re, *d_si, *d_se, *d_fi, *d_fe;
  double *d_uit, *d_uet, *d_rit, *d_ret, *d_factort;
  double *d_partial, *d_scal;
  int *d_err;
  double *d_io[6];
  // local node tables
  int nq = 0;
  int *d_q_sub, *d_q_loc, *d_q_node, *d_q_nbr;
  double *d_q_mass, *d_q_stencil;
  // interior / interface / dual / primal layouts
  int nI_tot = 0, nG_tot = 0, nD_tot = 0, nP_tot = 0, nint_nodes = 0;
  std::vector<int> nI, nG, nD, nP, int_off, giff_off, ldual_off, lprim_off;
  std::vector<int> band_I;  // dof half-bandwidth of each interior block (nodes ordered by global id)
  std::vector<std::vector<int>> ifirst_I;  // per K matrix: first interior column of each interface row
  int *d_ifirst = nullptr;
  int *d_int_node, *d_iface_node, *d_R, *d_Rt_ptr, *d_Rt_idx, *d_vec_off_I;
  int *d_ldual_off, *d_lprim_off, *d_nD, *d_nI, *d_prim_x, *d_pl_ptr, *d_pl_idx, *d_giff_off;
  double *d_mult_iface;
  int *d_T_ptr, *d_T_col, *d_Tt_ptr, *d_Tt_col;
  double *d_T_val, *d_Tt_val;
  int nt_tot = 0;
  int *d_tl_sub, *d_tl_loc, *d_tl_ptr, *d_tl_row, *d_tl_off;
  double *d_tl_val;
  float *d_tl_valf;  // float copy of d_tl_val for the FP32 augmented-matrix build
  // dense layouts
  EngineShape shK, shA, shC, shCo;
  MatDesc *d_Kdesc, *d_Adesc, *d_Cdesc, *d_Codesc;
  long long K_el = 0, A_el = 0, So_el = 0, Z_el = 0, SDD_el = 0, Blk_el = 0, CA_el = 0, Sinv_el = 0, Dd_el = 0;
  int K_blk = 0, A_blk = 0, C_blk = 0;  // slots of the diagonal-block stores
  int ld_co = 0;
  // coarse problem: S_PP as FP64 CSR (entries sum the listed local values), solve scratch
  int co_nnz = 0;
  int *d_co_rptr = nullptr, *d_co_row = nullptr, *d_co_col = nullptr, *d_co_sptr = nullptr;
  long long *d_co_src = nullptr;
  double *d_Co64 = nullptr, *d_co_c = nullptr, *d_co_rho = nullptr;
  int *d_co_noptr = nullptr;  // np + 1 zeros: empty assembly lists (a coarse solve of a given c)
  // small coarse problems: dense FP64 S_PP, its FP64 inverse, Newton-Schulz scratch
  double *d_Co64d = nullptr, *d_CoInv64 = nullptr, *d_CoW = nullptr, *d_CoY = nullptr;
  CoarseSolve cs;
  GemvSet gv_schur, gv_local, gv_psit, gv_sdd, gv_lgi, gv_lgit, gv_drest, gv_dext;
  GemvSet gv_psi;  // Psi^T r_Delta alone (the coarse right-hand side's local parts)
  // the operator S_Gamma and the local solve [X; Psi^T] as symmetric products (X, S_Gamma
  // symmetric: each lower tile read once); used instead of gv_schur / gv_local when set
  SymvSet sv_schur, sv_local;
  // FP32 with tensor cores: the inverse of every matrix's current 128 x 128 diagonal block
  // (128 x 128 floats per matrix of the largest batch), for the panel solves
  float *d_pinv = nullptr;
  GemmTask *d_gemm = nullptr;
  int n_gemm = 0;
  int *d_ext_idx = nullptr;
  MatDesc *d_Sdesc = nullptr;
  CopySet cp_sorig, cp_sdd, cp_blk, cp_zx, cp_sinv, cp_coinv;
  int ncls = 0, npairs = 0, nlt = 0, nwt = 0, max_nc = 0;
  ClassTask *d_cls;
  PairTask *d_pairs;
  LamTask *d_lt;
  WTask *d_wt;
  WEnt *d_went;
  // work vectors
  double *d_fI, *d_yI, *d_fG, *d_fhat, *d_uG, *d_yloc, *d_rbar, *d_zbar, *d_rD, *d_ydc, *d_w1, *d_w2, *d_gP,
      *d_crhs, *d_rP, *d_rD2;
  double *d_kx, *d_kr, *d_kz, *d_kp, *d_kq, *d_kb;
  KrylovState *d_ks;
  unsigned int *d_counter = nullptr;
  GmresState *d_gs = nullptr;
  double *d_gV = nullptr, *d_gz = nullptr, *d_gt = nullptr, *d_gpart = nullptr, *d_gh = nullptr;
  double *d_ha, *d_hb;
  int hist_cap = 0;
  Dense<float> df;
  Dense<double> dd;

  bool linearized = false;
  long long n_jac = 0;  // counted Jacobian evaluations (the precond_every schedule)
  std::string last_error;
  Profiler prof;
  // learned initial guess
  MlpDev mlp;
  bool mlp_on = false;
  int hist_count = 0, mlp_steps_trained = 0;
  int n_tr_ent = 0;  // trace entries (subdomain, interface node of it)
  int *d_t_sub = nullptr, *d_t_pos = nullptr, *d_t_node = nullptr;
  int *d_tr_ptr = nullptr, *d_tr_ent = nullptr;  // interface node -> its trace entries (j * n_tr + a)
  double *d_dG = nullptr;                        // predicted interface increment (2g + field)
  double *d_uh1i, *d_uh1e, *d_uh2i, *d_uh2e, *d_gi, *d_ge;
  double rtol_scale = 1.0;
  // factorisation tuning (bidomain_autotune): outer panel width, batch groups, tensor cores
  int tune_ob = 256, tune_groups = 1;
  int tune_panel_tc = 0;  // 1: panel solves on the tensor cores too (with d_pinv; tensor cores on)
  cudaGraphExec_t pcg_exec[2] = {nullptr, nullptr};  // captured PCG chunk per method
  size_t pcg_nodes[2] = {0, 0};
  double gemv_schur_flops = 0, gemv_schur_bytes = 0, gemv_local_flops = 0, gemv_local_bytes = 0;

  bool mixed() const { return opt.precision == BD_MIXED; }
  int check_err() {
    int e = 0;
    ck(cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "read error flag");
    ck(cudaStreamSynchronize(s), "sync");
    if (e) ck(cudaMemsetAsync(d_err, 0, sizeof(int), s), "clear error flag");
    if (e & DEV_ERR_NOT_SPD) return BD_ERR_NOT_SPD;
    if (e & DEV_ERR_NAN) return BD_ERR_NAN;
    if (e & DEV_ERR_TIMEOUT) return BD_ERR_TIMEOUT;
    return BD_OK;
  }
};

namespace {

// ---------------------------------------------------------------------------
// learned initial guess: buffers, deterministic He-uniform initialisation
// ---------------------------------------------------------------------------
// The untrained network: He-uniform weights from a fixed splitmix64 stream, zero
// biases, last layer scaled by 0.1; Adam moments and counters at zero.
void mlp_init_weights(bd_handle &h) {
  MlpDev &M = h.mlp;
  cudaStream_t s = h.s;
  const int H = M.n_hidden;
  std::vector<float> w(M.n_params, 0.f);
  uint64_t st = 0x9E3779B97F4A7C15ULL;
  auto uni = [&]() {
    st += 0x9E3779B97F4A7C15ULL;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](long long off, long long n, int fan_in, double scale) {
    const double lim = std::sqrt(6.0 / fan_in) * scale;
    for (long long i = 0; i < n; ++i) w[off + i] = (float)((2.0 * uni() - 1.0) * lim);
  };
  fill(M.off_W1, (long long)H * M.n_in, M.n_in, 1.0);
  fill(M.off_W2, (long long)H * H, H, 1.0);
  fill(M.off_W3, (long long)M.n_out * H, H, 0.1);
  ck(cudaMemcpyAsync(M.w, w.data(), sizeof(float) * M.n_params, cudaMemcpyHostToDevice, s), "mlp init");
  mlp_refresh_bf16(M, s);
  ck(cudaMemsetAsync(M.am, 0, sizeof(float) * M.n_params, s), "memset");
  ck(cudaMemsetAsync(M.av, 0, sizeof(float) * M.n_params, s), "memset");
  M.t = 0;
  h.mlp_steps_trained = 0;
  h.hist_count = 0;
}

void setup_mlp(bd_handle &h) {
  DevMem &m = h.mem;
  cudaStream_t s = h.s;
  MlpDev &M = h.mlp;
  // trace nodes of subdomain j: its interface nodes, in its local order
  int n_tr = 0;
  for (auto &sp : h.plan.subs) n_tr = std::max(n_tr, (int)sp.nodes.size() - sp.n_interior);
  M.n_tr = n_tr;
  M.batch = h.nsub;
  M.n_in = 6 * n_tr;
  M.n_out = 2 * n_tr;
  auto pad64 = [](int n) { return (n + 63) & ~63; };
  M.ld_in = pad64(M.n_in);
  M.ld_out = pad64(M.n_out);
  M.ld_b = pad64(M.batch);
  const int H = M.n_hidden, B = M.batch;
  M.off_W1 = 0;
  M.off_b1 = M.off_W1 + (long long)H * M.n_in;
  M.off_W2 = M.off_b1 + H;
  M.off_b2 = M.off_W2 + (long long)H * H;
  M.off_W3 = M.off_b2 + H;
  M.off_b3 = M.off_W3 + (long long)M.n_out * H;
  M.n_params = M.off_b3 + M.n_out;
  M.w = m.alloc<float>(M.n_params);
  M.g = m.alloc<float>(M.n_params);
  M.am = m.alloc<float>(M.n_params);
  M.av = m.alloc<float>(M.n_params);
  M.b1 = M.w + M.off_b1;
  M.b2 = M.w + M.off_b2;
  M.b3 = M.w + M.off_b3;
  // bf16 operand buffers: zeroed once, so their padding stays zero
  auto bf = [&](size_t n) {
    __nv_bfloat16 *p = m.alloc<__nv_bfloat16>(n);
    ck(cudaMemsetAsync(p, 0, sizeof(__nv_bfloat16) * n, s), "memset");
    return p;
  };
  M.W1b = bf((size_t)H * M.ld_in);
  M.W2b = bf((size_t)H * H);
  M.W2bT = bf((size_t)H * H);
  M.W3b = bf((size_t)M.n_out * H);
  M.W3bT = bf((size_t)H * M.ld_out);
  M.Xb = bf((size_t)B * M.ld_in);
  M.XbT = bf((size_t)M.n_in * M.ld_b);
  M.H1b = bf((size_t)B * H);
  M.H1bT = bf((size_t)H * M.ld_b);
  M.H2b = bf((size_t)B * H);
  M.H2bT = bf((size_t)H * M.ld_b);
  M.dYb = bf((size_t)B * M.ld_out);
  M.dYbT = bf((size_t)M.n_out * M.ld_b);
  M.dZ2b = bf((size_t)B * H);
  M.dZ2bT = bf((size_t)H * M.ld_b);
  M.dZ1bT = bf((size_t)H * M.ld_b);
  M.Z1 = m.alloc<float>((size_t)B * H);
  M.Z2 = m.alloc<float>((size_t)B * H);
  M.Y = m.alloc<float>((size_t)B * M.n_out);
  M.T = m.alloc<float>((size_t)B * M.n_out);
  M.mask = m.alloc<float>((size_t)B * M.n_out);
  M.Xf = m.alloc<float>((size_t)B * M.n_in);
  M.dY = m.alloc<float>((size_t)B * M.n_out);
  M.dZ2 = m.alloc<float>((size_t)B * H);
  M.dZ1 = m.alloc<float>((size_t)B * H);
  mlp_init_weights(h);
  // trace entries and, per interface node, the entries holding it (prediction average)
  std::vector<int> t_sub, t_pos, t_node;
  std::vector<std::vector<int>> lists(h.nif / 2);
  for (int j = 0; j < h.nsub; ++j) {
    const SubPlan &sp = h.plan.subs[j];
    for (int a = 0; a + sp.n_interior < (int)sp.nodes.size(); ++a) {
      const int x = sp.nodes[sp.n_interior + a];
      t_sub.push_back(j);
      t_pos.push_back(a);
      t_node.push_back(x);
      lists[h.plan.node_to_iface[x]].push_back(j * n_tr + a);
    }
  }
  h.n_tr_ent = (int)t_sub.size();
  h.d_t_sub = m.upload(t_sub, s);
  h.d_t_pos = m.upload(t_pos, s);
  h.d_t_node = m.upload(t_node, s);
  std::vector<int> ptr(1, 0), ent;
  for (auto &l : lists) { for (int v : l) ent.push_back(v); ptr.push_back((int)ent.size()); }
  h.d_tr_ptr = m.upload(ptr, s);
  h.d_tr_ent = m.upload(ent, s);
  h.d_dG = m.alloc<double>(h.nif);
  double **hv[] = {&h.d_uh1i, &h.d_uh1e, &h.d_uh2i, &h.d_uh2e, &h.d_gi, &h.d_ge};
  for (double **v : hv) *v = m.alloc<double>(h.N);
  h.mlp_on = true;
}

// One Adam step of the MLP on the features / targets / mask already in place;
// returns nothing (the loss lands in d_scal[4] when `want_loss`).
void mlp_train_once(bd_handle &h, bool want_loss) {
  MlpDev &M = h.mlp;
  mlp_forward(M, h.d_err, h.s);
  mlp_backward(M, 1.f / (2.f * h.n_tr_ent), h.d_partial, h.d_err, h.s);
  if (want_loss) launch_sum_partials(kRedBlocks, h.d_partial, h.d_scal + 4, h.s);
  mlp_adam(M, (float)h.opt.mlp_lr, h.s);
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
void setup_handle(bd_handle &h) {
  Plan &p = h.plan;
  cudaStream_t s = h.s;
  DevMem &m = h.mem;
  h.N = p.n_node;
  h.NE = p.n_elem;
  h.nsub = p.n_sub;
  h.nif = p.n_iface();
  h.nd = p.n_dual;
  h.np = p.n_primal;
  h.gauge_iface = 2 * p.node_to_iface[p.gauge_node] + 1;
  h.gauge_primal = p.gauge_primal;
  const int N = h.N;
  // ---- global FEM tables
  h.d_node_ijk = m.upload(p.node_ijk, s);
  h.d_elem_ijk = m.upload(p.elem_ijk, s);
  h.d_elem_grid = m.upload(p.elem_grid, s);
  h.d_elem_sub = m.upload(p.elem_sub, s);
  std::vector<int> nbr_soa(27L * N);
  for (int x = 0; x < N; ++x)
    for (int sl = 0; sl < 27; ++sl) nbr_soa[(long)sl * N + x] = p.nbr27[27L * x + sl];
  h.d_nbr = m.upload(nbr_soa, s);
  // element matrices and lumped masses, then node masses gathered from them
  GeoParams geo{};
  geo.kind = p.geo.kind;
  geo.lz = p.l[2];
  for (int d = 0; d < 3; ++d) { geo.h[d] = p.h[d]; geo.o[d] = p.origin[d]; }
  for (int k = 0; k < 6; ++k) geo.axes[k] = p.geo.axes[k];
  h.d_Ke = m.alloc<double>(128L * h.NE);
  double *d_Me = m.alloc<double>(8L * h.NE);
  launch_element_matrices(h.NE, h.d_elem_ijk, geo, h.fp, h.d_Ke, d_Me, s);
  h.d_mass = m.alloc<double>(N);
  launch_mass_gather(N, nullptr, nullptr, h.d_node_ijk, h.d_elem_grid, h.d_elem_sub, p.n, d_Me, h.d_mass, s);
  {
    std::vector<double> mass(N);
    ck(cudaMemcpyAsync(mass.data(), h.d_mass, sizeof(double) * N, cudaMemcpyDeviceToHost, s), "mass");
    ck(cudaStreamSynchronize(s), "mass");
    h.sum_mass = 0.0;
    for (double v : mass) h.sum_mass += v;
  }
  h.d_stencil = m.alloc<double>(54L * N);
  std::vector<int> all_nodes(N);
  for (int x = 0; x < N; ++x) all_nodes[x] = x;
  int *d_all = m.upload(all_nodes, s);
  launch_stencil_gather(N, d_all, nullptr, h.d_node_ijk, h.d_elem_grid, h.d_elem_sub, p.n, h.d_Ke, h.d_stencil, N, s);
  // ---- state vectors
  double **vecs[] = {&h.d_ui, &h.d_ue, &h.d_w, &h.d_uin, &h.d_uen, &h.d_wn, &h.d_factor, &h.d_ri, &h.d_re, &h.d_si,
                     &h.d_se, &h.d_fi, &h.d_fe, &h.d_uit, &h.d_uet, &h.d_rit, &h.d_ret, &h.d_factort};
  for (double **v : vecs) {
    *v = m.alloc<double>(N);
    ck(cudaMemsetAsync(*v, 0, sizeof(double) * N, s), "memset");
  }
  h.d_partial = m.alloc<double>(3 * kRedBlocks);
  h.d_scal = m.alloc<double>(64);
  h.d_err = m.alloc<int>(1);
  ck(cudaMemsetAsync(h.d_err, 0, sizeof(int), s), "memset");
  // ---- local node tables and layouts
  const int S = h.nsub;
  h.nI.resize(S); h.nG.resize(S); h.nD.resize(S); h.nP.resize(S); h.band_I.resize(S); h.ifirst_I.resize(S);
  h.int_off.resize(S); h.giff_off.resize(S); h.ldual_off.resize(S); h.lprim_off.resize(S);
  std::vector<int> q_sub, q_loc, q_node, q_nbr, int_node, R, prim_x, vec_off_I(S);
  for (int j = 0; j < S; ++j) {
    const SubPlan &sp = p.subs[j];
    h.nI[j] = sp.nI(); h.nG[j] = sp.nG(); h.nD[j] = sp.nD(); h.nP[j] = sp.nP();
    h.int_off[j] = h.nint_nodes;
    vec_off_I[j] = 2 * h.nint_nodes;
    h.giff_off[j] = h.nG_tot;
    h.ldual_off[j] = h.nD_tot;
    h.lprim_off[j] = h.nP_tot;
    int nband = 0;  // node half-bandwidth of the interior block (nodes ordered by global id)
    for (int a = 0; a < (int)sp.nodes.size(); ++a) {
      q_sub.push_back(j); q_loc.push_back(a); q_node.push_back(sp.nodes[a]);
      for (int sl = 0; sl < 27; ++sl) {
        const int b = sp.nbr[27 * a + sl];
        q_nbr.push_back(b);
        if (a < sp.n_interior && b >= 0 && b < sp.n_interior) nband = std::max(nband, std::abs(a - b));
      }
    }
    // dofs 2a + field: the couplings of nodes a, b lie within |2a - 2b| + 1 of the diagonal
    h.band_I[j] = 2 * nband + 1;
    // interface rows of K: the first interior column each couples to (its L row is zero
    // left of it), as a suffix minimum so the bound is non-decreasing
    {
      const int ng = (int)sp.nodes.size() - sp.n_interior;
      std::vector<int> first(2 * ng, 2 * sp.n_interior);
      for (int a = sp.n_interior; a < (int)sp.nodes.size(); ++a) {
        int fb = sp.n_interior;
        for (int sl = 0; sl < 27; ++sl) {
          const int b = sp.nbr[27 * a + sl];
          if (b >= 0 && b < sp.n_interior) fb = std::min(fb, b);
        }
        first[2 * (a - sp.n_interior)] = first[2 * (a - sp.n_interior) + 1] = 2 * fb;
      }
      for (int g = 2 * ng - 2; g >= 0; --g) first[g] = std::min(first[g], first[g + 1]);
      h.ifirst_I[j] = std::move(first);
    }
    for (int a = 0; a < sp.n_interior; ++a) int_node.push_back(sp.nodes[a]);
    for (int a = sp.n_interior; a < (int)sp.nodes.size(); ++a) {
      const int g = p.node_to_iface[sp.nodes[a]];
      R.push_back(2 * g); R.push_back(2 * g + 1);
    }
    for (int q : sp.primal) prim_x.push_back(h.nd + q);
    h.nint_nodes += sp.n_interior;
    h.nG_tot += h.nG[j];
    h.nD_tot += h.nD[j];
    h.nP_tot += h.nP[j];
  }
  h.nI_tot = 2 * h.nint_nodes;
  h.nq = (int)q_sub.size();
  h.d_q_sub = m.upload(q_sub, s); h.d_q_loc = m.upload(q_loc, s); h.d_q_node = m.upload(q_node, s);
  h.d_q_nbr = m.upload(q_nbr, s);
  h.d_q_mass = m.alloc<double>(h.nq);
  launch_mass_gather(h.nq, h.d_q_node, h.d_q_sub, h.d_node_ijk, h.d_elem_grid, h.d_elem_sub, p.n, d_Me, h.d_q_mass, s);
  h.d_q_stencil = m.alloc<double>(54L * h.nq);
  launch_stencil_gather(h.nq, h.d_q_node, h.d_q_sub, h.d_node_ijk, h.d_elem_grid, h.d_elem_sub, p.n, h.d_Ke,
                        h.d_q_stencil, 0, s);
  h.d_int_node = m.upload(int_node, s);
  h.d_iface_node = m.upload(p.iface_nodes, s);
  h.d_R = m.upload(R, s);
  h.d_vec_off_I = m.upload(vec_off_I, s);
  h.d_giff_off = m.upload(h.giff_off, s);
  h.d_ldual_off = m.upload(h.ldual_off, s);
  h.d_lprim_off = m.upload(h.lprim_off, s);
  h.d_nD = m.upload(h.nD, s);
  h.d_nI = m.upload(h.nI, s);
  h.d_prim_x = m.upload(prim_x, s);
  // R^T as CSR over global interface dofs (subdomain order inside a row)
  {
    std::vector<std::vector<int>> rows(h.nif);
    for (int t = 0; t < (int)R.size(); ++t) rows[R[t]].push_back(t);
    std::vector<int> ptr(1, 0), idx;
    for (auto &r : rows) { for (int t : r) idx.push_back(t); ptr.push_back((int)idx.size()); }
    h.d_Rt_ptr = m.upload(ptr, s);
    h.d_Rt_idx = m.upload(idx, s);
    std::vector<double> mult(h.nif);
    for (int g = 0; g < h.nif; ++g) mult[g] = 1.0 / (double)p.mult[p.iface_nodes[g / 2]];
    h.d_mult_iface = m.upload(mult, s);
  }
  // primal assembly list (coarse right-hand side)
  {
    std::vector<std::vector<int>> rows(h.np);
    for (int j = 0; j < S; ++j)
      for (int a = 0; a < h.nP[j]; ++a) rows[p.subs[j].primal[a]].push_back(h.lprim_off[j] + a);
    std::vector<int> ptr(1, 0), idx;
    for (auto &r : rows) { for (int t : r) idx.push_back(t); ptr.push_back((int)idx.size()); }
    h.d_pl_ptr = m.upload(ptr, s);
    h.d_pl_idx = m.upload(idx, s);
  }
  h.d_T_ptr = m.upload(p.T_ptr, s); h.d_T_col = m.upload(p.T_col, s); h.d_T_val = m.upload(p.T_val, s);
  h.d_Tt_ptr = m.upload(p.Tt_ptr, s); h.d_Tt_col = m.upload(p.Tt_col, s); h.d_Tt_val = m.upload(p.Tt_val, s);
  // local change of basis, flattened CSC
  {
    std::vector<int> tl_sub, tl_loc, tl_ptr(1, 0), tl_row, tl_off(S);
    std::vector<double> tl_val;
    for (int j = 0; j < S; ++j) {
      std::vector<int> ptr, row;
      std::vector<double> val;
      local_T(p, j, ptr, row, val);
      tl_off[j] = (int)tl_sub.size();
      const int base = (int)tl_row.size();
      for (int a = 0; a + 1 < (int)ptr.size(); ++a) {
        tl_sub.push_back(j);
        tl_loc.push_back(a);
        tl_ptr.push_back(base + ptr[a + 1]);
      }
      tl_row.insert(tl_row.end(), row.begin(), row.end());
      tl_val.insert(tl_val.end(), val.begin(), val.end());
    }
    h.nt_tot = (int)tl_sub.size();
    h.d_tl_sub = m.upload(tl_sub, s); h.d_tl_loc = m.upload(tl_loc, s); h.d_tl_ptr = m.upload(tl_ptr, s);
    h.d_tl_row = m.upload(tl_row, s); h.d_tl_val = m.upload(tl_val, s);
    h.d_tl_valf = m.upload(std::vector<float>(tl_val.begin(), tl_val.end()), s); h.d_tl_off = m.upload(tl_off, s);
  }
  // ---- dense layouts
  std::vector<MatDesc> kd(S), ad(S);
  std::vector<long long> ifirst_off(S);
  {
    std::vector<int> flat;
    for (int j = 0; j < S; ++j) {
      ifirst_off[j] = (long long)flat.size();
      flat.insert(flat.end(), h.ifirst_I[j].begin(), h.ifirst_I[j].end());
    }
    h.d_ifirst = m.upload(flat, s);
  }
  std::vector<long long> so_off(S), zx_off(S), zp_off(S), sdd_off(S);
  std::vector<int> ldx(S), ldg(S);
  h.shK = EngineShape{S, 0, 0, {}, {}};
  h.shA = EngineShape{S, 0, 0, {}, {}};
  for (int j = 0; j < S; ++j) {
    const int n = h.nI[j] + h.nG[j];
    kd[j] = MatDesc{h.K_el, pad8(n), n, h.nI[j], h.K_blk};
    kd[j].band = h.band_I[j];  // the interior block is banded: its updates skip the zeros past the band
    kd[j].ifirst = h.d_ifirst + ifirst_off[j];  // and the interface rows of L_GI start late
    h.K_blk += ceil_div(h.nI[j], kNB);
    h.K_el += pad32((long long)pad8(n) * n);
    const int ma = 2 * h.nD[j] + h.nP[j];
    ad[j] = MatDesc{h.A_el, pad8(ma), ma, h.nD[j], h.A_blk};
    ad[j].id0 = h.nD[j] + h.nP[j];  // [[Sb_DD, Sb_DP, I], [Sb_PD, Sb_PP, 0], [I, 0, 0]]
    h.A_blk += ceil_div(h.nD[j], kNB);
    h.A_el += pad32((long long)pad8(ma) * ma);
    ldg[j] = pad8(h.nG[j]);
    so_off[j] = h.So_el;
    h.So_el += pad32((long long)ldg[j] * h.nG[j]);
    ldx[j] = pad8(h.nD[j]);
    zx_off[j] = h.Z_el;
    h.Z_el += pad32((long long)ldx[j] * h.nD[j]);
    zp_off[j] = h.Z_el;
    h.Z_el += pad32((long long)ldx[j] * h.nP[j]);
    sdd_off[j] = h.SDD_el;
    h.SDD_el += pad32((long long)ldx[j] * h.nD[j]);
    h.shK.m.push_back(n); h.shK.e.push_back(h.nI[j]); h.shK.band.push_back(h.band_I[j]);
    h.shK.ifirst.push_back(h.ifirst_I[j].data());  // ifirst_I is not resized after setup
    h.shA.m.push_back(ma); h.shA.e.push_back(h.nD[j]); h.shA.id0.push_back(ad[j].id0);
    h.shK.max_m = std::max(h.shK.max_m, n); h.shK.max_e = std::max(h.shK.max_e, h.nI[j]);
    h.shA.max_m = std::max(h.shA.max_m, ma); h.shA.max_e = std::max(h.shA.max_e, h.nD[j]);
  }
  h.d_Kdesc = m.upload(kd, s);
  h.d_Adesc = m.upload(ad, s);
  {
    std::vector<MatDesc> sdv(S);
    for (int j = 0; j < S; ++j) sdv[j] = MatDesc{so_off[j], ldg[j], h.nG[j], 0, 0};
    h.d_Sdesc = m.upload(sdv, s);
  }
  // ---- deluxe classes, pairs and FETI-DP multipliers
  std::vector<ClassTask> cls;
  std::vector<PairTask> pairs;
  std::vector<MatDesc> cdesc;
  std::vector<LamTask> lts;
  std::vector<CopyTask> cp_blk, cp_sinv;
  std::map<std::pair<int, int>, int> pair_of;  // (class, sub) -> pair index
  h.shC = EngineShape{0, 0, 0, {}, {}};
  // position of each class inside each subdomain's dual vector
  std::vector<std::map<int, int>> dpos(S);
  for (int j = 0; j < S; ++j) {
    int pos = 0;
    for (int c : p.subs[j].classes) { dpos[j][c] = pos; pos += 2 * p.cls_dual_nodes[c]; }
  }
  int lam_off = 0;
  for (int c = 0; c < p.n_cls; ++c) {
    const int n = 2 * p.cls_dual_nodes[c];
    if (n == 0) continue;
    ClassTask ct{};
    ct.n = n;
    ct.dual_start = p.cls_dual_start[c];
    ct.sinv_off = h.Sinv_el;
    ct.pair_beg = (int)pairs.size();
    std::vector<int> subs(p.cls_subs.begin() + p.cls_sub_ptr[c], p.cls_subs.begin() + p.cls_sub_ptr[c + 1]);
    for (int j : subs) {
      PairTask pt{};
      pt.blk_off = h.Blk_el;
      pt.ldual_off = h.ldual_off[j] + dpos[j][c];
      pt.sub = j;
      pair_of[{c, j}] = (int)pairs.size();
      CopyTask cb{};
      cb.src_off = ad[j].off; cb.src_ld = ad[j].ld; cb.r0 = cb.c0 = dpos[j][c]; cb.rows = cb.cols = n;
      cb.mode = 3; cb.sign = 1.0; cb.dst_off = pt.blk_off; cb.dst_ld = n;
      cp_blk.push_back(cb);
      pairs.push_back(pt);
      h.Blk_el += pad32((long long)n * n);
    }
    ct.pair_end = (int)pairs.size();
    for (int a = 0; a < (int)subs.size(); ++a)
      for (int b = a + 1; b < (int)subs.size(); ++b) {
        LamTask lt{};
        lt.lam_off = lam_off;
        lt.n = n;
        lt.pa = pair_of[{c, subs[a]}];
        lt.pb = pair_of[{c, subs[b]}];
        lt.sinv_off = ct.sinv_off;
        lts.push_back(lt);
        lam_off += n;
      }
    const int mc = 2 * n;
    MatDesc md{h.CA_el, pad8(mc), mc, n, h.C_blk};
    md.id0 = n;  // [[sum_j S_C^(j), I], [I, 0]]
    h.C_blk += ceil_div(n, kNB);
    h.CA_el += pad32((long long)pad8(mc) * mc);
    cdesc.push_back(md);
    h.shC.m.push_back(mc); h.shC.e.push_back(n); h.shC.id0.push_back(n);
    h.shC.max_m = std::max(h.shC.max_m, mc); h.shC.max_e = std::max(h.shC.max_e, n);
    CopyTask cs{};
    cs.src_off = md.off; cs.src_ld = md.ld; cs.r0 = cs.c0 = n; cs.rows = cs.cols = n; cs.mode = 3; cs.sign = -1.0;
    cs.dst_off = ct.sinv_off; cs.dst_ld = n;
    cp_sinv.push_back(cs);
    h.Sinv_el += pad32((long long)n * n);
    h.max_nc = std::max(h.max_nc, n);
    cls.push_back(ct);
  }
  h.shC.count = (int)cls.size();
  h.ncls = (int)cls.size();
  h.npairs = (int)pairs.size();
  h.nlam = lam_off;
  h.nlt = (int)lts.size();
  // W tasks (per pair) and their multiplier entries
  std::vector<WTask> wts(pairs.size());
  std::vector<std::vector<WEnt>> wents(pairs.size());
  for (const LamTask &lt : lts) {
    wents[lt.pa].push_back(WEnt{pairs[lt.pb].blk_off, lt.lam_off, +1});
    wents[lt.pb].push_back(WEnt{pairs[lt.pa].blk_off, lt.lam_off, -1});
  }
  std::vector<WEnt> went;
  for (size_t q = 0; q < pairs.size(); ++q) {
    WTask &w = wts[q];
    w.ldual_off = pairs[q].ldual_off;
    w.n = 0;
    w.ent_beg = (int)went.size();
    for (auto &e : wents[q]) went.push_back(e);
    w.ent_end = (int)went.size();
  }
  for (const ClassTask &ct : cls)
    for (int q = ct.pair_beg; q < ct.pair_end; ++q) { wts[q].n = ct.n; wts[q].sinv_off = ct.sinv_off; }
  h.nwt = (int)wts.size();
  h.d_cls = m.upload(cls, s);
  h.d_pairs = m.upload(pairs, s);
  h.d_lt = m.upload(lts, s);
  h.d_wt = m.upload(wts, s);
  h.d_went = m.upload(went, s);
  h.d_Cdesc = m.upload(cdesc, s);
  // explicit deluxe operators: per class, D_C = [D_C^(j1) | D_C^(j2) | ...] (n x k n, row-major)
  {
    std::vector<GemmTask> gt;
    std::vector<GemvDesc> rest, ext;
    std::vector<int> ext_idx;
    for (const ClassTask &ct : cls) {
      const int n = ct.n, k = ct.pair_end - ct.pair_beg;
      const long long base = h.Dd_el;
      for (int q = ct.pair_beg; q < ct.pair_end; ++q) {
        const int pl = q - ct.pair_beg;
        gt.push_back(GemmTask{ct.sinv_off, pairs[q].blk_off, base + (long long)pl * n, n, k * n});
        rest.push_back(GemvDesc{base + (long long)pl * n, k * n, n, n, ct.dual_start, pairs[q].ldual_off, 0});
      }
      ext.push_back(GemvDesc{base, k * n, n, k * n, (int)ext_idx.size(), ct.dual_start, 1});
      for (int q = ct.pair_beg; q < ct.pair_end; ++q)
        for (int v = 0; v < n; ++v) ext_idx.push_back(pairs[q].ldual_off + v);
      h.Dd_el += pad32((long long)n * k * n);
    }
    h.n_gemm = (int)gt.size();
    h.d_gemm = m.upload(gt, s);
    h.d_ext_idx = m.upload(ext_idx, s);
    auto mk = [&](const std::vector<GemvDesc> &v) {
      GemvSet g;
      g.n = (int)v.size();
      for (auto &t : v) { g.max_rows = std::max(g.max_rows, t.rows); g.max_cols = std::max(g.max_cols, t.cols); }
      g.d = m.upload(v, s);
      return g;
    };
    h.gv_drest = mk(rest);
    h.gv_dext = mk(ext);
  }
  // ---- coarse problem
  {
    const int np = h.np;
    h.ld_co = pad8(2 * np);
    MatDesc co{0, h.ld_co, 2 * np, np, 0};
    co.id0 = np;  // [[S_PP, I], [I, 0]]
    h.d_Codesc = m.upload(std::vector<MatDesc>{co}, s);
    h.shCo = EngineShape{1, np, 2 * np, {2 * np}, {np}};
    h.shCo.id0 = {np};
    if (h.mixed()) {  // the autotuner may turn the tensor cores on
      const int most = std::max({h.shK.count, h.shA.count, h.shC.count, 1});
      h.d_pinv = m.alloc<float>((size_t)most * 128 * 128);
    }
    // sparse pattern of S_PP: the (p, q) pairs that some subdomain couples, with the
    // offsets of their local contributions in the augmented matrices (subdomain order)
    std::map<std::pair<int, int>, std::vector<long long>> ent;
    for (int j = 0; j < S; ++j) {
      const SubPlan &sp = p.subs[j];
      const int nd = h.nD[j];
      for (int a = 0; a < h.nP[j]; ++a)
        for (int b = 0; b < h.nP[j]; ++b) {
          const int hi = std::max(a, b), lo = std::min(a, b);
          ent[{sp.primal[a], sp.primal[b]}].push_back(ad[j].off + (long long)(nd + hi) * ad[j].ld + nd + lo);
        }
    }
    for (int q = 0; q < np; ++q) ent[{q, q}];  // every diagonal entry is stored (the gauge's is pinned)
    std::vector<int> rptr(np + 1, 0), row, col, sptr(1, 0);
    std::vector<long long> src;
    for (auto &kv : ent) {  // std::map order = row-major, columns ascending
      row.push_back(kv.first.first);
      col.push_back(kv.first.second);
      rptr[kv.first.first + 1] += 1;
      for (long long v : kv.second) src.push_back(v);
      sptr.push_back((int)src.size());
    }
    for (int q = 0; q < np; ++q) rptr[q + 1] += rptr[q];
    h.co_nnz = (int)row.size();
    h.d_co_rptr = m.upload(rptr, s);
    h.d_co_row = m.upload(row, s);
    h.d_co_col = m.upload(col, s);
    h.d_co_sptr = m.upload(sptr, s);
    h.d_co_src = m.upload(src, s);
    h.d_Co64 = m.alloc<double>(h.co_nnz);
    h.d_co_c = m.alloc<double>(np);
    h.d_co_rho = m.alloc<double>(np);
    h.d_co_noptr = m.upload(std::vector<int>(np + 1, 0), s);
    if (np <= kCoarseSmall) {
      const size_t nn = (size_t)np * np;
      h.d_Co64d = m.alloc<double>(nn);
      h.d_CoInv64 = m.alloc<double>(nn);
      h.d_CoW = m.alloc<double>(nn);
      h.d_CoY = m.alloc<double>(nn);
    }
  }
  // ---- GEMV and copy task sets
  auto gset = [&](const std::vector<GemvDesc> &v) {
    GemvSet g;
    g.n = (int)v.size();
    for (auto &t : v) { g.max_rows = std::max(g.max_rows, t.rows); g.max_cols = std::max(g.max_cols, t.cols); }
    g.d = m.upload(v, s);
    return g;
  };
  auto cset = [&](const std::vector<CopyTask> &v) {
    CopySet c;
    c.n = (int)v.size();
    for (auto &t : v) c.max_elems = std::max(c.max_elems, (long long)t.rows * t.cols);
    c.d = m.upload(v, s);
    return c;
  };
  std::vector<GemvDesc> g_schur, g_local, g_psit, g_sdd, g_lgi, g_lgit;
  std::vector<SymvTask> s_schur, s_local;
  std::vector<GemvDesc> g_psi;
  std::vector<CopyTask> c_sorig, c_sdd, c_zx;
  for (int j = 0; j < S; ++j) {
    const int ng = h.nG[j], ni = h.nI[j], nd = h.nD[j], npj = h.nP[j];
    g_schur.push_back(GemvDesc{so_off[j], ldg[j], ng, ng, h.giff_off[j], h.giff_off[j], 1});
    s_schur.push_back(SymvTask{so_off[j], 0, ldg[j], ng, 0, h.giff_off[j], h.giff_off[j], 0, 1});
    s_local.push_back(SymvTask{zx_off[j], 0, ldx[j], nd, 0, h.ldual_off[j], h.ldual_off[j], 0, 0});
    g_psi.push_back(GemvDesc{zp_off[j], ldx[j], npj, nd, h.ldual_off[j], h.nD_tot + h.lprim_off[j], 0});
    g_local.push_back(GemvDesc{zx_off[j], ldx[j], nd, nd, h.ldual_off[j], h.ldual_off[j], 0});
    g_local.push_back(GemvDesc{zp_off[j], ldx[j], npj, nd, h.ldual_off[j], h.nD_tot + h.lprim_off[j], 0});
    g_psit.push_back(GemvDesc{zp_off[j], ldx[j], npj, nd, h.lprim_off[j], h.ldual_off[j], 3});
    g_sdd.push_back(GemvDesc{sdd_off[j], ldx[j], nd, nd, h.ldual_off[j], h.ldual_off[j], 0});
    const long long lgi = kd[j].off + (long long)ni * kd[j].ld;
    g_lgi.push_back(GemvDesc{lgi, kd[j].ld, ng, ni, vec_off_I[j], h.giff_off[j], 0});
    g_lgit.push_back(GemvDesc{lgi, kd[j].ld, ng, ni, h.giff_off[j], vec_off_I[j], 3});
    CopyTask c{};
    c.src_off = kd[j].off; c.src_ld = kd[j].ld; c.r0 = c.c0 = ni; c.rows = c.cols = ng; c.mode = 3; c.sign = 1.0;
    c.dst_off = so_off[j]; c.dst_ld = ldg[j];
    c_sorig.push_back(c);
    CopyTask d{};
    d.src_off = ad[j].off; d.src_ld = ad[j].ld; d.r0 = d.c0 = 0; d.rows = d.cols = nd; d.mode = 3; d.sign = 1.0;
    d.dst_off = sdd_off[j]; d.dst_ld = ldx[j];
    c_sdd.push_back(d);
    CopyTask x{};
    x.src_off = ad[j].off; x.src_ld = ad[j].ld; x.r0 = x.c0 = nd + npj; x.rows = x.cols = nd; x.mode = 3;
    x.sign = -1.0; x.dst_off = zx_off[j]; x.dst_ld = ldx[j];
    c_zx.push_back(x);
    CopyTask y{};
    y.src_off = ad[j].off; y.src_ld = ad[j].ld; y.r0 = nd + npj; y.c0 = nd; y.rows = npj; y.cols = nd; y.mode = 1;
    y.sign = -1.0; y.dst_off = zp_off[j]; y.dst_ld = ldx[j];
    c_zx.push_back(y);
  }
  for (auto &t : g_schur) { h.gemv_schur_flops += 2.0 * t.rows * t.cols; h.gemv_schur_bytes += (double)t.rows * t.cols; }
  for (auto &t : g_local) { h.gemv_local_flops += 2.0 * t.rows * t.cols; h.gemv_local_bytes += (double)t.rows * t.cols; }
  h.gv_schur = gset(g_schur);
  h.gv_local = gset(g_local);
  h.gv_psi = gset(g_psi);
  {
    const size_t el = h.mixed() ? sizeof(float) : sizeof(double);
    int sms = 0;
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h.device), "SM count");
    auto sset = [&](const std::vector<SymvTask> &v) {
      SymvSet g;
      for (auto &t : v) g.max_n = std::max(g.max_n, t.n);
      const size_t np = (size_t)ceil_div(g.max_n, 32) * 32;
      if (el * (9 * np + 8 * 32 * 33) > dense_smem_limit()) return SymvSet{};  // the full GEMV then
      g.n = (int)v.size();
      g.d = m.upload(v, s);
      // split every matrix over enough CTAs to fill the resident slots evenly
      const int occ = h.mixed() ? symv_occupancy<float>(g.max_n) : symv_occupancy<double>(g.max_n);
      g.split = symv_split(g.n, g.max_n, sms * occ);
      if (g.split > 1) {
        g.ld_scr = (int)np;
        g.scratch = m.alloc<unsigned char>(el * (size_t)g.n * g.split * g.ld_scr);
        g.counter = m.alloc<int>(g.n);
        ck(cudaMemsetAsync(g.counter, 0, sizeof(int) * g.n, s), "memset counters");
      }
      return g;
    };
    h.sv_schur = sset(s_schur);
    h.sv_local = sset(s_local);
    // bytes read by the products of one application (the profile's library bytes)
    if (h.sv_schur.n) {
      h.gemv_schur_bytes = 0.0;
      for (auto &t : s_schur) h.gemv_schur_bytes += (double)sym_tile_entries(t.n);
    }
    if (h.sv_local.n) {
      h.gemv_local_bytes = 0.0;
      for (auto &t : s_local) h.gemv_local_bytes += (double)sym_tile_entries(t.n);
      for (auto &t : g_psi) h.gemv_local_bytes += (double)t.rows * t.cols;
    }
  }
  h.gv_psit = gset(g_psit);
  h.gv_sdd = gset(g_sdd);
  h.gv_lgi = gset(g_lgi);
  h.gv_lgit = gset(g_lgit);

  {
    CoarseSolve &c = h.cs;
    c.np = h.np;
    c.gauge = h.gauge_primal;
    // refinement steps: one restores FP64 backward stability of an FP64 explicit inverse
    // (small problems: refined to FP64 once per Jacobian); from the FP32 inverse of a large
    // problem in BD_MIXED each step gains about -log10(u32 cond(S_PP)) digits (2.7 on the
    // 128x128x32 slab, where the fourth step reaches the FP64 floor)
    c.X64 = h.d_CoInv64;
    c.nref = (h.mixed() && !c.X64) ? 4 : 1;
    c.pl_ptr = h.d_pl_ptr;
    c.pl_idx = h.d_pl_idx;
    c.sptr = h.d_co_rptr;
    c.scol = h.d_co_col;
    c.sval = h.d_Co64;
    c.ld_x = pad8(h.np);
  }
  h.cp_sorig = cset(c_sorig);
  h.cp_sdd = cset(c_sdd);
  h.cp_zx = cset(c_zx);
  h.cp_blk = cset(cp_blk);
  h.cp_sinv = cset(cp_sinv);
  {
    CopyTask c{};
    c.src_off = 0; c.src_ld = h.ld_co; c.r0 = c.c0 = h.np; c.rows = c.cols = h.np; c.mode = 3; c.sign = -1.0;
    c.dst_off = 0; c.dst_ld = pad8(h.np);  // rows of the inverse 32-byte aligned (vector loads)
    h.cp_coinv = cset({c});
  }
  {  // the dense kernels stage vectors and tiles in shared memory
    const size_t el = h.mixed() ? sizeof(float) : sizeof(double);
    size_t need = el * (6 * 32 * 33 + (size_t)h.shK.max_e + 4);
    for (const GemvSet *g : {&h.gv_schur, &h.gv_local, &h.gv_psit, &h.gv_sdd, &h.gv_lgi, &h.gv_lgit, &h.gv_drest,
                             &h.gv_dext})
      need = std::max(need, el * (size_t)std::max(g->max_rows, g->max_cols));
    need = std::max(need, el * (size_t)pad8(h.np));  // the coarse GEMV stages the coarse vector
    if (need > dense_smem_limit())
      throw Status(BD_ERR_ARG, "local problem too large for the shared-memory staging of the dense kernels (" +
                                   std::to_string(need) + " bytes); use more subdomains");
  }
  // ---- dense buffers
  auto alloc_dense = [&](auto &D) {
    using T = std::remove_pointer_t<decltype(D.K)>;
    D.K = m.alloc<T>(h.K_el);
    D.Aug = m.alloc<T>(h.A_el);
    D.Sorig = m.alloc<T>(h.So_el);
    D.Z = m.alloc<T>(h.Z_el);
    D.SDD = m.alloc<T>(h.SDD_el);
    D.Blk = m.alloc<T>(h.Blk_el);
    D.CA = m.alloc<T>(h.CA_el);
    D.Sinv = m.alloc<T>(h.Sinv_el);
    D.Dd = m.alloc<T>(h.Dd_el);
    D.Linv = m.alloc<T>((size_t)std::max({h.A_blk, h.C_blk, 1}) * kNB * kNB);
    D.LdK = m.alloc<T>((size_t)std::max(h.K_blk, 1) * kNB * kNB);
    D.Co = m.alloc<T>((size_t)h.ld_co * 2 * h.np);
    D.LdCo = m.alloc<T>((size_t)std::max(1, ceil_div(h.np, kNB)) * kNB * kNB);
    D.CoInv = m.alloc<T>((size_t)h.np * pad8(h.np));
    ck(cudaMemsetAsync(D.CoInv, 0, sizeof(T) * (size_t)h.np * pad8(h.np), s), "memset");  // zero padding
  };
  if (h.mixed()) alloc_dense(h.df);
  else alloc_dense(h.dd);
  // ---- work vectors
  h.d_fI = m.alloc<double>(h.nI_tot); h.d_yI = m.alloc<double>(h.nI_tot);
  h.d_fG = m.alloc<double>(h.nif); h.d_fhat = m.alloc<double>(h.nif); h.d_uG = m.alloc<double>(h.nif);
  h.d_yloc = m.alloc<double>(h.nG_tot);
  h.d_rbar = m.alloc<double>(h.nd + h.np); h.d_zbar = m.alloc<double>(h.nd + h.np);
  h.d_rD = m.alloc<double>(h.nD_tot); h.d_rD2 = m.alloc<double>(h.nD_tot);
  h.d_ydc = m.alloc<double>(h.nD_tot + h.nP_tot);
  h.d_w1 = m.alloc<double>(h.nD_tot); h.d_w2 = m.alloc<double>(h.nD_tot);
  h.d_gP = m.alloc<double>(h.nP_tot);
  h.d_crhs = m.alloc<double>(h.np); h.d_rP = m.alloc<double>(h.np);
  const int kn = std::max(h.nif, h.nlam);
  double **kv[] = {&h.d_kx, &h.d_kr, &h.d_kz, &h.d_kp, &h.d_kq, &h.d_kb};
  for (double **v : kv) *v = m.alloc<double>(kn);
  h.d_ks = m.alloc<KrylovState>(1);
  h.d_counter = m.alloc<unsigned int>(1);
  ck(cudaMemsetAsync(h.d_counter, 0, sizeof(unsigned int), s), "memset");
  if (h.opt.krylov == BD_GMRES) {
    const int mr = std::min(std::max(h.opt.gmres_restart, 1), kMaxRestart);
    h.opt.gmres_restart = mr;
    h.d_gs = m.alloc<GmresState>(1);
    h.d_gV = m.alloc<double>((size_t)(mr + 1) * kn);
    h.d_gz = m.alloc<double>(kn);
    h.d_gt = m.alloc<double>(kn);
    h.d_gpart = m.alloc<double>((size_t)(kMaxRestart + 1) * 32);
    h.d_gh = m.alloc<double>(3 * (kMaxRestart + 1));
  }
  h.hist_cap = std::max(1, h.opt.ksp_max_it) + 2;
  h.d_ha = m.alloc<double>(2 * (size_t)h.hist_cap);  // alphas then betas
  h.d_hb = h.d_ha + h.hist_cap;
  const int io = std::max({2 * N, h.nif, h.nlam});
  for (int i = 0; i < 6; ++i) h.d_io[i] = m.alloc<double>(io);
  if (h.opt.learned_guess) setup_mlp(h);
  ck(cudaStreamSynchronize(s), "setup");
}

// ---------------------------------------------------------------------------
// Jacobian: local matrices, factorisations, Schur complements, deluxe, coarse
// ---------------------------------------------------------------------------
// The subdomain batch is factorised in tune_groups consecutive groups (smaller
// groups keep their trailing matrices in L2).
template <class T>
void run_engine_groups(bd_handle &h, const EngineShape &all, const MatDesc *d_desc, T *base, T *linv) {
  const int G = std::max(1, std::min(h.tune_groups, all.count));
  const int per = (all.count + G - 1) / G;
  for (int a = 0; a < all.count; a += per) {
    const int b = std::min(all.count, a + per);
    EngineShape g{b - a, 0, 0, {}, {}};
    g.ob = h.tune_ob;
    for (int q = a; q < b; ++q) {
      g.m.push_back(all.m[q]);
      g.e.push_back(all.e[q]);
      if (!all.band.empty()) g.band.push_back(all.band[q]);
      if (!all.id0.empty()) g.id0.push_back(all.id0[q]);
      if (!all.ifirst.empty()) g.ifirst.push_back(all.ifirst[q]);
      g.max_m = std::max(g.max_m, all.m[q]);
      g.max_e = std::max(g.max_e, all.e[q]);
    }
    engine_partial_cholesky<T>(g, d_desc + a, base, h.d_err, h.s, linv, &h.prof, h.opt.use_tensor_cores != 0,
                               h.tune_panel_tc ? h.d_pinv : nullptr);
  }
}

// precond = false: only the operator (local factors and Schur complements); the
// BDDC preconditioner built from an earlier Jacobian stays in place.
template <class T>
void linearize_t(bd_handle &h, Dense<T> &D, bool precond) {
  cudaStream_t s = h.s;
  ck(cudaMemsetAsync(D.K, 0, sizeof(T) * h.K_el, s), "memset K");
  launch_assemble_local<T>(h.nq, h.d_q_sub, h.d_q_loc, h.d_q_node, h.d_q_nbr, h.d_q_stencil, h.d_q_mass, h.d_factor,
                           h.tau, h.d_Kdesc, D.K, s);
  run_engine_groups<T>(h, h.shK, h.d_Kdesc, D.K, D.LdK);
  launch_copy<T, T>(h.cp_sorig.n, h.cp_sorig.max_elems, h.cp_sorig.d, D.K, D.Sorig, s);
  if (!precond) return;
  const T *tval;
  if constexpr (std::is_same<T, float>::value) tval = h.d_tl_valf;
  else tval = h.d_tl_val;
  launch_build_aug<T>(h.nsub, h.shA.max_m, h.d_Sdesc, D.Sorig, h.d_Adesc, D.Aug, h.d_nD, h.d_tl_off, h.d_tl_ptr,
                      h.d_tl_row, tval, s);
  launch_copy<T, T>(h.cp_sdd.n, h.cp_sdd.max_elems, h.cp_sdd.d, D.Aug, D.SDD, s);
  launch_copy<T, T>(h.cp_blk.n, h.cp_blk.max_elems, h.cp_blk.d, D.Aug, D.Blk, s);
  run_engine_groups<T>(h, h.shA, h.d_Adesc, D.Aug, D.Linv);
  launch_copy<T, T>(h.cp_zx.n, h.cp_zx.max_elems, h.cp_zx.d, D.Aug, D.Z, s);
  launch_class_aug<T>(h.ncls, h.max_nc, h.d_cls, h.d_pairs, D.Blk, h.d_Cdesc, D.CA, s);
  engine_partial_cholesky<T>(h.shC, h.d_Cdesc, D.CA, h.d_err, s, D.Linv, &h.prof, h.opt.use_tensor_cores != 0,
                             h.tune_panel_tc ? h.d_pinv : nullptr);
  launch_copy<T, T>(h.cp_sinv.n, h.cp_sinv.max_elems, h.cp_sinv.d, D.CA, D.Sinv, s);
  if (h.opt.scaling == BD_SCALING_RHO) {
    const double si = std::max({h.fp.sigma_i[0], h.fp.sigma_i[1], h.fp.sigma_i[2]});
    const double se = std::max({h.fp.sigma_e[0], h.fp.sigma_e[1], h.fp.sigma_e[2]});
    launch_rho_blocks<T>(h.ncls, h.d_cls, h.d_pairs, si, se, D.Sinv, D.Blk, s);
  }
  launch_small_gemm<T>(h.n_gemm, h.max_nc, h.d_gemm, D.Sinv, D.Blk, D.Dd, s);
  // coarse: S_PiPi assembled in FP64 (sparse) and, in the local precision, into the augmented
  // matrix whose partial Cholesky leaves the explicit inverse; the solve refines against FP64
  ck(cudaMemsetAsync(D.Co, 0, sizeof(T) * (size_t)h.ld_co * 2 * h.np, s), "memset coarse");
  if (h.d_Co64d) ck(cudaMemsetAsync(h.d_Co64d, 0, sizeof(double) * (size_t)h.np * h.np, s), "memset coarse");
  launch_coarse_assemble<T>(h.co_nnz, h.np, h.gauge_primal, h.d_co_row, h.d_co_col, h.d_co_sptr, h.d_co_src, D.Aug,
                            h.d_Co64, D.Co, h.ld_co, h.d_Co64d, s);
  {  // one large matrix: its trailing updates go to the tensor cores like the local ones
    EngineShape co = h.shCo;
    co.ob = h.tune_ob;
    engine_partial_cholesky<T>(co, h.d_Codesc, D.Co, h.d_err, s, D.LdCo, &h.prof, h.opt.use_tensor_cores != 0,
                               h.tune_panel_tc ? h.d_pinv : nullptr);
  }
  launch_copy<T, T>(h.cp_coinv.n, h.cp_coinv.max_elems, h.cp_coinv.d, D.Co, D.CoInv, s);
  if (h.d_CoInv64) coarse_refine64<T>(h.np, D.CoInv, pad8(h.np), h.d_Co64d, h.d_CoInv64, h.d_CoW, h.d_CoY, s);
}

// counted = true for the Jacobian evaluations of the solve (Newton, bidomain_linearize):
// with precond_every = k the preconditioner is rebuilt when their count is a multiple of k.
void linearize(bd_handle &h, bool counted = false) {
  h.prof.begin(PROF_LINEARIZE, h.s);
  bool precond = true;
  if (counted) {
    precond = h.n_jac % std::max(1, h.opt.precond_every) == 0;
    ++h.n_jac;
  }
  if (h.mixed()) linearize_t(h, h.df, precond);
  else linearize_t(h, h.dd, precond);
  h.prof.end(PROF_LINEARIZE, h.s, 0.0, 0.0);
  h.linearized = true;
}

// ---- operators (device vectors; `done` = early-exit flag of a Krylov loop) ----
template <class T>
// f: the PCG reduction to fuse into the last kernel (nullptr: none)
void schur_t(bd_handle &h, Dense<T> &D, const double *x, double *y, const int *done, const DotFuse *f = nullptr) {
  h.prof.begin(PROF_GEMV, h.s);
  if (h.sv_schur.n)
    launch_symv<T>(h.sv_schur, D.Sorig, x, h.d_R, h.d_yloc, done, h.s);
  else
    launch_gemv<T>(h.gv_schur.n, h.gv_schur.max_rows, h.gv_schur.max_cols, h.gv_schur.d, D.Sorig, x, h.d_R,
                   h.d_yloc, 1.0, done, h.s);
  h.prof.end(PROF_GEMV, h.s, h.gemv_schur_flops, h.gemv_schur_bytes * sizeof(T));
  if (f) launch_gather_sum_dot(h.nif, h.d_Rt_ptr, h.d_Rt_idx, h.d_yloc, y, h.gauge_iface, *f, h.s);
  else launch_gather_sum(h.nif, h.d_Rt_ptr, h.d_Rt_idx, h.d_yloc, y, h.gauge_iface, 1.0, nullptr, done, h.s);
}

// St^-1 applied to (primal part rP or 0, local dual parts rD): zbar[nd:] = z_Pi, ydc[0:nD_tot] = z_Delta.
// rP_csr: the primal part as a sparse product instead (rP unused).
template <class T>
void st_inv_t(bd_handle &h, Dense<T> &D, const double *rP, const double *rD, const int *done,
              const CsrIn *rP_csr = nullptr) {
  h.prof.begin(PROF_GEMV, h.s);
  if (h.sv_local.n) {
    // Psi^T r_Delta first: the coarse solve needs only it, so it runs on the second stream
    // while X r_Delta (the symmetric product) runs here
    launch_gemv<T>(h.gv_psi.n, h.gv_psi.max_rows, h.gv_psi.max_cols, h.gv_psi.d, D.Z, rD, nullptr, h.d_ydc, 1.0,
                   done, h.s);
    ck(cudaEventRecord(h.ev_fork, h.s), "record");
    ck(cudaStreamWaitEvent(h.s2, h.ev_fork, 0), "wait");
    launch_coarse_solve<T>(h.cs, D.CoInv, h.d_ydc + h.nD_tot, rP_csr ? nullptr : rP, rP_csr, h.d_zbar + h.nd,
                           h.d_co_c, h.d_co_rho, done, h.s2);
    ck(cudaEventRecord(h.ev_join, h.s2), "record");
    launch_symv<T>(h.sv_local, D.Z, rD, nullptr, h.d_ydc, done, h.s);
    h.prof.end(PROF_GEMV, h.s, h.gemv_local_flops, h.gemv_local_bytes * sizeof(T));
    ck(cudaStreamWaitEvent(h.s, h.ev_join, 0), "wait");
  } else {
    launch_gemv<T>(h.gv_local.n, h.gv_local.max_rows, h.gv_local.max_cols, h.gv_local.d, D.Z, rD, nullptr,
                   h.d_ydc, 1.0, done, h.s);
    h.prof.end(PROF_GEMV, h.s, h.gemv_local_flops, h.gemv_local_bytes * sizeof(T));
    // z_Pi = S_PiPi^-1 (rP - sum_j Psi^T r_D) into zbar[nd:]
    launch_coarse_solve<T>(h.cs, D.CoInv, h.d_ydc + h.nD_tot, rP_csr ? nullptr : rP, rP_csr, h.d_zbar + h.nd,
                           h.d_co_c, h.d_co_rho, done, h.s);
  }
  // ydc_Delta -= Psi z_Pi
  launch_gemv_t_task<T>(h.gv_psit.n, h.gv_psit.max_rows, h.gv_psit.max_cols, h.gv_psit.d, D.Z, h.d_zbar,
                        h.d_prim_x, h.d_ydc, -1.0, done, h.s);
}

// rbar = T^T r is never stored: the deluxe restriction evaluates its dual rows while
// staging, the coarse right-hand side its primal rows (row nd + gauge_primal is
// zeroed there).  f: the PCG reduction to fuse into the last kernel.
template <class T>
void bddc_t(bd_handle &h, Dense<T> &D, const double *r, double *z, const int *done, const DotFuse *f = nullptr) {
  const CsrIn rbar{h.d_Tt_ptr, h.d_Tt_col, h.d_Tt_val, r};
  const CsrIn rbar_p{h.d_Tt_ptr + h.nd, h.d_Tt_col, h.d_Tt_val, r};
  // deluxe restriction r_C^(j) = D_C^(j)T rbar_C
  launch_gemv_t_task<T>(h.gv_drest.n, h.gv_drest.max_rows, h.gv_drest.max_cols, h.gv_drest.d, D.Dd, nullptr,
                        nullptr, h.d_rD, 1.0, done, h.s, &rbar);
  st_inv_t(h, D, nullptr, h.d_rD, done, &rbar_p);
  // deluxe extension zbar_C = sum_j D_C^(j) z_C^(j) (one row of [D^(j1) | D^(j2) | ...] per output)
  launch_gemv_task<T>(h.gv_dext.n, h.gv_dext.max_rows, h.gv_dext.max_cols, h.gv_dext.d, D.Dd, h.d_ydc,
                      h.d_ext_idx, h.d_zbar, 1.0, done, h.s);
  if (f) launch_spmv_dot(h.nif, h.d_T_ptr, h.d_T_col, h.d_T_val, h.d_zbar, z, h.gauge_iface, *f, h.s);
  else launch_spmv(h.nif, h.d_T_ptr, h.d_T_col, h.d_T_val, h.d_zbar, z, h.gauge_iface, done, h.s);
}

template <class T>
void feti_F_t(bd_handle &h, Dense<T> &D, const double *lam, double *y, const int *done) {
  launch_jump_t(h.nwt, h.max_nc, h.d_wt, h.d_went, lam, h.d_w1, done, h.s);
  st_inv_t(h, D, nullptr, h.d_w1, done);
  launch_jump(h.nlt, h.max_nc, h.d_lt, h.d_pairs, h.d_ydc, y, done, h.s);
}

template <class T>
void feti_M_t(bd_handle &h, Dense<T> &D, const double *mu, double *y, const int *done) {
  launch_jump_dt<T>(h.nwt, h.max_nc, h.d_wt, h.d_went, D.Blk, D.Sinv, mu, h.d_w1, done, h.s);
  launch_gemv<T>(h.gv_sdd.n, h.gv_sdd.max_rows, h.gv_sdd.max_cols, h.gv_sdd.d, D.SDD, h.d_w1, nullptr, h.d_w2, 1.0,
                 done, h.s);
  launch_jump_d<T>(h.nlt, h.max_nc, h.d_lt, h.d_pairs, D.Blk, D.Sinv, h.d_w2, y, done, h.s);
}

#define DISPATCH(H, fn, ...) ((H).mixed() ? fn((H), (H).df, __VA_ARGS__) : fn((H), (H).dd, __VA_ARGS__))

// ---- device-side PCG ---------------------------------------------------------
constexpr int kChunk = 8;

template <class Op, class Pc, class OpF, class PcF>
int pcg(bd_handle &h, int n, const double *b, double *x, Op A, Pc M, bd_solve_stats *st, OpF AF, PcF MF) {
  cudaStream_t s = h.s;
  KrylovState ks{};
  ks.rtol = std::min(h.opt.ksp_rtol * h.rtol_scale, 0.1);
  ks.atol = h.opt.ksp_atol;
  ks.dtol = h.opt.ksp_dtol;
  ks.maxit = h.opt.ksp_max_it;
  ks.hist_cap = h.hist_cap;
  ck(cudaMemcpyAsync(h.d_ks, &ks, sizeof(ks), cudaMemcpyHostToDevice, s), "ks");
  const int *done = &h.d_ks->done;
  launch_fill(n, x, 0.0, s);
  launch_copy_vec(n, b, h.d_kr, nullptr, s);
  M(h.d_kr, h.d_kz, nullptr);
  launch_dot2(n, h.d_kr, h.d_kz, h.d_kz, h.d_kz, h.d_partial, h.d_scal, nullptr, s);
  launch_pcg_start(h.d_ks, h.d_scal, s);
  launch_copy_vec(n, h.d_kz, h.d_kp, done, s);
  KrylovState out{};
  auto body = [&]() {
    // AF / MF apply the operator / preconditioner with the following reduction fused
    // into their last kernel and return true, or return false to leave it separate
    const DotFuse f0{0, h.d_kp, h.d_partial, h.d_counter, h.d_ks, h.d_ha};
    const DotFuse f1{1, h.d_kr, h.d_partial, h.d_counter, h.d_ks, h.d_ha};
    for (int c = 0; c < kChunk; ++c) {
      if (!AF(h.d_kp, h.d_kq, done, f0)) {
        A(h.d_kp, h.d_kq, done);
        launch_pcg_dot_step(n, 0, h.d_kp, h.d_kq, nullptr, nullptr, h.d_partial, h.d_counter, h.d_ks, h.d_ha, s);
      }
      launch_pcg_xr(n, h.d_ks, h.d_kp, h.d_kq, x, h.d_kr, s);
      if (!MF(h.d_kr, h.d_kz, done, f1)) {
        M(h.d_kr, h.d_kz, done);
        launch_pcg_dot_step(n, 1, h.d_kr, h.d_kz, h.d_kz, h.d_kz, h.d_partial, h.d_counter, h.d_ks, h.d_ha, s);
      }
      launch_pcg_p(n, h.d_ks, h.d_kz, h.d_kp, s);
    }
  };
  const int key = h.opt.method == BD_FETIDP ? 1 : 0;
  if (h.opt.use_graphs && !h.pcg_exec[key]) {
    // capture one chunk of iterations once; every launch reads fixed handle buffers
    const int prof_on = h.prof.on;
    h.prof.on = 0;
    const long long l0 = launch_count();
    cudaGraph_t g = nullptr;
    ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture");
    body();
    ck(cudaStreamEndCapture(s, &g), "capture end");
    count_launch((int)(l0 - launch_count()));
    ck(cudaGraphGetNodes(g, nullptr, &h.pcg_nodes[key]), "graph nodes");
    ck(cudaGraphInstantiate(&h.pcg_exec[key], g, 0), "graph instantiate");
    cudaGraphDestroy(g);
    h.prof.on = prof_on;
  }
  for (int it = 0; it <= h.opt.ksp_max_it; it += kChunk) {
    if (h.opt.use_graphs) {
      ck(cudaGraphLaunch(h.pcg_exec[key], s), "graph launch");
      count_launch((int)h.pcg_nodes[key]);
    } else {
      body();
    }
    ck(cudaGetLastError(), "pcg launch");
    ck(cudaMemcpyAsync(&out, h.d_ks, sizeof(out), cudaMemcpyDeviceToHost, s), "ks read");
    ck(cudaStreamSynchronize(s), "pcg sync");
    if (out.done) break;
  }
  if (!out.done) out.reason = BD_ERR_KRYLOV_MAXIT;
  if (st) {
    st->its = out.it;
    st->reason = out.reason;
    st->res0 = out.zn0;
    st->res = out.zn;
    st->cond = 0.0;
    const int k = std::min(out.it, h.hist_cap);
    if (k > 0) {
      std::vector<double> a(k), bb(std::max(k - 1, 1));
      ck(cudaMemcpy(a.data(), h.d_ha, sizeof(double) * k, cudaMemcpyDeviceToHost), "hist");
      if (k > 1) ck(cudaMemcpy(bb.data(), h.d_hb, sizeof(double) * (k - 1), cudaMemcpyDeviceToHost), "hist");
      std::vector<double> d(k), e(std::max(k - 1, 0));
      for (int i = 0; i < k; ++i) {
        d[i] = 1.0 / a[i] + (i > 0 ? bb[i - 1] / a[i - 1] : 0.0);
        if (i + 1 < k) e[i] = std::sqrt(bb[i]) / a[i];
      }
      st->cond = tridiag_cond(d, e);
    }
  }
  return out.reason;
}

// ---- device-side GMRES(m) (left preconditioning, CGS2) -------------------------
template <class Op, class Pc>
int gmres(bd_handle &h, int n, const double *b, double *x, Op A, Pc M, bd_solve_stats *st) {
  cudaStream_t s = h.s;
  const int m = h.opt.gmres_restart;
  GmresState init{};
  init.rtol = std::min(h.opt.ksp_rtol * h.rtol_scale, 0.1);
  init.atol = h.opt.ksp_atol;
  init.dtol = h.opt.ksp_dtol;
  init.restart = m;
  init.maxit = h.opt.ksp_max_it;
  ck(cudaMemcpyAsync(h.d_gs, &init, sizeof(init), cudaMemcpyHostToDevice, s), "gmres state");
  const int *stop = &h.d_gs->stop;
  double *h1 = h.d_gh, *h2 = h.d_gh + (kMaxRestart + 1), *zz = h.d_gh + 2 * (kMaxRestart + 1);
  launch_fill(n, x, 0.0, s);
  M(b, h.d_gz, nullptr);
  launch_dot2(n, h.d_gz, h.d_gz, nullptr, nullptr, h.d_partial, h.d_scal, nullptr, s);
  launch_gmres_begin(n, h.d_gz, h.d_gV, h.d_gs, h.d_scal, 1, s);
  GmresState out{};
  for (;;) {
    for (int j = 0; j < m; ++j) {
      A(h.d_gV + (long long)j * n, h.d_gt, stop);
      M(h.d_gt, h.d_gz, stop);
      launch_gmres_step(n, j, h.d_gV, h.d_gz, h.d_gpart, h1, h2, zz, h.d_gs, s);
    }
    launch_gmres_end(n, h.d_gV, x, h.d_gs, s);
    ck(cudaGetLastError(), "gmres launch");
    ck(cudaMemcpyAsync(&out, h.d_gs, sizeof(out), cudaMemcpyDeviceToHost, s), "gmres read");
    ck(cudaStreamSynchronize(s), "gmres sync");
    if (out.converged || out.reason != 0) break;
    // restart from r = M^-1 (b - A x)
    A(x, h.d_gt, nullptr);
    launch_axpby(n, 1.0, b, -1.0, h.d_gt, s);
    M(h.d_gt, h.d_gz, nullptr);
    launch_dot2(n, h.d_gz, h.d_gz, nullptr, nullptr, h.d_partial, h.d_scal, nullptr, s);
    launch_gmres_begin(n, h.d_gz, h.d_gV, h.d_gs, h.d_scal, 0, s);
  }
  if (st) {
    st->its = out.its;
    st->reason = out.reason;
    st->res0 = out.res0;
    st->res = out.res;
    st->cond = 0.0;
  }
  return out.reason;
}

// ---- Jacobian solve J s = f (f = (fi, fe) device SoA) ---------------------------
template <class T>
int solve_t(bd_handle &h, Dense<T> &D, const double *fi, const double *fe, double *si, double *se,
            bd_solve_stats *st) {
  cudaStream_t s = h.s;
  // interior data: y_I = L_II^-1 f_I
  launch_gather_pairs(h.nint_nodes, h.d_int_node, fi, fe, h.d_fI, 1.0, nullptr, s);
  h.prof.begin(PROF_TRSV, s);
  launch_trsv<T>(h.nsub, h.shK.max_e, h.d_Kdesc, h.d_vec_off_I, D.K, D.LdK, h.d_fI, h.d_yI, false, s);
  h.prof.end(PROF_TRSV, s, 0.0, 0.0);
  launch_gemv<T>(h.gv_lgi.n, h.gv_lgi.max_rows, h.gv_lgi.max_cols, h.gv_lgi.d, D.K, h.d_yI, nullptr, h.d_yloc, 1.0,
                 nullptr, s);
  launch_gather_pairs(h.nif / 2, h.d_iface_node, fi, fe, h.d_fG, 1.0, nullptr, s);
  int reason;
  if (h.opt.method == BD_BDDC) {
    // f_hat = f_G - sum_j R_j^T L_GI y_I  (= K_GI K_II^-1 f_I)
    launch_gather_sum(h.nif, h.d_Rt_ptr, h.d_Rt_idx, h.d_yloc, h.d_fhat, h.gauge_iface, -1.0, h.d_fG, nullptr, s);
    auto A = [&](const double *x, double *y, const int *dn) { schur_t(h, D, x, y, dn); };
    auto M = [&](const double *x, double *y, const int *dn) { bddc_t(h, D, x, y, dn); };
    auto AF = [&](const double *x, double *y, const int *dn, const DotFuse &f) {
      schur_t(h, D, x, y, dn, &f);
      return true;
    };
    auto MF = [&](const double *x, double *y, const int *dn, const DotFuse &f) {
      bddc_t(h, D, x, y, dn, &f);
      return true;
    };
    h.prof.begin(PROF_KRYLOV, s);
    reason = h.opt.krylov == BD_GMRES ? gmres(h, h.nif, h.d_fhat, h.d_uG, A, M, st)
                                      : pcg(h, h.nif, h.d_fhat, h.d_uG, A, M, st, AF, MF);
    h.prof.end(PROF_KRYLOV, s, 0.0, 0.0);
  } else {
    // f~: local g = f_G[R] / mult - L_GI y_I, gbar = T_loc^T g -> (rD, gP); rP = sum gP
    launch_gather_scale_sub(h.nG_tot, h.d_R, h.d_fG, h.d_mult_iface, h.d_yloc, s);
    launch_tloc_t(h.nt_tot, h.d_tl_sub, h.d_tl_loc, h.d_tl_ptr, h.d_tl_row, h.d_tl_val, h.d_giff_off, h.d_yloc,
                  h.d_nD, h.d_ldual_off, h.d_lprim_off, h.d_rD2, h.d_gP, s);
    launch_gather_sum(h.np, h.d_pl_ptr, h.d_pl_idx, h.d_gP, h.d_rP, h.gauge_primal, 1.0, nullptr, nullptr, s);
    st_inv_t(h, D, h.d_rP, h.d_rD2, nullptr);
    launch_jump(h.nlt, h.max_nc, h.d_lt, h.d_pairs, h.d_ydc, h.d_kb, nullptr, s);
    auto A = [&](const double *x, double *y, const int *dn) { feti_F_t(h, D, x, y, dn); };
    auto M = [&](const double *x, double *y, const int *dn) { feti_M_t(h, D, x, y, dn); };
    auto unfused = [](const double *, double *, const int *, const DotFuse &) { return false; };
    h.prof.begin(PROF_KRYLOV, s);
    reason = h.opt.krylov == BD_GMRES ? gmres(h, h.nlam, h.d_kb, h.d_kx, A, M, st)
                                      : pcg(h, h.nlam, h.d_kb, h.d_kx, A, M, st, unfused, unfused);
    h.prof.end(PROF_KRYLOV, s, 0.0, 0.0);
    // w = St^-1 (f~ - B^T lambda); u_G = T (dual mean, primal)
    launch_jump_t(h.nwt, h.max_nc, h.d_wt, h.d_went, h.d_kx, h.d_w1, nullptr, s);
    launch_axpby(h.nD_tot, 1.0, h.d_rD2, -1.0, h.d_w1, s);
    st_inv_t(h, D, h.d_rP, h.d_w1, nullptr);
    launch_dual_mean(h.ncls, h.max_nc, h.d_cls, h.d_pairs, h.d_ydc, h.d_zbar, s);
    launch_spmv(h.nif, h.d_T_ptr, h.d_T_col, h.d_T_val, h.d_zbar, h.d_uG, h.gauge_iface, nullptr, s);
  }
  // interior recovery: u_I = L_II^-T (y_I - L_GI^T u_G)
  launch_gemv_t<T>(h.gv_lgit.n, h.gv_lgit.max_rows, h.gv_lgit.max_cols, h.gv_lgit.d, D.K, h.d_uG, h.d_R, h.d_yI, -1.0,
                   nullptr, s);
  h.prof.begin(PROF_TRSV, s);
  launch_trsv<T>(h.nsub, h.shK.max_e, h.d_Kdesc, h.d_vec_off_I, D.K, D.LdK, h.d_yI, h.d_fI, true, s);
  h.prof.end(PROF_TRSV, s, 0.0, 0.0);
  launch_scatter_pairs(h.nint_nodes, h.d_int_node, h.d_fI, si, se, s);
  launch_scatter_pairs(h.nif / 2, h.d_iface_node, h.d_uG, si, se, s);
  ck(cudaGetLastError(), "solve");
  return reason;
}

int solve(bd_handle &h, const double *fi, const double *fe, double *si, double *se, bd_solve_stats *st) {
  return h.mixed() ? solve_t(h, h.df, fi, fe, si, se, st) : solve_t(h, h.dd, fi, fe, si, se, st);
}

StimParams stim_params(const bd_handle &h, const bd_stimulus *st, double t_next) {
  StimParams sp{};
  for (int d = 0; d < 3; ++d) { sp.h[d] = h.plan.h[d]; sp.o[d] = h.plan.origin[d]; }
  if (st) {
    sp.amp = st->amp;
    for (int k = 0; k < 6; ++k) sp.box[k] = st->box[k];
    sp.active = (st->t_on <= t_next && t_next < st->t_off && st->amp != 0.0) ? 1 : 0;
  }
  return sp;
}

double read_scalar(bd_handle &h, const double *d) {
  double v = 0.0;
  ck(cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, h.s), "read scalar");
  ck(cudaStreamSynchronize(h.s), "sync");
  return v;
}

// residual at u + lam s into (rit, ret, factort, uit, uet); returns ||F - G||^2
double trial_residual(bd_handle &h, const StimParams &sp, const double *si, const double *se, double lam) {
  h.prof.begin(PROF_RESID, h.s);
  launch_residual(h.N, h.d_stencil, h.d_nbr, h.d_mass, h.d_node_ijk, h.d_ui, h.d_ue, si, se, lam, h.d_wn, h.d_uin,
                  h.d_uen, h.fp, sp, h.d_rit, h.d_ret, h.d_factort, h.d_uit, h.d_uet, h.d_partial, h.d_scal, h.s);
  // moved per node: 54 stencil values, 27 neighbour ids, M, w, u^n (2), u (2), s (2), i,j,k; written: r (2), factor, u (2)
  h.prof.end(PROF_RESID, h.s, 0.0, (double)h.N * (54 * 8 + 27 * 4 + 12 + 8 * (si ? 8 : 6) + 8 * 5));
  return read_scalar(h, h.d_scal);
}

// ---- learned guess: interior from the predicted interface increment --------------
// u0 = u^n + d with d_Gamma the network's prediction and d_I from the interior recovery
// of Section 4.1 with the factors of the last Jacobian: d_I = K_II^-1 (-r_I - K_IG d_Gamma),
// r = F(u^n) - G (in ri, re).  Writes u0 into (gi, ge).
template <class T>
void guess_interior_t(bd_handle &h, Dense<T> &D, int) {
  cudaStream_t s = h.s;
  launch_gather_pairs(h.nint_nodes, h.d_int_node, h.d_ri, h.d_re, h.d_fI, -1.0, nullptr, s);
  launch_trsv<T>(h.nsub, h.shK.max_e, h.d_Kdesc, h.d_vec_off_I, D.K, D.LdK, h.d_fI, h.d_yI, false, s);
  launch_gemv_t<T>(h.gv_lgit.n, h.gv_lgit.max_rows, h.gv_lgit.max_cols, h.gv_lgit.d, D.K, h.d_dG, h.d_R, h.d_yI, -1.0,
                   nullptr, s);
  launch_trsv<T>(h.nsub, h.shK.max_e, h.d_Kdesc, h.d_vec_off_I, D.K, D.LdK, h.d_yI, h.d_fI, true, s);
  launch_scatter_pairs(h.nint_nodes, h.d_int_node, h.d_fI, h.d_gi, h.d_ge, s);
  launch_scatter_pairs(h.nif / 2, h.d_iface_node, h.d_dG, h.d_gi, h.d_ge, s);
  launch_axpby(h.N, 1.0, h.d_uin, 1.0, h.d_gi, s);
  launch_axpby(h.N, 1.0, h.d_uen, 1.0, h.d_ge, s);
}

// ---- one time step (Sections 3b, 3c) -------------------------------------------
int step(bd_handle &h, const bd_stimulus *stim, bd_step_stats *out) {
  cudaStream_t s = h.s;
  const double t_next = (h.step_n + 1) * h.tau;
  const StimParams sp = stim_params(h, stim, t_next);
  bd_step_stats st{};
  h.prof.begin(PROF_STEP, s);
  launch_gating(h.N, h.d_uin, h.d_uen, h.d_w, h.d_wn, h.fp, s);
  // u^0 = u^n (the fallback)
  ck(cudaMemcpyAsync(h.d_ui, h.d_uin, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
  ck(cudaMemcpyAsync(h.d_ue, h.d_uen, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
  double fn2 = trial_residual(h, sp, nullptr, nullptr, 0.0);
  std::swap(h.d_ui, h.d_uit); std::swap(h.d_ue, h.d_uet);
  std::swap(h.d_ri, h.d_rit); std::swap(h.d_re, h.d_ret); std::swap(h.d_factor, h.d_factort);
  // tolerances stay anchored to the fallback residual ||F(u^n) - G||
  const double fn0 = std::sqrt(fn2);
  st.res0 = fn0;
  h.rtol_scale = 1.0;
  if (h.mlp_on && h.hist_count >= 2) {
    // learned guess u^n + MLP(traces of u^n, u^{n-1}, u^{n-2}); kept only if its residual is smaller
    h.prof.begin(PROF_MLP, s);
    mlp_features(h.mlp, h.n_tr_ent, h.d_t_sub, h.d_t_pos, h.d_t_node, h.d_uin, h.d_uen, h.d_uh1i, h.d_uh1e,
                 h.d_uh2i, h.d_uh2e, nullptr, nullptr, s);
    mlp_forward(h.mlp, h.d_err, s);
    mlp_trace_increment(h.mlp, h.nif / 2, h.d_tr_ptr, h.d_tr_ent, h.d_dG, s);
    DISPATCH(h, guess_interior_t, 0);
    h.prof.end(PROF_MLP, s, 0.0, 0.0);
    std::swap(h.d_ui, h.d_gi); std::swap(h.d_ue, h.d_ge);  // residual at the guess
    const double g2 = trial_residual(h, sp, nullptr, nullptr, 0.0);
    std::swap(h.d_ui, h.d_gi); std::swap(h.d_ue, h.d_ge);
    st.res_guess = std::sqrt(g2);
    if (h.mlp_steps_trained >= h.opt.mlp_warmup && std::isfinite(g2) && g2 < fn2) {
      std::swap(h.d_ui, h.d_uit); std::swap(h.d_ue, h.d_uet);
      std::swap(h.d_ri, h.d_rit); std::swap(h.d_re, h.d_ret); std::swap(h.d_factor, h.d_factort);
      h.rtol_scale = std::min(fn0 / std::sqrt(std::max(g2, 1e-300)), 1e4);
      fn2 = g2;
      st.guess_used = 1;
    }
  }
  int reason = BD_OK;
  int k = 0;
  bool refresh = true;  // form J at the current iterate (always without lagging)
  for (; k < h.opt.newton_max_it; ++k) {
    if (!std::isfinite(fn2)) { reason = BD_ERR_NAN; break; }
    if (std::sqrt(fn2) <= std::max(h.opt.snes_atol, h.opt.snes_rtol * fn0)) break;
    const bool fresh = refresh || !h.opt.lag_jacobian;
    if (fresh) {
      linearize(h, true);
      int e = h.check_err();
      if (e) { reason = e; break; }
      refresh = false;
    }
    launch_axpby(h.N, -1.0, h.d_ri, 0.0, h.d_fi, s);
    launch_axpby(h.N, -1.0, h.d_re, 0.0, h.d_fe, s);
    bd_solve_stats ls{};
    int r = solve(h, h.d_fi, h.d_fe, h.d_si, h.d_se, &ls);
    h.rtol_scale = 1.0;
    st.krylov_its += ls.its;
    st.cond_max = std::max(st.cond_max, ls.cond);
    if (r != BD_OK) { reason = r; break; }
    // cubic backtracking line search on f = ||R||^2 / 2, slope = -||R||^2
    const double alpha = 1e-4, f0 = 0.5 * fn2, slope = -fn2;
    double lam = 1.0;
    double g = trial_residual(h, sp, h.d_si, h.d_se, lam);
    bool ok = 0.5 * g <= f0 + alpha * lam * slope;
    if (!ok) {
      double lam_prev = lam, f_prev = 0.5 * g;
      double lt = -slope / (2.0 * (0.5 * g - f0 - slope));
      lam = std::max(std::min(lt, 0.5 * lam), 0.1 * lam);
      for (int ls_it = 0; ls_it < 40 && !ok; ++ls_it) {
        if (lam < 1e-12) break;
        g = trial_residual(h, sp, h.d_si, h.d_se, lam);
        const double fl = 0.5 * g;
        if (fl <= f0 + alpha * lam * slope) { ok = true; break; }
        const double t1 = fl - f0 - lam * slope, t2 = f_prev - f0 - lam_prev * slope, dl = lam - lam_prev;
        const double a = (t1 / (lam * lam) - t2 / (lam_prev * lam_prev)) / dl;
        const double b = (-lam_prev * t1 / (lam * lam) + lam * t2 / (lam_prev * lam_prev)) / dl;
        if (a == 0.0) lt = -slope / (2.0 * b);
        else lt = (-b + std::sqrt(std::max(b * b - 3.0 * a * slope, 0.0))) / (3.0 * a);
        lam_prev = lam;
        f_prev = fl;
        lam = std::max(std::min(lt, 0.5 * lam), 0.1 * lam);
      }
    }
    if (!ok && !fresh) {  // a lagged Jacobian gave no descent: keep the iterate, form J here
      refresh = true;
      continue;
    }
    std::swap(h.d_ui, h.d_uit); std::swap(h.d_ue, h.d_uet);
    std::swap(h.d_ri, h.d_rit); std::swap(h.d_re, h.d_ret); std::swap(h.d_factor, h.d_factort);
    fn2 = g;
    if (!ok) { reason = BD_ERR_NEWTON; ++k; break; }
    // ||lam s|| <= stol ||u||
    launch_dot3(h.N, h.d_si, h.d_si, h.d_se, h.d_se, h.d_ui, h.d_ui, h.d_partial, h.d_scal, s);
    launch_dot3(h.N, h.d_ue, h.d_ue, h.d_ue, h.d_ue, h.d_ue, h.d_ue, h.d_partial, h.d_scal + 3, s);
    double sc[6];
    ck(cudaMemcpyAsync(sc, h.d_scal, sizeof(sc), cudaMemcpyDeviceToHost, s), "read");
    ck(cudaStreamSynchronize(s), "sync");
    const double snorm = lam * std::sqrt(sc[0] + sc[1]);
    const double unorm = std::sqrt(sc[2] + sc[3]);
    if (snorm <= h.opt.snes_stol * unorm) { ++k; break; }
  }
  if (k >= h.opt.newton_max_it && reason == BD_OK && !(std::sqrt(fn2) <= std::max(h.opt.snes_atol, h.opt.snes_rtol * fn0)))
    reason = BD_ERR_NEWTON;
  st.newton_its = k;
  st.res_final = std::sqrt(fn2);
  if (h.mlp_on && h.hist_count >= 2 && h.step_n < h.opt.mlp_train_steps && reason == BD_OK) {
    // online training on (traces, u^{n+1} - u^n), before the gauge shift
    h.prof.begin(PROF_MLP, s);
    MlpDev &M = h.mlp;
    ck(cudaMemsetAsync(M.T, 0, sizeof(float) * M.batch * M.n_out, s), "memset");
    ck(cudaMemsetAsync(M.mask, 0, sizeof(float) * M.batch * M.n_out, s), "memset");
    mlp_features(M, h.n_tr_ent, h.d_t_sub, h.d_t_pos, h.d_t_node, h.d_uin, h.d_uen, h.d_uh1i, h.d_uh1e,
                 h.d_uh2i, h.d_uh2e, h.d_ui, h.d_ue, s);
    for (int ep = 0; ep < std::max(1, h.opt.mlp_epochs); ++ep) mlp_train_once(h, ep == 0);
    h.prof.end(PROF_MLP, s, 0.0, 0.0);
    st.mlp_loss = read_scalar(h, h.d_scal + 4);
    h.mlp_steps_trained += 1;
  }
  if (h.mlp_on) {  // history of the last states (gauge as stored)
    ck(cudaMemcpyAsync(h.d_uh2i, h.d_uh1i, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
    ck(cudaMemcpyAsync(h.d_uh2e, h.d_uh1e, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
    ck(cudaMemcpyAsync(h.d_uh1i, h.d_uin, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
    ck(cudaMemcpyAsync(h.d_uh1e, h.d_uen, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
    h.hist_count = std::min(h.hist_count + 1, 2);
  }
  // gauge: zero lumped-mass mean of u_e, then u^n <- u, w <- w^{n+1}
  launch_dot3(h.N, h.d_mass, h.d_ue, h.d_mass, h.d_ue, h.d_mass, h.d_ue, h.d_partial, h.d_scal, s);
  launch_fill(1, h.d_scal + 1, h.sum_mass, s);
  launch_gauge_shift(h.N, h.d_ui, h.d_ue, h.d_scal, s);
  ck(cudaMemcpyAsync(h.d_uin, h.d_ui, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
  ck(cudaMemcpyAsync(h.d_uen, h.d_ue, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
  ck(cudaMemcpyAsync(h.d_w, h.d_wn, sizeof(double) * h.N, cudaMemcpyDeviceToDevice, s), "copy");
  h.prof.end(PROF_STEP, s, 0.0, 0.0);
  ck(cudaStreamSynchronize(s), "step");
  if (h.prof.on) h.prof.harvest();
  h.step_n += 1;
  st.reason = reason;
  if (out) *out = st;
  return reason;
}

// ---- host / device pointer helpers ------------------------------------------------
const double *in_ptr(bd_handle &h, const double *p, size_t n, int on_device, int slot) {
  if (on_device) return p;
  ck(cudaMemcpyAsync(h.d_io[slot], p, n * sizeof(double), cudaMemcpyHostToDevice, h.s), "h2d");
  return h.d_io[slot];
}
double *out_ptr(bd_handle &h, double *p, int on_device, int slot) { return on_device ? p : h.d_io[slot]; }
void finish_out(bd_handle &h, double *host, const double *dev, size_t n, int on_device) {
  if (!on_device) ck(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, h.s), "d2h");
  ck(cudaStreamSynchronize(h.s), "sync");
}

thread_local std::string g_last_error;

template <class F>
int guard(bd_handle *h, F &&f) {
  try {
    return f();
  } catch (const Status &e) {
    g_last_error = e.what();
    if (h) h->last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc &) {
    return BD_ERR_NOMEM;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    return BD_ERR_ARG;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// schur_apply_noalloc: the S_hat x product of schur_apply with its scratch (the
// per-subdomain products S_Gamma^(j) R_j x before interface assembly) in a
// file-scope device array instead of the handle's cudaMalloc'd buffer.  For
// callers that must not allocate device memory when they apply the operator,
// e.g. code that runs under a fixed device-memory budget or inside a host
// framework that owns every allocation.  Capacity: kNoAllocScratch doubles
// (4 MiB, held by every GPU that loads this library until the process exits).
// ---------------------------------------------------------------------------
static constexpr long long kNoAllocScratch = 1LL << 19;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

namespace {

// Device address of the scratch array on device `dev`, looked up once per device
// with that device current (the host-side symbol is only a stand-in, not an address).
int noalloc_scratch(int dev, double **out) {
  static std::mutex mu;
  static std::map<int, double *> addr;
  std::lock_guard<std::mutex> lock(mu);
  auto it = addr.find(dev);
  if (it == addr.end()) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return BD_ERR_CUDA;
    it = addr.emplace(dev, static_cast<double *>(p)).first;
  }
  *out = it->second;
  return BD_OK;
}

template <class T>
void schur_noalloc_t(bd_handle &h, Dense<T> &D, const double *x, double *y, double *scratch) {
  if (h.sv_schur.n)
    launch_symv<T>(h.sv_schur, D.Sorig, x, h.d_R, scratch, nullptr, h.s);
  else
    launch_gemv<T>(h.gv_schur.n, h.gv_schur.max_rows, h.gv_schur.max_cols, h.gv_schur.d, D.Sorig, x, h.d_R,
                   scratch, 1.0, nullptr, h.s);
  launch_gather_sum(h.nif, h.d_Rt_ptr, h.d_Rt_idx, scratch, y, h.gauge_iface, 1.0, nullptr, nullptr, h.s);
}

}  // namespace

extern "C" int schur_apply_noalloc(bd_handle *h, const double *x, double *y) {
  if (!h || !x || !y) return BD_ERR_ARG;
  auto fail = [&](int code, const std::string &msg) {
    h->last_error = "schur_apply_noalloc: " + msg;
    return code;
  };
  if (!h->linearized) return fail(BD_ERR_STATE, "no Jacobian yet (call bidomain_linearize or bidomain_step)");
  if ((long long)h->nG_tot > kNoAllocScratch)
    return fail(BD_ERR_SCRATCH, std::to_string(h->nG_tot) + " interface unknowns over the subdomains exceed " +
                                    std::to_string(kNoAllocScratch));
  // the scratch address is per device: it must be the handle's, which must be current
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(BD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != h->device)
    return fail(BD_ERR_STATE, "device " + std::to_string(dev) + " is current, the handle lives on device " +
                                  std::to_string(h->device));
  double *scratch = nullptr;
  if (noalloc_scratch(dev, &scratch) != BD_OK) return fail(BD_ERR_CUDA, "cudaGetSymbolAddress failed");
  if (h->mixed()) schur_noalloc_t(*h, h->df, x, y, scratch);
  else schur_noalloc_t(*h, h->dd, x, y, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  if (e != cudaSuccess) return fail(BD_ERR_CUDA, cudaGetErrorString(e));
  return BD_OK;
}

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

static Geometry mesh_geometry(const bd_mesh &m) {
  Geometry g;
  g.kind = m.geometry;
  for (int k = 0; k < 6; ++k) g.axes[k] = m.axes[k];
  for (int k = 0; k < 2; ++k) { g.phi[k] = m.phi[k]; g.theta[k] = m.theta[k]; }
  return g;
}

int bd_plan_create(const bd_mesh *mesh, int primal, bd_plan **out) {
  if (!mesh || !out) return BD_ERR_ARG;
  return guard(nullptr, [&] {
    auto pl = std::make_unique<bd_plan>();
    std::string err = build_plan(pl->p, mesh->n, mesh->l, mesh->s, mesh->elem_mask, primal, mesh_geometry(*mesh));
    if (!err.empty()) { g_last_error = err; return BD_ERR_ARG; }
    *out = pl.release();
    return BD_OK;
  });
}

static int fill_sizes(const Plan &p, bd_sizes *o) {
  o->n_node = p.n_node; o->n_elem = p.n_elem; o->n_sub = p.n_sub; o->n_cls = p.n_cls;
  o->n_iface = p.n_iface(); o->n_dual = p.n_dual; o->n_primal = p.n_primal;
  long long nl = 0;
  for (int c = 0; c < p.n_cls; ++c) {
    const long long k = p.cls_sub_ptr[c + 1] - p.cls_sub_ptr[c];
    nl += 2LL * p.cls_dual_nodes[c] * (k * (k - 1) / 2);
  }
  o->n_lambda = (int)nl;
  o->gauge_node = p.gauge_node; o->gauge_primal = p.gauge_primal;
  return BD_OK;
}

int bd_plan_sizes(const bd_plan *plan, bd_sizes *out) {
  if (!plan || !out) return BD_ERR_ARG;
  return fill_sizes(plan->p, out);
}

static int index_sets(const Plan &p, int which, int64_t *out, int64_t cap, int64_t *len) {
  std::vector<int64_t> v;
  auto add = [&](const std::vector<int> &x) { v.insert(v.end(), x.begin(), x.end()); };
  switch (which) {
    case BD_IDX_ELEM_SUB: add(p.elem_sub); break;
    case BD_IDX_NODE_MULT: add(p.mult); break;
    case BD_IDX_IFACE_NODES: add(p.iface_nodes); break;
    case BD_IDX_CLS_TYPE: add(p.cls_type); break;
    case BD_IDX_CLS_PTR: add(p.cls_ptr); break;
    case BD_IDX_CLS_NODES: add(p.cls_nodes); break;
    case BD_IDX_CLS_SUB_PTR: add(p.cls_sub_ptr); break;
    case BD_IDX_CLS_SUBS: add(p.cls_subs); break;
    case BD_IDX_CLS_DUAL_START: add(p.cls_dual_start); break;
    case BD_IDX_SUB_NODE_PTR: {
      v.push_back(0);
      for (auto &sp : p.subs) v.push_back(v.back() + (int64_t)sp.nodes.size());
      break;
    }
    case BD_IDX_SUB_NODES: for (auto &sp : p.subs) add(sp.nodes); break;
    case BD_IDX_SUB_NINT: for (auto &sp : p.subs) v.push_back(sp.n_interior); break;
    case BD_IDX_SUB_DUAL_PTR: {
      v.push_back(0);
      for (auto &sp : p.subs) v.push_back(v.back() + (int64_t)sp.dual.size());
      break;
    }
    case BD_IDX_SUB_DUAL: for (auto &sp : p.subs) add(sp.dual); break;
    case BD_IDX_SUB_PRIMAL_PTR: {
      v.push_back(0);
      for (auto &sp : p.subs) v.push_back(v.back() + (int64_t)sp.primal.size());
      break;
    }
    case BD_IDX_SUB_PRIMAL: for (auto &sp : p.subs) add(sp.primal); break;
    case BD_IDX_GAUGE: v.push_back(p.gauge_node); v.push_back(p.gauge_primal); break;
    default: return BD_ERR_ARG;
  }
  if (len) *len = (int64_t)v.size();
  if (!out) return BD_OK;
  if (cap < (int64_t)v.size()) return BD_ERR_ARG;
  std::copy(v.begin(), v.end(), out);
  return BD_OK;
}

int bd_plan_index_sets(const bd_plan *plan, int which, int64_t *out, int64_t cap, int64_t *len) {
  if (!plan) return BD_ERR_ARG;
  return index_sets(plan->p, which, out, cap, len);
}

void bd_plan_destroy(bd_plan *plan) { delete plan; }

int bd_options_default(bd_options *o) {
  if (!o) return BD_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->method = BD_BDDC;
  o->krylov = BD_PCG;
  o->primal = BD_PRIMAL_VE;
  o->precision = BD_FP64;
  o->gmres_restart = 30;
  o->ksp_max_it = 1000;
  o->newton_max_it = 50;
  o->use_graphs = 0;
  o->ksp_rtol = 1e-8; o->ksp_atol = 1e-10; o->ksp_dtol = 1e4;
  o->snes_rtol = 1e-4; o->snes_atol = 1e-8; o->snes_stol = 1e-8;
  o->learned_guess = 0; o->mlp_train_steps = 200; o->mlp_warmup = 5; o->mlp_epochs = 4; o->mlp_lr = 1e-3;
  o->use_tensor_cores = 0;
  o->lag_jacobian = 0;
  o->scaling = BD_SCALING_DELUXE;
  o->precond_every = 1;
  return BD_OK;
}

int bidomain_setup(const bd_mesh *mesh, const bd_conductivity *cond, const bd_ionic *ionic, double tau,
                   const bd_options *opt, void *stream, bd_handle **out) {
  if (!mesh || !cond || !ionic || !out || !(tau > 0)) return BD_ERR_ARG;
  return guard(nullptr, [&] {
    auto h = std::make_unique<bd_handle>();
    if (opt) h->opt = *opt;
    else bd_options_default(&h->opt);
    const bd_options &o = h->opt;
    if ((o.method != BD_BDDC && o.method != BD_FETIDP) || (o.krylov != BD_PCG && o.krylov != BD_GMRES) ||
        (o.precision != BD_FP64 && o.precision != BD_MIXED) || o.ksp_max_it < 1 || o.newton_max_it < 1 ||
        (o.scaling != BD_SCALING_DELUXE && o.scaling != BD_SCALING_RHO) || o.precond_every < 1 ||
        (o.precond_every > 1 && o.method != BD_BDDC))
      return BD_ERR_ARG;
    std::string err = build_plan(h->plan, mesh->n, mesh->l, mesh->s, mesh->elem_mask, o.primal,
                                 mesh_geometry(*mesh));
    if (!err.empty()) { g_last_error = err; return BD_ERR_ARG; }
    h->tau = tau;
    for (int d = 0; d < 3; ++d) { h->fp.sigma_i[d] = cond->sigma_i[d]; h->fp.sigma_e[d] = cond->sigma_e[d]; }
    h->fp.G = ionic->G; h->fp.eta1 = ionic->eta1; h->fp.eta2 = ionic->eta2; h->fp.vth = ionic->vth;
    h->fp.vp = ionic->vp; h->fp.chi_cm = ionic->chi_cm; h->fp.tau = tau;
    ck(cudaGetDevice(&h->device), "cudaGetDevice");
    if (stream) h->s = (cudaStream_t)stream;
    else { ck(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking), "stream"); h->own_stream = true; }
    ck(cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking), "stream");
    ck(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "event");
    ck(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming), "event");
    if (h->opt.use_tensor_cores && h->opt.precision == BD_MIXED && !tc_configure()) {
      g_last_error = "tensor-core kernel configuration failed";
      return BD_ERR_CUDA;
    }
    if (h->opt.precision != BD_MIXED) h->opt.use_tensor_cores = 0;
    h->tune_panel_tc = h->opt.use_tensor_cores == 2 ? 1 : 0;
    if (h->opt.learned_guess && !gemm_tc_configure()) {
      g_last_error = "tensor-core GEMM configuration failed";
      return BD_ERR_CUDA;
    }
    if (!dense_configure()) {
      g_last_error = "dense kernel configuration failed";
      return BD_ERR_CUDA;
    }
    setup_handle(*h);
    *out = h.release();
    return BD_OK;
  });
}

int bidomain_sizes(const bd_handle *h, bd_sizes *out) {
  if (!h || !out) return BD_ERR_ARG;
  return fill_sizes(h->plan, out);
}

int bidomain_index_sets(const bd_handle *h, int which, int64_t *out, int64_t cap, int64_t *len) {
  if (!h) return BD_ERR_ARG;
  return index_sets(h->plan, which, out, cap, len);
}

int bidomain_set_state(bd_handle *h, const double *ui, const double *ue, const double *w, double t, int on_device) {
  if (!h || !ui || !ue || !w) return BD_ERR_ARG;
  return guard(h, [&] {
    const size_t n = h->N;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ck(cudaMemcpyAsync(h->d_uin, ui, n * sizeof(double), k, h->s), "state");
    ck(cudaMemcpyAsync(h->d_uen, ue, n * sizeof(double), k, h->s), "state");
    ck(cudaMemcpyAsync(h->d_w, w, n * sizeof(double), k, h->s), "state");
    ck(cudaStreamSynchronize(h->s), "sync");
    const long step = std::lround(t / h->tau);
    if (step != h->step_n) h->hist_count = 0;  // the learned guess's history belongs to another time
    h->step_n = step;
    return BD_OK;
  });
}

int bidomain_get_state(bd_handle *h, double *ui, double *ue, double *w, double *t, int on_device) {
  if (!h) return BD_ERR_ARG;
  return guard(h, [&] {
    const size_t n = h->N;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (ui) ck(cudaMemcpyAsync(ui, h->d_uin, n * sizeof(double), k, h->s), "state");
    if (ue) ck(cudaMemcpyAsync(ue, h->d_uen, n * sizeof(double), k, h->s), "state");
    if (w) ck(cudaMemcpyAsync(w, h->d_w, n * sizeof(double), k, h->s), "state");
    ck(cudaStreamSynchronize(h->s), "sync");
    if (t) *t = h->step_n * h->tau;
    return BD_OK;
  });
}

int bidomain_step(bd_handle *h, const bd_stimulus *stim, bd_step_stats *stats) {
  if (!h) return BD_ERR_ARG;
  return guard(h, [&] { return step(*h, stim, stats); });
}

int bidomain_gating(bd_handle *h, const double *ui, const double *ue, const double *w, double *w_next,
                    int on_device) {
  if (!h || !ui || !ue || !w || !w_next) return BD_ERR_ARG;
  return guard(h, [&] {
    const size_t n = h->N;
    const double *a = in_ptr(*h, ui, n, on_device, 0), *b = in_ptr(*h, ue, n, on_device, 1),
                 *c = in_ptr(*h, w, n, on_device, 2);
    double *o = out_ptr(*h, w_next, on_device, 3);
    launch_gating(h->N, a, b, c, o, h->fp, h->s);
    finish_out(*h, w_next, o, n, on_device);
    return BD_OK;
  });
}

int bidomain_residual(bd_handle *h, const bd_stimulus *stim, double t_next, const double *ui, const double *ue,
                      const double *w_next, const double *ui_n, const double *ue_n, double *r, int on_device) {
  if (!h || !ui || !ue || !w_next || !ui_n || !ue_n || !r) return BD_ERR_ARG;
  return guard(h, [&] {
    const size_t n = h->N;
    const double *a = in_ptr(*h, ui, n, on_device, 0), *b = in_ptr(*h, ue, n, on_device, 1),
                 *c = in_ptr(*h, w_next, n, on_device, 2), *d = in_ptr(*h, ui_n, n, on_device, 3),
                 *e = in_ptr(*h, ue_n, n, on_device, 4);
    double *o = out_ptr(*h, r, on_device, 5);
    launch_residual(h->N, h->d_stencil, h->d_nbr, h->d_mass, h->d_node_ijk, a, b, nullptr, nullptr, 0.0, c, d, e,
                    h->fp, stim_params(*h, stim, t_next), o, o + n, nullptr, nullptr, nullptr, h->d_partial,
                    nullptr, h->s);
    finish_out(*h, r, o, 2 * n, on_device);
    return BD_OK;
  });
}

int bidomain_linearize(bd_handle *h, const double *ui, const double *ue, const double *w_next, int on_device) {
  if (!h || !ui || !ue || !w_next) return BD_ERR_ARG;
  return guard(h, [&] {
    const size_t n = h->N;
    const double *a = in_ptr(*h, ui, n, on_device, 0), *b = in_ptr(*h, ue, n, on_device, 1),
                 *c = in_ptr(*h, w_next, n, on_device, 2);
    launch_residual(h->N, h->d_stencil, h->d_nbr, h->d_mass, h->d_node_ijk, a, b, nullptr, nullptr, 0.0, c, a, b,
                    h->fp, stim_params(*h, nullptr, 0.0), h->d_rit, h->d_ret, h->d_factor, nullptr, nullptr,
                    h->d_partial, nullptr, h->s);
    linearize(*h, true);
    return h->check_err();
  });
}

int schur_apply(bd_handle *h, const double *x, double *y, int on_device) {
  if (!h || !x || !y) return BD_ERR_ARG;
  if (!h->linearized) return BD_ERR_STATE;
  return guard(h, [&] {
    const double *a = in_ptr(*h, x, h->nif, on_device, 0);
    double *o = out_ptr(*h, y, on_device, 1);
    DISPATCH(*h, schur_t, a, o, nullptr);
    finish_out(*h, y, o, h->nif, on_device);
    return BD_OK;
  });
}

int bddc_apply(bd_handle *h, const double *r, double *z, int on_device) {
  if (!h || !r || !z) return BD_ERR_ARG;
  if (!h->linearized) return BD_ERR_STATE;
  return guard(h, [&] {
    const double *a = in_ptr(*h, r, h->nif, on_device, 0);
    double *o = out_ptr(*h, z, on_device, 1);
    DISPATCH(*h, bddc_t, a, o, nullptr);
    finish_out(*h, z, o, h->nif, on_device);
    return BD_OK;
  });
}

int fetidp_apply(bd_handle *h, const double *lambda, double *mu, int on_device) {
  if (!h || !lambda || !mu) return BD_ERR_ARG;
  if (!h->linearized) return BD_ERR_STATE;
  return guard(h, [&] {
    const double *a = in_ptr(*h, lambda, h->nlam, on_device, 0);
    double *o = out_ptr(*h, mu, on_device, 1);
    DISPATCH(*h, feti_M_t, a, o, nullptr);
    finish_out(*h, mu, o, h->nlam, on_device);
    return BD_OK;
  });
}

int fetidp_operator(bd_handle *h, const double *lambda, double *y, int on_device) {
  if (!h || !lambda || !y) return BD_ERR_ARG;
  if (!h->linearized) return BD_ERR_STATE;
  return guard(h, [&] {
    const double *a = in_ptr(*h, lambda, h->nlam, on_device, 0);
    double *o = out_ptr(*h, y, on_device, 1);
    DISPATCH(*h, feti_F_t, a, o, nullptr);
    finish_out(*h, y, o, h->nlam, on_device);
    return BD_OK;
  });
}

int krylov_solve(bd_handle *h, const double *f, double *s, int on_device, bd_solve_stats *stats) {
  if (!h || !f || !s) return BD_ERR_ARG;
  if (!h->linearized) return BD_ERR_STATE;
  return guard(h, [&] {
    const size_t n = h->N;
    const double *a = in_ptr(*h, f, 2 * n, on_device, 0);
    double *o = out_ptr(*h, s, on_device, 1);
    int r = solve(*h, a, a + n, o, o + n, stats);
    finish_out(*h, s, o, 2 * n, on_device);
    if (r == BD_OK) r = h->check_err();
    return r;
  });
}

int bidomain_mlp_sizes(bd_handle *h, int *n_in, int *n_hidden, int *n_out, int *batch) {
  if (!h) return BD_ERR_ARG;
  if (!h->mlp_on) return BD_ERR_STATE;
  if (n_in) *n_in = h->mlp.n_in;
  if (n_hidden) *n_hidden = h->mlp.n_hidden;
  if (n_out) *n_out = h->mlp.n_out;
  if (batch) *batch = h->mlp.batch;
  return BD_OK;
}

int bidomain_mlp_params(bd_handle *h, float *w, int set) {
  if (!h || !w) return BD_ERR_ARG;
  if (!h->mlp_on) return BD_ERR_STATE;
  return guard(h, [&] {
    MlpDev &M = h->mlp;
    if (set) {
      ck(cudaMemcpyAsync(M.w, w, sizeof(float) * M.n_params, cudaMemcpyHostToDevice, h->s), "mlp params");
      mlp_refresh_bf16(M, h->s);
    } else {
      ck(cudaMemcpyAsync(w, M.w, sizeof(float) * M.n_params, cudaMemcpyDeviceToHost, h->s), "mlp params");
    }
    ck(cudaStreamSynchronize(h->s), "sync");
    return BD_OK;
  });
}

int bidomain_mlp_loss_grad(bd_handle *h, const float *X, const float *T, const float *mask, double *loss,
                           float *grad) {
  if (!h || !X || !T || !mask) return BD_ERR_ARG;
  if (!h->mlp_on) return BD_ERR_STATE;
  return guard(h, [&] {
    MlpDev &M = h->mlp;
    const size_t nx = (size_t)M.batch * M.n_in, ny = (size_t)M.batch * M.n_out;
    std::vector<float> mk(mask, mask + ny);
    double cnt = 0.0;
    for (float v : mk) cnt += v;
    ck(cudaMemcpyAsync(M.Xf, X, sizeof(float) * nx, cudaMemcpyHostToDevice, h->s), "mlp X");
    ck(cudaMemcpyAsync(M.T, T, sizeof(float) * ny, cudaMemcpyHostToDevice, h->s), "mlp T");
    ck(cudaMemcpyAsync(M.mask, mask, sizeof(float) * ny, cudaMemcpyHostToDevice, h->s), "mlp mask");
    mlp_inputs_from_f32(M, h->s);
    mlp_forward(M, h->d_err, h->s);
    mlp_backward(M, (float)(1.0 / std::max(cnt, 1.0)), h->d_partial, h->d_err, h->s);
    launch_sum_partials(kRedBlocks, h->d_partial, h->d_scal + 4, h->s);
    if (loss) *loss = read_scalar(*h, h->d_scal + 4);
    if (grad) ck(cudaMemcpyAsync(grad, M.g, sizeof(float) * M.n_params, cudaMemcpyDeviceToHost, h->s), "grad");
    ck(cudaStreamSynchronize(h->s), "sync");
    return BD_OK;
  });
}

int bidomain_coarse_size(bd_handle *h, int *n_primal, int *nnz) {
  if (!h) return BD_ERR_ARG;
  if (n_primal) *n_primal = h->np;
  if (nnz) *nnz = h->co_nnz;
  return BD_OK;
}

int bidomain_coarse_matrix(bd_handle *h, int *rowptr, int *col, double *val) {
  if (!h || !rowptr || !col || !val) return BD_ERR_ARG;
  if (!h->linearized) return BD_ERR_STATE;
  return guard(h, [&] {
    ck(cudaMemcpyAsync(rowptr, h->d_co_rptr, sizeof(int) * (h->np + 1), cudaMemcpyDeviceToHost, h->s), "coarse");
    ck(cudaMemcpyAsync(col, h->d_co_col, sizeof(int) * h->co_nnz, cudaMemcpyDeviceToHost, h->s), "coarse");
    ck(cudaMemcpyAsync(val, h->d_Co64, sizeof(double) * h->co_nnz, cudaMemcpyDeviceToHost, h->s), "coarse");
    ck(cudaStreamSynchronize(h->s), "sync");
    return BD_OK;
  });
}

int bidomain_coarse_solve(bd_handle *h, const double *c, double *z, int nref) {
  if (!h || !c || !z) return BD_ERR_ARG;
  if (!h->linearized) return BD_ERR_STATE;
  return guard(h, [&] {
    CoarseSolve cs = h->cs;
    cs.pl_ptr = h->d_co_noptr;  // no local products: c itself is the right-hand side
    if (nref >= 0) cs.nref = nref;
    double *dc = h->d_io[0], *dz = h->d_io[1];
    ck(cudaMemcpyAsync(dc, c, sizeof(double) * h->np, cudaMemcpyHostToDevice, h->s), "coarse c");
    if (h->mixed())
      launch_coarse_solve<float>(cs, h->df.CoInv, h->d_ydc, dc, nullptr, dz, h->d_co_c, h->d_co_rho, nullptr, h->s);
    else
      launch_coarse_solve<double>(cs, h->dd.CoInv, h->d_ydc, dc, nullptr, dz, h->d_co_c, h->d_co_rho, nullptr, h->s);
    ck(cudaMemcpyAsync(z, dz, sizeof(double) * h->np, cudaMemcpyDeviceToHost, h->s), "coarse z");
    ck(cudaStreamSynchronize(h->s), "sync");
    return BD_OK;
  });
}

int bidomain_mlp_adam_step(bd_handle *h, const float *grad, double lr) {
  if (!h || !grad) return BD_ERR_ARG;
  if (!h->mlp_on) return BD_ERR_STATE;
  return guard(h, [&] {
    MlpDev &M = h->mlp;
    ck(cudaMemcpyAsync(M.g, grad, sizeof(float) * M.n_params, cudaMemcpyHostToDevice, h->s), "mlp grad");
    mlp_adam(M, (float)lr, h->s);
    ck(cudaStreamSynchronize(h->s), "sync");
    return BD_OK;
  });
}

int bidomain_mlp_reset(bd_handle *h) {
  if (!h) return BD_ERR_ARG;
  if (!h->mlp_on) return BD_ERR_STATE;
  return guard(h, [&] {
    mlp_init_weights(*h);
    ck(cudaStreamSynchronize(h->s), "sync");
    return BD_OK;
  });
}

int bidomain_autotune(bd_handle *h, bd_tune_result *out) {
  if (!h) return BD_ERR_ARG;
  if (!h->linearized) return BD_ERR_STATE;
  return guard(h, [&] {
    cudaStream_t s = h->s;
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0), "event");
    ck(cudaEventCreate(&e1), "event");
    const int prof_on = h->prof.on;
    h->prof.on = 0;
    const int tc0 = h->opt.use_tensor_cores ? 1 + h->tune_panel_tc : 0, ob0 = h->tune_ob, g0 = h->tune_groups;
    auto set_tc = [&](int tc) {  // 0 SIMT, 1 tensor-core updates, 2 also the panel solves
      h->opt.use_tensor_cores = tc > 0;
      h->tune_panel_tc = tc == 2 && h->d_pinv;
    };
    auto time_it = [&]() {
      linearize(*h);  // warm
      float best = 1e30f;
      for (int r = 0; r < 2; ++r) {
        ck(cudaEventRecord(e0, s), "event");
        linearize(*h);
        ck(cudaEventRecord(e1, s), "event");
        ck(cudaEventSynchronize(e1), "event");
        float ms = 0.f;
        ck(cudaEventElapsedTime(&ms, e0, e1), "event");
        best = std::min(best, ms);
      }
      return best;
    };
    const float base_ms = time_it();
    float best_ms = base_ms;
    int best_ob = ob0, best_g = g0, best_tc = tc0, n = 0;
    for (int tc : {0, 1, 2}) {
      if (tc && !h->mixed()) continue;
      if (tc == 2 && !h->d_pinv) continue;
      for (int ob : {128, 256, 512})
        for (int g : {1, 2, 4}) {
          set_tc(tc);
          h->tune_ob = ob;
          h->tune_groups = g;
          const float ms = time_it();
          ++n;
          if (ms < best_ms) { best_ms = ms; best_ob = ob; best_g = g; best_tc = tc; }
        }
    }
    set_tc(best_tc);
    h->tune_ob = best_ob;
    h->tune_groups = best_g;
    linearize(*h);
    h->prof.on = prof_on;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int st = h->check_err();
    if (out) {
      out->outer_panel = best_ob;
      out->groups = best_g;
      out->tensor_cores = best_tc;
      out->candidates = n;
      out->best_ms = best_ms;
      out->default_ms = base_ms;
    }
    return st;
  });
}

int bidomain_profile(bd_handle *h, int enable) {
  if (!h) return BD_ERR_ARG;
  return guard(h, [&] {
    ck(cudaStreamSynchronize(h->s), "sync");
    h->prof.reset();
    h->prof.on = (enable == 1 || enable == 2) ? enable : 0;
    return BD_OK;
  });
}

int bidomain_profile_read(bd_handle *h, int which, double *out) {
  if (!h || !out || which < 0 || which >= PROF_NCLASS) return BD_ERR_ARG;
  return guard(h, [&] {
    ck(cudaStreamSynchronize(h->s), "sync");
    h->prof.harvest();
    for (int k = 0; k < 4; ++k) out[k] = h->prof.tot[which][k];
    return BD_OK;
  });
}

int64_t bidomain_launch_count(void) { return (int64_t)launch_count(); }

int bidomain_destroy(bd_handle *h) {
  if (!h) return BD_ERR_ARG;
  cudaStreamSynchronize(h->s);
  if (h->s2) cudaStreamSynchronize(h->s2);
  cudaStream_t s = h->s, s2 = h->s2;
  cudaEvent_t e1 = h->ev_fork, e2 = h->ev_join;
  const bool own = h->own_stream;
  for (auto &g : h->pcg_exec)
    if (g) cudaGraphExecDestroy(g);
  delete h;
  if (e1) cudaEventDestroy(e1);
  if (e2) cudaEventDestroy(e2);
  if (s2) cudaStreamDestroy(s2);
  if (own) cudaStreamDestroy(s);
  return BD_OK;
}

const char *bidomain_last_error(const bd_handle *h) {
  return h ? h->last_error.c_str() : g_last_error.c_str();
}

const char *bidomain_strerror(int status) {
  switch (status) {
    case BD_OK: return "ok";
    case BD_ERR_ARG: return "invalid argument";
    case BD_ERR_NOT_SPD: return "local matrix not positive definite (non-positive pivot)";
    case BD_ERR_KRYLOV_MAXIT: return "Krylov method reached the iteration limit";
    case BD_ERR_KRYLOV_DIVERGED: return "Krylov method diverged";
    case BD_ERR_NEWTON: return "Newton iteration or line search failed";
    case BD_ERR_NAN: return "NaN or Inf encountered";
    case BD_ERR_TIMEOUT: return "device wait exceeded its budget";
    case BD_ERR_CUDA: return "CUDA runtime error";
    case BD_ERR_NOMEM: return "out of device memory";
    case BD_ERR_STATE: return "call made in the wrong order";
    case BD_ERR_SCRATCH: return "problem exceeds the static scratch of the no-allocation entry point";
    default: return "unknown status";
  }
}

}  // extern "C"
