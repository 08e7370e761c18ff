// Batched dense kernels: partial Cholesky engine, GEMV, triangular solves.
//
// The engine is a right-looking blocked Cholesky restricted to the first e
// columns of each matrix, followed by one long-K symmetric rank-e update of
// the trailing block.  With K = [[K_II, K_IG], [K_GI, K_GG]] and e = n_I this
// yields L_II, L_GI and the local Schur complement S_Gamma = K_GG - L_GI L_GI^T
// (static condensation, Section 4.1).  With the augmented matrix
// [[S_DD, S_DP, I], [S_PD, S_PP, 0], [I, 0, 0]] and e = n_D it yields, in the
// trailing block, S_PP - S_PD S_DD^-1 S_DP (the local coarse matrix of
// Section 4.4), -S_DD^-1 S_DP and -S_DD^-1 (the local constrained solve).
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <vector>

#include "kernels.cuh"

namespace bd {

template <typename T> __device__ inline T dsqrt(T v);
template <> __device__ inline float dsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ inline double dsqrt<double>(double v) { return sqrt(v); }

// ---- panel step 1: factor the w x w diagonal block in place and form L_kk^-1 --
// 1024 threads per matrix: thread (r, t) owns entry (r, t) of the block.  Step c
// updates the trailing entries with the unscaled column c divided by its pivot,
// so one barrier per column suffices; the columns are scaled at the end.
// Warp 0 then forms L_kk^-1 (lane j solves L y = e_j) for the panel solve.
template <typename T>
__global__ void __launch_bounds__(1024) k_potrf(const MatDesc *__restrict__ desc, T *__restrict__ base, int k0,
                                                int *__restrict__ err, T *__restrict__ linv) {
  const MatDesc d = desc[blockIdx.x];
  if (k0 >= d.e) return;
  const int w = min(kNB, d.e - k0);
  T *A = base + d.off;
  __shared__ T Ls[kNB][kNB + 1];
  __shared__ T piv[kNB];
  const int r = threadIdx.x >> 5, t = threadIdx.x & 31;
  Ls[r][t] = (r < w && t <= r) ? A[(long long)(k0 + r) * d.ld + k0 + t] : (r == t ? T(1) : T(0));
  __syncthreads();
  bool bad = false;
  for (int c = 0; c < w; ++c) {
    T dcc = Ls[c][c];
    if (!(dcc > T(0))) { bad = true; dcc = T(1); }
    if (r == c && t == c) piv[c] = dcc;
    if (t > c && r >= t && r < w) Ls[r][t] -= Ls[r][c] * Ls[t][c] / dcc;
    __syncthreads();
  }
  if (bad && threadIdx.x == 0) atomicOr(err, DEV_ERR_NOT_SPD);
  // scale: L[r][c] = A_c[r][c] / sqrt(d_c), L[c][c] = sqrt(d_c)
  T lv = T(0);
  if (r < w && t <= r) lv = (r == t) ? dsqrt(piv[t]) : Ls[r][t] / dsqrt(piv[t]);
  else if (r == t) lv = T(1);
  __syncthreads();
  Ls[r][t] = lv;
  __syncthreads();
  if (r < w && t <= r) A[(long long)(k0 + r) * d.ld + k0 + t] = lv;
  // L_kk^-1 by recursive doubling: inv([[A, 0], [B, C]]) = [[A^-1, 0], [-C^-1 B A^-1, C^-1]]
  __shared__ T Yi[kNB][kNB + 1];
  __shared__ T Tm[kNB][kNB + 1];
  Yi[r][t] = (r == t) ? T(1) / Ls[r][r] : T(0);
  __syncthreads();
  for (int b = 1; b < kNB; b <<= 1) {
    const int base0 = (r / (2 * b)) * (2 * b);
    const bool active = (t / (2 * b) == r / (2 * b)) && ((r - base0) >= b) && ((t - base0) < b);
    if (active) {  // Tm = B A^-1 over the top half
      T acc = T(0);
      for (int k = t; k < base0 + b; ++k) acc += Ls[r][k] * Yi[k][t];
      Tm[r][t] = acc;
    }
    __syncthreads();
    if (active) {  // Y = -C^-1 (B A^-1) over the bottom half
      T acc = T(0);
      for (int k = base0 + b; k <= r; ++k) acc += Yi[r][k] * Tm[k][t];
      Yi[r][t] = -acc;
    }
    __syncthreads();
  }
  linv[(long long)blockIdx.x * kNB * kNB + r * kNB + t] = Yi[r][t];
}

// ---- panel step 2: rows below the diagonal block, x = a L_kk^-T ----------------
// 128 rows per CTA; the 128 x 32 tile is staged in shared memory with coalesced
// loads (warp q reads rows, lane = column) and each thread forms one row.
template <typename T>
__global__ void __launch_bounds__(128) k_trsm(const MatDesc *__restrict__ desc, T *__restrict__ base, int k0,
                                              const T *__restrict__ linv) {
  const MatDesc d = desc[blockIdx.y];
  if (k0 >= d.e) return;
  const int w = min(kNB, d.e - k0);
  const int rbeg = k0 + w + blockIdx.x * 128;
  if (rbeg >= d.m) return;
  T *A = base + d.off;
  __shared__ T Li[kNB][kNB];
  __shared__ T X[128][kNB + 1];
  const T *src = linv + (long long)blockIdx.y * kNB * kNB;
  for (int t = threadIdx.x; t < kNB * kNB; t += 128) Li[t / kNB][t % kNB] = src[t];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nrows = min(128, d.m - rbeg);
  for (int q = wid; q < nrows; q += 4)
    X[q][lane] = (lane < w) ? A[(long long)(rbeg + q) * d.ld + k0 + lane] : T(0);
  __syncthreads();
  if (threadIdx.x < nrows) {
    T x[kNB];
#pragma unroll
    for (int c = 0; c < kNB; ++c) x[c] = X[threadIdx.x][c];
    // x_out[c] = sum_{t <= c} x[t] (L^-1)[c][t]: independent dot products
#pragma unroll
    for (int c = kNB - 1; c >= 0; --c) {
      T v = T(0);
#pragma unroll
      for (int t = 0; t <= c; ++t) v += x[t] * Li[c][t];
      x[c] = v;
    }
#pragma unroll
    for (int c = 0; c < kNB; ++c) X[threadIdx.x][c] = x[c];
  }
  __syncthreads();
  for (int q = wid; q < nrows; q += 4)
    if (lane < w) A[(long long)(rbeg + q) * d.ld + k0 + lane] = X[q][lane];
}

// ---- rank-k update of lower tiles --------------------------------------------
// Two-level right-looking blocking: inner panels of kNB columns inside outer
// panels [K0, K1) of kOB columns.
// mode 0 (inner): rows [k0+w, m), cols [k0+w, min(K1, e)), K = [k0, k0+w)
// mode 2 (outer): rows [K1, m),   cols [K1, e),            K = [K0, K1)
// mode 1 (final): rows [e, m),    cols [e, m),             K = [0, e)
// C[r][c] -= sum_k A[r][k] A[c][k]; 64x64 tiles, 256 threads, 4x4 per thread.
constexpr int kTB = 64, kKC = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_rankk(const MatDesc *__restrict__ desc, T *__restrict__ base, int mode,
                                               int k0, int K0, int K1, int nct) {
  const MatDesc d = desc[blockIdx.y];
  int row0, colend, kb, ke;
  if (mode == 0) {
    if (k0 >= d.e) return;
    const int w = min(kNB, d.e - k0);
    row0 = k0 + w;
    colend = min(K1, d.e);
    kb = k0;
    ke = k0 + w;
  } else if (mode == 2) {
    if (K1 >= d.e) return;
    row0 = K1;
    colend = d.e;
    kb = K0;
    ke = K1;
  } else {
    row0 = d.e;
    colend = d.m;
    kb = 0;
    ke = d.e;
  }
  const int ti = blockIdx.x / nct, tj = blockIdx.x % nct;
  if (tj > ti) return;
  const int r0 = row0 + ti * kTB, c0 = row0 + tj * kTB;
  if (r0 >= d.m || c0 >= colend || ke <= kb) return;
  T *A = base + d.off;
  __shared__ T As[kKC][kTB + 1];  // row pad 65: the strided stores below hit distinct banks
  __shared__ T Bs[kKC][kTB + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const int lr = tid >> 2, lk = (tid & 3) * 8;
  for (int kk = kb; kk < ke; kk += kKC) {
    {
      const int ra = r0 + lr, rb = c0 + lr;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = kk + lk + q;
        As[lk + q][lr] = (ra < d.m && k < ke) ? A[(long long)ra * d.ld + k] : T(0);
        Bs[lk + q][lr] = (rb < colend && k < ke) ? A[(long long)rb * d.ld + k] : T(0);
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kKC; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= d.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < colend) A[(long long)r * d.ld + c] -= acc[i][j];
    }
  }
}

std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }
long long launch_count() { return g_launches.load(); }

// Lower-triangle entries updated by a rank-k launch: panel mode rows [t0, m) x cols [t0, e), c <= r.
static double trapezoid(long long t0, long long e, long long m) {
  const long long k = e - t0;
  return (double)(k * (m - t0) - k * (k - 1) / 2);
}

// ---- FP32 rank-k update: 128x128 CTA tiles, 8x8 outputs per thread ----------
// Same modes and index ranges as k_rankk.  K is consumed in chunks of 16 with
// the next chunk prefetched into registers while the current one is used.
constexpr int kTB2 = 128, kKC2 = 16;

__global__ void __launch_bounds__(256) k_rankk128(const MatDesc *__restrict__ desc, float *__restrict__ base,
                                                  int mode, int k0, int K0, int K1, int nct) {
  const MatDesc d = desc[blockIdx.y];
  int row0, colend, kb, ke;
  if (mode == 0) {
    if (k0 >= d.e) return;
    const int w = min(kNB, d.e - k0);
    row0 = k0 + w; colend = min(K1, d.e); kb = k0; ke = k0 + w;
  } else if (mode == 2) {
    if (K1 >= d.e) return;
    row0 = K1; colend = d.e; kb = K0; ke = K1;
  } else {
    row0 = d.e; colend = d.m; kb = 0; ke = d.e;
  }
  const int ti = blockIdx.x / nct, tj = blockIdx.x % nct;
  if (tj > ti) return;
  const int r0 = row0 + ti * kTB2, c0 = row0 + tj * kTB2;
  if (r0 >= d.m || c0 >= colend || ke <= kb) return;
  float *A = base + d.off;
  __shared__ __align__(16) float As[2][kKC2][kTB2 + 4];
  __shared__ __align__(16) float Bs[2][kKC2][kTB2 + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // loader: thread -> (row lr, k offset lk): 128 rows x 16 k = 2 x 4 floats per thread per operand
  const int lr = tid >> 1, lk = (tid & 1) * 8;
  const int ra = r0 + lr, rb = c0 + lr;
  const bool va = ra < d.m, vb = rb < colend;
  const float *pa = A + (long long)ra * d.ld, *pb = A + (long long)rb * d.ld;
  float la[8], lb[8];
  auto load = [&](int kk) {
#pragma unroll
    for (int q = 0; q < 8; q += 4) {
      const int k = kk + lk + q;
      if (k + 3 < ke) {
        const float4 x = va ? *reinterpret_cast<const float4 *>(pa + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 y = vb ? *reinterpret_cast<const float4 *>(pb + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        la[q] = x.x; la[q + 1] = x.y; la[q + 2] = x.z; la[q + 3] = x.w;
        lb[q] = y.x; lb[q + 1] = y.y; lb[q + 2] = y.z; lb[q + 3] = y.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          la[q + u] = (va && k + u < ke) ? pa[k + u] : 0.f;
          lb[q + u] = (vb && k + u < ke) ? pb[k + u] : 0.f;
        }
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      As[buf][lk + q][lr] = la[q];
      Bs[buf][lk + q][lr] = lb[q];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  load(kb);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int kk = kb; kk < ke; kk += kKC2) {
    const bool more = kk + kKC2 < ke;
    if (more) load(kk + kKC2);
#pragma unroll
    for (int k = 0; k < kKC2; ++k) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] += av[i] * bv[j];
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  // thread owns rows {ty*4 + i, 64 + ty*4 + i} and columns {tx*4 + j, 64 + tx*4 + j}
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (r >= d.m) continue;
    float *crow = A + (long long)r * d.ld;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (c < colend) crow[c] -= acc[i][j];
    }
  }
}

template <typename T>
static void launch_rankk(const MatDesc *d_desc, T *base, int mode, int k0, int K0, int K1, int max_rows, int max_cols,
                         int count, cudaStream_t s) {
  const int nrt = ceil_div(max_rows, kTB), nct = ceil_div(max_cols, kTB);
  if (nrt == 0 || nct == 0) return;
  k_rankk<T><<<dim3(nrt * nct, count), 256, 0, s>>>(d_desc, base, mode, k0, K0, K1, nct);
  count_launch();
}
template <>
void launch_rankk<float>(const MatDesc *d_desc, float *base, int mode, int k0, int K0, int K1, int max_rows,
                         int max_cols, int count, cudaStream_t s) {
  const int nrt = ceil_div(max_rows, kTB2), nct = ceil_div(max_cols, kTB2);
  if (nrt == 0 || nct == 0) return;
  k_rankk128<<<dim3(nrt * nct, count), 256, 0, s>>>(d_desc, base, mode, k0, K0, K1, nct);
  count_launch();
}

template <typename T>
void engine_partial_cholesky(const EngineShape &sh, const MatDesc *d_desc, T *base, int *d_err, cudaStream_t s,
                             T *linv, ProfHook *prof, bool tc) {
  if (sh.count == 0) return;
  const int ob = std::max(kNB, (sh.ob / kNB) * kNB);
  for (int K0 = 0; K0 < sh.max_e; K0 += ob) {
    const int K1 = K0 + ob;
    for (int k0 = K0; k0 < std::min(K1, sh.max_e); k0 += kNB) {
      int max_below = 0, max_cols = 0;
      double fl_panel = 0.0, fl_upd = 0.0, by_upd = 0.0;
      for (int b = 0; b < sh.count; ++b) {
        if (k0 >= sh.e[b]) continue;
        const int w = std::min(kNB, sh.e[b] - k0);
        const int below = sh.m[b] - k0 - w;
        const int cend = std::min(K1, sh.e[b]);
        max_below = std::max(max_below, below);
        max_cols = std::max(max_cols, cend - k0 - w);
        fl_panel += (double)w * w * w / 3.0 + (double)below * w * w;
        const double ent = trapezoid(k0 + w, cend, sh.m[b]);
        fl_upd += 2.0 * w * ent;
        by_upd += sizeof(T) * (2.0 * ent + (double)w * (below + cend - k0 - w));
      }
      if (prof) prof->begin(PROF_PANEL, s);
      k_potrf<T><<<sh.count, 1024, 0, s>>>(d_desc, base, k0, d_err, linv);
      count_launch();
      if (max_below > 0) {
        dim3 gp(ceil_div(max_below, 128), sh.count);
        k_trsm<T><<<gp, 128, 0, s>>>(d_desc, base, k0, linv);
        count_launch();
      }
      if (prof) prof->end(PROF_PANEL, s, fl_panel, 0.0);
      if (max_below > 0 && max_cols > 0) {
        if (prof) prof->begin(PROF_RANKK, s);
        launch_rankk<T>(d_desc, base, 0, k0, K0, K1, max_below, max_cols, sh.count, s);
        if (prof) prof->end(PROF_RANKK, s, fl_upd, by_upd);
      }
    }
    // outer update of the trailing columns [K1, e) with the finished outer panel
    int max_rows = 0, max_cols = 0;
    double fl = 0.0, by = 0.0;
    for (int b = 0; b < sh.count; ++b) {
      if (K1 >= sh.e[b]) continue;
      max_rows = std::max(max_rows, sh.m[b] - K1);
      max_cols = std::max(max_cols, sh.e[b] - K1);
      const double ent = trapezoid(K1, sh.e[b], sh.m[b]);
      fl += 2.0 * ob * ent;
      by += sizeof(T) * (2.0 * ent + (double)ob * (sh.m[b] - K1));
    }
    if (max_rows > 0 && max_cols > 0) {
      if (prof) prof->begin(PROF_RANKK, s);
      if constexpr (std::is_same<T, float>::value) {
        if (tc) launch_rankk_tc(d_desc, base, 2, K0, K1, max_rows, max_cols, sh.count, d_err, s);
        else launch_rankk<T>(d_desc, base, 2, 0, K0, K1, max_rows, max_cols, sh.count, s);
      } else {
        launch_rankk<T>(d_desc, base, 2, 0, K0, K1, max_rows, max_cols, sh.count, s);
      }
      if (prof) prof->end(PROF_RANKK, s, fl, by);
    }
  }
  int max_t = 0;
  double fl = 0.0, by = 0.0;
  for (int b = 0; b < sh.count; ++b) {
    max_t = std::max(max_t, sh.m[b] - sh.e[b]);
    const double n2 = sh.m[b] - sh.e[b];
    const double ent = n2 * (n2 + 1) / 2.0;
    fl += 2.0 * sh.e[b] * ent;
    by += sizeof(T) * (2.0 * ent + n2 * sh.e[b]);
  }
  if (max_t > 0) {
    if (prof) prof->begin(PROF_RANKK, s);
    if constexpr (std::is_same<T, float>::value) {
      if (tc) launch_rankk_tc(d_desc, base, 1, 0, 0, max_t, max_t, sh.count, d_err, s);
      else launch_rankk<T>(d_desc, base, 1, 0, 0, 0, max_t, max_t, sh.count, s);
    } else {
      launch_rankk<T>(d_desc, base, 1, 0, 0, 0, max_t, max_t, sh.count, s);
    }
    if (prof) prof->end(PROF_RANKK, s, fl, by);
  }
}

// ---- batched GEMV ------------------------------------------------------------
// One CTA (8 warps) per (task, block of kGemvRows rows): each warp owns two rows
// with independent accumulators; x is staged in shared memory.
constexpr int kGemvRows = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemv(const GemvDesc *__restrict__ tasks, const T *__restrict__ A,
                                              const double *__restrict__ x, const int *__restrict__ xidx,
                                              double *__restrict__ y, double alpha, const int *__restrict__ done) {
  if (done && *done) return;
  const GemvDesc t = tasks[blockIdx.y];
  const int rbeg = blockIdx.x * kGemvRows;
  if (rbeg >= t.rows) return;
  extern __shared__ unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  for (int c = threadIdx.x; c < t.cols; c += blockDim.x)
    xs[c] = (T)((t.flags & 1) ? x[xidx[t.x_off + c]] : x[t.x_off + c]);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int r0 = rbeg + wid, r1 = rbeg + wid + 8;
  const bool v0 = r0 < t.rows, v1 = r1 < t.rows;
  const T *row0 = A + t.a_off + (long long)(v0 ? r0 : rbeg) * t.ld;
  const T *row1 = A + t.a_off + (long long)(v1 ? r1 : rbeg) * t.ld;
  T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0);
  int c = lane;
  for (; c + 32 < t.cols; c += 64) {
    const T x0 = xs[c], x1 = xs[c + 32];
    a0 += row0[c] * x0;
    a1 += row0[c + 32] * x1;
    b0 += row1[c] * x0;
    b1 += row1[c + 32] * x1;
  }
  if (c < t.cols) {
    a0 += row0[c] * xs[c];
    b0 += row1[c] * xs[c];
  }
  const T s0 = warp_sum(a0 + a1), s1 = warp_sum(b0 + b1);
  if (lane == 0) {
    if (v0) {
      const double v = alpha * (double)s0;
      y[t.y_off + r0] = (t.flags & 2) ? y[t.y_off + r0] + v : v;
    }
    if (v1) {
      const double v = alpha * (double)s1;
      y[t.y_off + r1] = (t.flags & 2) ? y[t.y_off + r1] + v : v;
    }
  }
}

// y[a] = (acc ? y[a] : 0) + alpha sum_p A[p][a] x[p]; one thread per column a.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv_t(const GemvDesc *__restrict__ tasks, const T *__restrict__ A,
                                                const double *__restrict__ x, const int *__restrict__ xidx,
                                                double *__restrict__ y, double alpha, const int *__restrict__ done) {
  if (done && *done) return;
  const GemvDesc t = tasks[blockIdx.y];
  extern __shared__ unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  for (int p = threadIdx.x; p < t.rows; p += blockDim.x)
    xs[p] = (T)((t.flags & 1) ? x[xidx[t.x_off + p]] : x[t.x_off + p]);
  __syncthreads();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= t.cols) return;
  const T *col = A + t.a_off + a;
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int p = 0;
  for (; p + 3 < t.rows; p += 4) {
    a0 += col[(long long)p * t.ld] * xs[p];
    a1 += col[(long long)(p + 1) * t.ld] * xs[p + 1];
    a2 += col[(long long)(p + 2) * t.ld] * xs[p + 2];
    a3 += col[(long long)(p + 3) * t.ld] * xs[p + 3];
  }
  for (; p < t.rows; ++p) a0 += col[(long long)p * t.ld] * xs[p];
  const double v = alpha * (double)((a0 + a1) + (a2 + a3));
  y[t.y_off + a] = (t.flags & 2) ? y[t.y_off + a] + v : v;
}

template <typename T>
void launch_gemv(int ntasks, int max_rows, int max_cols, const GemvDesc *d_tasks, const T *A, const double *x,
                 const int *xidx, double *y, double alpha, const int *done, cudaStream_t s) {
  if (ntasks == 0 || max_rows == 0) return;
  dim3 g(ceil_div(max_rows, kGemvRows), ntasks);
  const size_t sm = sizeof(T) * (size_t)std::max(1, max_cols);
  k_gemv<T><<<g, 256, sm, s>>>(d_tasks, A, x, xidx, y, alpha, done);
  count_launch();
}

template <typename T>
void launch_gemv_t(int ntasks, int max_rows, int max_cols, const GemvDesc *d_tasks, const T *A, const double *x,
                   const int *xidx, double *y, double alpha, const int *done, cudaStream_t s) {
  if (ntasks == 0 || max_cols == 0) return;
  dim3 g(ceil_div(max_cols, 256), ntasks);
  const size_t sm = sizeof(T) * (size_t)std::max(1, max_rows);
  k_gemv_t<T><<<g, 256, sm, s>>>(d_tasks, A, x, xidx, y, alpha, done);
  count_launch();
}

// ---- batched triangular solves (one CTA of 32 warps per matrix) ---------------
// lower: y = L^-1 b, left-looking over 32-row blocks, one warp per block row;
// upper: y = L^-T b, right-to-left, warps striding over the rows below the block.
// The 32x32 diagonal block is staged in shared memory; the vector lives there too.
template <typename T>
__global__ void __launch_bounds__(1024) k_trsv(const MatDesc *__restrict__ desc, const int *__restrict__ vec_off,
                                               const T *__restrict__ base, const double *__restrict__ b,
                                               double *__restrict__ y, int transpose) {
  const MatDesc d = desc[blockIdx.x];
  const int n = d.e;
  const T *L = base + d.off;
  extern __shared__ unsigned char smem_raw[];
  T *v = reinterpret_cast<T *>(smem_raw);
  __shared__ T part[32][33];
  __shared__ T Lb[32][33];
  const int off = vec_off[blockIdx.x];
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = (T)b[off + i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nblk = ceil_div(n, 32);
  for (int q = 0; q < nblk; ++q) {
    const int bk = transpose ? nblk - 1 - q : q;
    const int r0 = bk * 32, r1 = min(n, r0 + 32);
    {  // diagonal block, coalesced: warp wid loads row r0 + wid
      const int i = wid, k = lane;
      Lb[i][k] = (r0 + i < r1 && k <= i) ? L[(long long)(r0 + i) * d.ld + r0 + k] : T(0);
    }
    __syncthreads();
    if (!transpose) {
      // v[r] -= sum_{c < r0} L[r][c] v[c]; warp wid owns row r0 + wid
      const int r = r0 + wid;
      if (r < r1) {
        const T *Lr = L + (long long)r * d.ld;
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int c = lane;
        for (; c + 96 < r0; c += 128) {
          a0 += Lr[c] * v[c];
          a1 += Lr[c + 32] * v[c + 32];
          a2 += Lr[c + 64] * v[c + 64];
          a3 += Lr[c + 96] * v[c + 96];
        }
        for (; c < r0; c += 32) a0 += Lr[c] * v[c];
        const T acc = warp_sum((a0 + a1) + (a2 + a3));
        if (lane == 0) v[r] -= acc;
      }
      __syncthreads();
      if (wid == 0) {
        const int r = r0 + lane;
        T vr = (r < r1) ? v[r] : T(0);
        for (int c = r0; c < r1; ++c) {
          const T xc = __shfl_sync(0xffffffffu, vr / ((r == c) ? Lb[lane][lane] : T(1)), c - r0);
          if (r == c) vr = xc;
          else if (r > c && r < r1) vr -= Lb[lane][c - r0] * xc;
        }
        if (r < r1) v[r] = vr;
      }
      __syncthreads();
    } else {
      // v[r] -= sum_{c >= r1} L[c][r] v[c] for r in the block; warp wid takes rows r1 + wid + 32 k
      T a0 = T(0), a1 = T(0);
      const int r = r0 + lane;
      if (r < r1) {
        int c = r1 + wid;
        for (; c + 32 < n; c += 64) {
          a0 += L[(long long)c * d.ld + r] * v[c];
          a1 += L[(long long)(c + 32) * d.ld + r] * v[c + 32];
        }
        for (; c < n; c += 32) a0 += L[(long long)c * d.ld + r] * v[c];
      }
      part[wid][lane] = a0 + a1;
      __syncthreads();
      if (wid == 0) {
        T s = T(0);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) s += part[k][lane];
        T vr = (r < r1) ? v[r] - s : T(0);
        for (int c = r1 - 1; c >= r0; --c) {
          const T xc = __shfl_sync(0xffffffffu, vr / ((r == c) ? Lb[lane][lane] : T(1)), c - r0);
          if (r == c) vr = xc;
          else if (r < c && r < r1) vr -= Lb[c - r0][lane] * xc;
        }
        if (r < r1) v[r] = vr;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[off + i] = (double)v[i];
}

template <typename T>
void launch_trsv(int count, int max_n, const MatDesc *d_desc, const int *vec_off, const T *base, const double *b,
                 double *y, bool transpose, cudaStream_t s) {
  if (count == 0) return;
  const size_t sm = sizeof(T) * (size_t)std::max(1, max_n);
  k_trsv<T><<<count, 1024, sm, s>>>(d_desc, vec_off, base, b, y, transpose ? 1 : 0);
  count_launch();
}

// Large local problems stage vectors of up to ~25k entries in shared memory.
bool dense_configure() {
  const int lim = 200 * 1024;
  bool ok = true;
  ok &= cudaFuncSetAttribute(k_trsv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_trsv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv_t<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv_t<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  return ok;
}

#define BD_INST(T)                                                                                              \
  template void engine_partial_cholesky<T>(const EngineShape &, const MatDesc *, T *, int *, cudaStream_t,    \
                                           T *, ProfHook *, bool);     \
  template void launch_gemv<T>(int, int, int, const GemvDesc *, const T *, const double *, const int *,        \
                               double *, double, const int *, cudaStream_t);                                   \
  template void launch_gemv_t<T>(int, int, int, const GemvDesc *, const T *, const double *, const int *,      \
                                 double *, double, const int *, cudaStream_t);                                 \
  template void launch_trsv<T>(int, int, const MatDesc *, const int *, const T *, const double *, double *,    \
                               bool, cudaStream_t);
BD_INST(float)
BD_INST(double)

}  // namespace bd
