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
#include <vector>

#include "kernels.cuh"

namespace bd {

template <typename T> __device__ inline T dsqrt(T v);
template <> __device__ inline float dsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ inline double dsqrt<double>(double v) { return sqrt(v); }

// ---- panel step 1: factor the w x w diagonal block in place and form L_kk^-1 --
// One warp per matrix.  Lane r keeps row r of the block in registers; column c
// of L is broadcast with shuffles, so the right-looking update has no shared-
// memory dependency chain.  L_kk^-1 (used by the panel solve) goes to `linv`.
template <typename T>
__global__ void __launch_bounds__(32) k_potrf(const MatDesc *__restrict__ desc, T *__restrict__ base, int k0,
                                              int *__restrict__ err, T *__restrict__ linv) {
  const MatDesc d = desc[blockIdx.x];
  if (k0 >= d.e) return;
  const int w = min(kNB, d.e - k0);
  T *A = base + d.off;
  __shared__ T Ls[kNB][kNB + 1];
  const int r = threadIdx.x;
#pragma unroll 8
  for (int q = 0; q < kNB; ++q)  // row q, lane = column: coalesced, independent loads
    Ls[q][r] = (q < w && r <= q) ? A[(long long)(k0 + q) * d.ld + k0 + r] : T(0);
  __syncwarp();
  T row[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) row[c] = Ls[r][c];
  bool bad = false;
#pragma unroll
  for (int c = 0; c < kNB; ++c) {
    if (c < w) {
      T dg = __shfl_sync(0xffffffffu, row[c], c);
      if (!(dg > T(0))) { bad = true; dg = T(1); }
      const T sq = dsqrt(dg);
      if (r == c) row[c] = sq;
      else if (r > c) row[c] = row[c] / sq;
      const T lrc = row[c];
#pragma unroll
      for (int t = c + 1; t < kNB; ++t) {
        const T ltc = __shfl_sync(0xffffffffu, row[c], t);
        if (r >= t) row[t] -= lrc * ltc;
      }
    }
  }
  if (bad && r == 0) atomicOr(err, DEV_ERR_NOT_SPD);
#pragma unroll
  for (int c = 0; c < kNB; ++c) Ls[r][c] = (c <= r && r < w && c < w) ? row[c] : (r == c ? T(1) : T(0));
  __syncwarp();
#pragma unroll 8
  for (int q = 0; q < w; ++q)  // write back row q, lane = column
    if (r <= q) A[(long long)(k0 + q) * d.ld + k0 + r] = Ls[q][r];
  // L_kk^-1: lane j solves L y = e_j by forward substitution (column j of the inverse)
  T y[kNB];
#pragma unroll
  for (int i = 0; i < kNB; ++i) {
    T v = (i == r) ? T(1) : T(0);
#pragma unroll
    for (int t = 0; t < i; ++t) v -= Ls[i][t] * y[t];
    y[i] = (i >= r) ? v / Ls[i][i] : T(0);
  }
  T *Li = linv + (long long)blockIdx.x * kNB * kNB;
#pragma unroll
  for (int i = 0; i < kNB; ++i) Li[i * kNB + r] = y[i];  // Li[i][j] = (L^-1)[i][j], lane = j
}

// ---- panel step 2: rows below the diagonal block, x = a L_kk^-T (one thread per row)
template <typename T>
__global__ void __launch_bounds__(128) k_trsm(const MatDesc *__restrict__ desc, T *__restrict__ base, int k0,
                                              const T *__restrict__ linv) {
  const MatDesc d = desc[blockIdx.y];
  if (k0 >= d.e) return;
  const int w = min(kNB, d.e - k0);
  if (k0 + w + blockIdx.x * 128 >= d.m) return;
  T *A = base + d.off;
  __shared__ T Li[kNB][kNB];
  const T *src = linv + (long long)blockIdx.y * kNB * kNB;
  for (int t = threadIdx.x; t < kNB * kNB; t += 128) Li[t / kNB][t % kNB] = src[t];
  __syncthreads();
  const int row = k0 + w + blockIdx.x * 128 + threadIdx.x;
  if (row >= d.m) return;
  T *a = A + (long long)row * d.ld + k0;
  T x[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) x[c] = (c < w) ? a[c] : T(0);
  // x_out[c] = sum_{t <= c} x[t] (L^-1)[c][t]: independent dot products
#pragma unroll
  for (int c = kNB - 1; c >= 0; --c) {
    T v = T(0);
#pragma unroll
    for (int t = 0; t <= c; ++t) v += x[t] * Li[c][t];
    x[c] = v;
  }
#pragma unroll
  for (int c = 0; c < kNB; ++c)
    if (c < w) a[c] = x[c];
}

// ---- rank-k update of lower tiles --------------------------------------------
// mode 0 (panel): rows [k0+w, m), cols [k0+w, e), K = panel [k0, k0+w)
// mode 1 (final): rows [e, m),    cols [e, m),    K = [0, e)
// C[r][c] -= sum_k A[r][k] A[c][k]; 64x64 tiles, 256 threads, 4x4 per thread.
constexpr int kTB = 64, kKC = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_rankk(const MatDesc *__restrict__ desc, T *__restrict__ base, int mode,
                                               int k0, int nct) {
  const MatDesc d = desc[blockIdx.y];
  int row0, colend, kb, ke;
  if (mode == 0) {
    if (k0 >= d.e) return;
    const int w = min(kNB, d.e - k0);
    row0 = k0 + w;
    colend = d.e;
    kb = k0;
    ke = k0 + w;
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

template <typename T>
void engine_partial_cholesky(const EngineShape &sh, const MatDesc *d_desc, T *base, int *d_err, cudaStream_t s,
                             T *linv, ProfHook *prof) {
  if (sh.count == 0) return;
  for (int k0 = 0; k0 < sh.max_e; k0 += kNB) {
    int max_below = 0, max_rt = 0, max_ct = 0;
    double fl_panel = 0.0, fl_upd = 0.0, by_upd = 0.0;
    for (int b = 0; b < sh.count; ++b) {
      if (k0 >= sh.e[b]) continue;
      const int w = std::min(kNB, sh.e[b] - k0);
      const int below = sh.m[b] - k0 - w;
      max_below = std::max(max_below, below);
      max_rt = std::max(max_rt, ceil_div(below, kTB));
      max_ct = std::max(max_ct, ceil_div(sh.e[b] - k0 - w, kTB));
      fl_panel += (double)w * w * w / 3.0 + (double)below * w * w;
      const double ent = trapezoid(k0 + w, sh.e[b], sh.m[b]);
      fl_upd += 2.0 * w * ent;
      by_upd += sizeof(T) * (2.0 * ent + (double)w * (below + sh.e[b] - k0 - w));
    }
    if (prof) prof->begin(PROF_PANEL, s);
    k_potrf<T><<<sh.count, 32, 0, s>>>(d_desc, base, k0, d_err, linv);
    count_launch();
    if (max_below > 0) {
      dim3 gp(ceil_div(max_below, 128), sh.count);
      k_trsm<T><<<gp, 128, 0, s>>>(d_desc, base, k0, linv);
      count_launch();
    }
    if (prof) prof->end(PROF_PANEL, s, fl_panel, 0.0);
    if (max_rt > 0 && max_ct > 0) {
      dim3 gu(max_rt * max_ct, sh.count);
      if (prof) prof->begin(PROF_RANKK, s);
      k_rankk<T><<<gu, 256, 0, s>>>(d_desc, base, 0, k0, max_ct);
      count_launch();
      if (prof) prof->end(PROF_RANKK, s, fl_upd, by_upd);
    }
  }
  int max_t = 0;
  double fl = 0.0, by = 0.0;
  for (int b = 0; b < sh.count; ++b) {
    max_t = std::max(max_t, ceil_div(sh.m[b] - sh.e[b], kTB));
    const double n2 = sh.m[b] - sh.e[b];
    const double ent = n2 * (n2 + 1) / 2.0;
    fl += 2.0 * sh.e[b] * ent;
    by += sizeof(T) * (2.0 * ent + n2 * sh.e[b]);
  }
  if (max_t > 0) {
    dim3 gf(max_t * max_t, sh.count);
    if (prof) prof->begin(PROF_RANKK, s);
    k_rankk<T><<<gf, 256, 0, s>>>(d_desc, base, 1, 0, max_t);
    count_launch();
    if (prof) prof->end(PROF_RANKK, s, fl, by);
  }
}

// ---- batched GEMV ------------------------------------------------------------
// One CTA (8 warps) per (task, block of 64 rows); x staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv(const GemvDesc *__restrict__ tasks, const T *__restrict__ A,
                                              const double *__restrict__ x, const int *__restrict__ xidx,
                                              double *__restrict__ y, double alpha, const int *__restrict__ done) {
  if (done && *done) return;
  const GemvDesc t = tasks[blockIdx.y];
  const int rbeg = blockIdx.x * 64;
  if (rbeg >= t.rows) return;
  extern __shared__ unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  for (int c = threadIdx.x; c < t.cols; c += blockDim.x)
    xs[c] = (T)((t.flags & 1) ? x[xidx[t.x_off + c]] : x[t.x_off + c]);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rend = min(t.rows, rbeg + 64);
  for (int r = rbeg + wid; r < rend; r += 8) {
    const T *row = A + t.a_off + (long long)r * t.ld;
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int c = lane;
    for (; c + 96 < t.cols; c += 128) {
      a0 += row[c] * xs[c];
      a1 += row[c + 32] * xs[c + 32];
      a2 += row[c + 64] * xs[c + 64];
      a3 += row[c + 96] * xs[c + 96];
    }
    for (; c < t.cols; c += 32) a0 += row[c] * xs[c];
    const T acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) {
      const double v = alpha * (double)acc;
      y[t.y_off + r] = (t.flags & 2) ? y[t.y_off + r] + v : v;
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
  dim3 g(ceil_div(max_rows, 64), ntasks);
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

#define BD_INST(T)                                                                                              \
  template void engine_partial_cholesky<T>(const EngineShape &, const MatDesc *, T *, int *, cudaStream_t,    \
                                           T *, ProfHook *);     \
  template void launch_gemv<T>(int, int, int, const GemvDesc *, const T *, const double *, const int *,        \
                               double *, double, const int *, cudaStream_t);                                   \
  template void launch_gemv_t<T>(int, int, int, const GemvDesc *, const T *, const double *, const int *,      \
                                 double *, double, const int *, cudaStream_t);                                 \
  template void launch_trsv<T>(int, int, const MatDesc *, const int *, const T *, const double *, double *,    \
                               bool, cudaStream_t);
BD_INST(float)
BD_INST(double)

}  // namespace bd
