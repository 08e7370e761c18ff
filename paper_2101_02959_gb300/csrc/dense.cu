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
// 1 / sqrt(v): the hardware estimate for float (relative error a few units in the
// last place, the level of FP32 rounding in the factors), the library routine for double
template <typename T> __device__ inline T drsqrt(T v);
template <> __device__ inline float drsqrt<float>(float v) { return rsqrtf(v); }
template <> __device__ inline double drsqrt<double>(double v) { return rsqrt(v); }

// 16-byte vectors of T (row starts of the batched matrices are 32-byte aligned).
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static float get(const float4 &v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }
  __device__ static void set(float4 &v, int q, float a) {
    if (q == 0) v.x = a; else if (q == 1) v.y = a; else if (q == 2) v.z = a; else v.w = a;
  }
  __device__ static float dot(const float4 a, const float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
  __device__ static void axpy(float *acc, const float4 a, float s) {
    acc[0] += a.x * s; acc[1] += a.y * s; acc[2] += a.z * s; acc[3] += a.w * s;
  }
};
template <> struct Vec16<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static double get(const double2 &v, int q) { return q == 0 ? v.x : v.y; }
  __device__ static void set(double2 &v, int q, double a) {
    if (q == 0) v.x = a; else v.y = a;
  }
  __device__ static double dot(const double2 a, const double2 b) { return a.x * b.x + a.y * b.y; }
  __device__ static void axpy(double *acc, const double2 a, double s) { acc[0] += a.x * s; acc[1] += a.y * s; }
};

// ---- 32 x 32 Cholesky in one warp: lane r holds row r in registers ------------
// Columns c < wb are eliminated (pivot broadcast by shuffle, scaled column, rank-1
// update of the rows below); rows and columns from wb on must hold the identity.
template <typename T>
__device__ __forceinline__ void warp_chol32(T (&a)[32], int lane, int wb, bool &bad) {
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    if (c < wb) {  // uniform across the warp
      T piv = __shfl_sync(0xffffffffu, a[c], c);
      if (!(piv > T(0))) { bad = true; piv = T(1); }
      const T inv = drsqrt(piv), sd = piv * inv;
      a[c] = (lane == c) ? sd : a[c] * inv;  // rows above c hold 0 here
#pragma unroll
      for (int t = c + 1; t < 32; ++t) {
        const T lt = __shfl_sync(0xffffffffu, a[c], t);
        if (lane >= t) a[t] -= a[c] * lt;
      }
    }
  }
}

// ---- outer panel: partial Cholesky of the columns [K0, K0 + w), w <= kPW ---------
// Two launches per outer panel.  The diagonal launch (ROWS = false, one CTA per
// matrix) stages the w x w diagonal block (lower triangle, identity outside w) in
// shared memory and factors it 32 columns at a time: warp 0 factors the 32 x 32
// diagonal sub-block in registers, one thread per remaining row solves
// x L_bb^T = a, and all threads apply the rank-32 update to the remaining columns
// (4 x 4 register tiles over a transposed copy of the solved columns).  It writes
// L_11 in place and the factored 32 x 32 diagonal sub-blocks to the block store
// (slots dblk + K0 / 32 + q).  The rows launch (ROWS = true) then solves the rows
// below, RB per CTA, the same way, reading the finished L_11 one 32-column slice at
// a time instead of factoring it.
constexpr int kPW = kEnginePanel;  // outer panel width
constexpr int kLDP = kPW + 4;      // row stride of the staged panel (16-byte aligned rows)
template <typename T> struct PanelRows;
template <> struct PanelRows<float> { static constexpr int RB = 128; };
template <> struct PanelRows<double> { static constexpr int RB = 16; };

template <typename T, bool ROWS>
constexpr size_t bigpanel_smem() {
  constexpr int RB = PanelRows<T>::RB, NR = kPW + RB, NS = ROWS ? RB : kPW;
  return sizeof(T) * ((size_t)NS * kLDP + 32 * NR + 32 * 32 + 32);
}

template <typename T, bool ROWS>
__global__ void __launch_bounds__(256, 2) k_bigpanel(const MatDesc *__restrict__ desc, T *__restrict__ base, int K0,
                                                     int *__restrict__ err, T *__restrict__ store) {
  constexpr int RB = PanelRows<T>::RB, NR = kPW + RB;
  constexpr int NS = ROWS ? RB : kPW;         // staged rows
  constexpr int OWN0 = ROWS ? 0 : kPW;        // staged index of the first own row (rows launch only)
  using VT = typename Vec16<T>::V;
  constexpr int VN = Vec16<T>::N, VPP = kPW / VN;  // vectors per staged row
  const MatDesc d = desc[blockIdx.y];
  if (K0 >= d.e) return;
  const int w = min(kPW, d.e - K0);
  // rows launch: the rows below the panel that it reaches (interior rows up to the band)
  const BandRows br = band_rows(d, K0 + w, K0 + w);
  const int v0 = blockIdx.x * RB;
  if (ROWS && v0 >= br.nv) return;
  const int nrows = ROWS ? min(RB, br.nv - v0) : 0;
  T *A = base + d.off;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *P = reinterpret_cast<T *>(smem_raw);  // [NS][kLDP]: (diagonal rows,) own rows
  T *PT = P + NS * kLDP;                   // [32][NR]: the current 32 columns, transposed (row p of the panel)
  T *Lt = PT + 32 * NR;                    // [32][32]: Lt[c][t] = L_bb[t][c]
  T *rd = Lt + 32 * 32;                    // [32]: 1 / L_bb[c][c]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // panel row p (diagonal rows p < kPW, own rows kPW + q) -> staged row
  auto prow = [&](int p) { return P + (p - kPW + OWN0) * kLDP; };
  // ---- stage: kBatch vector loads in flight per thread and batch
  constexpr int kVec = NS * VPP, kBatch = 8;
  for (int base_i = 0; base_i < kVec; base_i += 256 * kBatch) {
    VT buf[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int idx = base_i + tid + 256 * u;
      const int sr = idx / VPP, cv = idx % VPP;
      const bool diag = !ROWS && sr < kPW;
      const bool ok = idx < kVec && cv * VN < w && (diag ? sr < w : sr - OWN0 < nrows);
      const long long grow = diag ? K0 + sr : (ok ? br.row(v0 + sr - OWN0) : 0);
      buf[u] = ok ? *reinterpret_cast<const VT *>(A + grow * d.ld + K0 + cv * VN) : VT{};
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int idx = base_i + tid + 256 * u;
      const int sr = idx / VPP, cv = idx % VPP;
      if (idx < kVec) {
        const bool diag = !ROWS && sr < kPW;
        VT o;
#pragma unroll
        for (int q = 0; q < VN; ++q) {
          const int j = cv * VN + q;
          const T e = Vec16<T>::get(buf[u], q);
          if (diag) Vec16<T>::set(o, q, (sr < w && j < w && j <= sr) ? e : (j == sr ? T(1) : T(0)));
          else Vec16<T>::set(o, q, (sr - OWN0 < nrows && j < w) ? e : T(0));
        }
        *reinterpret_cast<VT *>(P + sr * kLDP + cv * VN) = o;
      }
    }
  }
  bool bad = false;
  const int nbk = ceil_div(w, 32);
  for (int bq = 0; bq < nbk; ++bq) {
    const int c0 = 32 * bq, wb = min(32, w - c0);
    const int nbelow = max(0, w - c0 - 32);  // diagonal-block rows below the sub-block
    __syncthreads();
    if (wid == 0) {
      T a[32];
      {
        const T *src = ROWS ? A + (long long)(K0 + c0 + (lane < wb ? lane : 0)) * d.ld + K0 + c0
                            : P + (c0 + lane) * kLDP + c0;
#pragma unroll
        for (int i = 0; i < 32 / VN; ++i) {
          const bool rd_ok = !ROWS || (lane < wb && i * VN <= lane);
          const VT v = rd_ok ? *reinterpret_cast<const VT *>(src + i * VN) : VT{};
#pragma unroll
          for (int q = 0; q < VN; ++q) {
            const int t = i * VN + q;
            a[t] = (lane < wb && t <= lane) ? Vec16<T>::get(v, q) : (t == lane ? T(1) : T(0));
          }
        }
      }
      if (!ROWS) warp_chol32(a, lane, wb, bad);
      T dg = T(1);
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const T v = (t <= lane) ? a[t] : T(0);
        if (t == lane) dg = v;
        if (!ROWS) P[(c0 + lane) * kLDP + c0 + t] = v;
        Lt[t * 32 + lane] = v;
      }
      rd[lane] = T(1) / dg;
      if (!ROWS) {
        T *sb = store + ((long long)d.dblk + K0 / kNB + bq) * kNB * kNB + lane * kNB;
#pragma unroll
        for (int i = 0; i < 32 / VN; ++i) {
          VT o;
#pragma unroll
          for (int q = 0; q < VN; ++q) Vec16<T>::set(o, q, (i * VN + q <= lane) ? a[i * VN + q] : T(0));
          *reinterpret_cast<VT *>(sb + i * VN) = o;
        }
      }
    } else if (ROWS) {
      // the finished L_11 rows below the sub-block, columns [c0, c0 + 32), transposed
      for (int idx = tid - 32; idx < nbelow * (32 / VN); idx += 256 - 32) {
        const int r = idx / (32 / VN), cv = idx % (32 / VN), p = c0 + 32 + r;
        const VT v = *reinterpret_cast<const VT *>(A + (long long)(K0 + p) * d.ld + K0 + c0 + cv * VN);
#pragma unroll
        for (int q = 0; q < VN; ++q) PT[(cv * VN + q) * NR + p] = Vec16<T>::get(v, q);
      }
    }
    __syncthreads();
    // rows below the sub-block: (diagonal rows [c0 + 32, w),) then the own rows
    const int ndiag = ROWS ? 0 : nbelow;
    const int nsolve = ndiag + nrows;
    for (int qr = tid; qr < nsolve; qr += 256) {
      const int p = qr < ndiag ? c0 + 32 + qr : kPW + (qr - ndiag);
      T x[32];
      T *src = prow(p) + c0;
#pragma unroll
      for (int i = 0; i < 32 / VN; ++i) {
        const VT v = *reinterpret_cast<const VT *>(src + i * VN);
#pragma unroll
        for (int q = 0; q < VN; ++q) x[i * VN + q] = Vec16<T>::get(v, q);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        x[c] *= rd[c];
#pragma unroll
        for (int i = (c + 1) / VN; i < 32 / VN; ++i) {
          const VT lv = *reinterpret_cast<const VT *>(&Lt[c * 32 + i * VN]);
#pragma unroll
          for (int q = 0; q < VN; ++q)
            if (i * VN + q > c) x[i * VN + q] -= Vec16<T>::get(lv, q) * x[c];
        }
      }
#pragma unroll
      for (int i = 0; i < 32 / VN; ++i) {
        VT o;
#pragma unroll
        for (int q = 0; q < VN; ++q) Vec16<T>::set(o, q, x[i * VN + q]);
        *reinterpret_cast<VT *>(src + i * VN) = o;
      }
#pragma unroll
      for (int t = 0; t < 32; ++t) PT[t * NR + p] = x[t];
    }
    __syncthreads();
    // rank-32 update of the panel columns [c0 + 32, w): rows as above (lower part for
    // the diagonal rows), 4 x 4 tiles; tiles straddle no part (both parts 4-aligned)
    const int jb = c0 + 32, ncol = w - jb;
    if (ncol > 0) {
      const int nd4 = (ndiag + 3) / 4, nr4 = (nrows + 3) / 4, nc4 = (ncol + 3) / 4;
      const int ntiles = (nd4 + nr4) * nc4;
      for (int mt = tid; mt < ntiles; mt += 256) {
        const int rq = mt / nc4, cq = mt % nc4;
        const bool own = rq >= nd4;
        const int p0 = own ? kPW + 4 * (rq - nd4) : jb + 4 * rq;
        const int j0 = jb + 4 * cq;
        if (!own && p0 + 3 < j0) continue;  // strictly above the diagonal
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
          T av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; i += VN) {
            const VT x = *reinterpret_cast<const VT *>(&PT[k * NR + p0 + i]);
            const VT y = *reinterpret_cast<const VT *>(&PT[k * NR + j0 + i]);
#pragma unroll
            for (int q = 0; q < VN; ++q) { av[i + q] = Vec16<T>::get(x, q); bv[i + q] = Vec16<T>::get(y, q); }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int p = p0 + i;
          if (own ? (p - kPW >= nrows) : (p >= w)) continue;
          T *row = prow(p);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j0 + j < w) row[j0 + j] -= acc[i][j];
        }
      }
    }
  }
  if (bad && tid == 0) atomicOr(err, DEV_ERR_NOT_SPD);
  __syncthreads();
  // own rows back to the matrix; the diagonal launch also writes L_11 (lower part)
  for (int idx = tid; idx < nrows * VPP; idx += 256) {
    const int q = idx / VPP, cv = idx % VPP;
    if (cv * VN >= w) continue;
    const T *src = P + (OWN0 + q) * kLDP + cv * VN;
    T *dst = A + (long long)br.row(v0 + q) * d.ld + K0 + cv * VN;
    if (cv * VN + VN <= w) {
      *reinterpret_cast<VT *>(dst) = *reinterpret_cast<const VT *>(src);
    } else {
      for (int u = 0; cv * VN + u < w; ++u) dst[u] = src[u];
    }
  }
  if (!ROWS) {
    for (int idx = tid; idx < w * w; idx += 256) {
      const int i = idx / w, j = idx % w;
      if (j <= i) A[(long long)(K0 + i) * d.ld + K0 + j] = P[i * kLDP + j];
    }
  }
}

// ---- inverse of a factored diagonal block (tensor-core panel solve) -------------
// L_11^-1 for the w x w factored diagonal block at [K0, K0 + w) of every matrix (one CTA
// each), into pinv (128 x 128 per matrix, row-major, zero outside the lower w x w part), so
// that the rows below the panel become one product L_21 = A_21 L_11^-T on the tensor cores.
// 32 x 32 blocks: the four diagonal blocks by substitution (warp b, lane = column, the column
// in registers), then the blocks at distance 1, 2, 3 below the diagonal,
// Y_ij = -Y_ii (sum_{k=j}^{i-1} L_ik Y_kj), all threads over the entries of one distance.
constexpr int kInvLD = kPW + 1;
constexpr size_t kInvSmem = sizeof(float) * (2 * (size_t)kPW * kInvLD + 3 * 32 * 33);

__global__ void __launch_bounds__(256, 1) k_diag_inverse(const MatDesc *__restrict__ desc,
                                                         const float *__restrict__ base, int K0,
                                                         float *__restrict__ pinv) {
  const MatDesc d = desc[blockIdx.y];
  if (K0 >= d.e) return;
  const int w = min(kPW, d.e - K0), nbk = (w + 31) / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *Ls = reinterpret_cast<float *>(smem_raw);  // [128][129] L_11, lower, identity past w
  float *Ys = Ls + kPW * kInvLD;                      // [128][129] the inverse
  float *Tm = Ys + kPW * kInvLD;                      // [3][32][33] sums of one distance
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float *A = base + d.off + (long long)K0 * d.ld + K0;
  for (int e = tid; e < kPW * kPW; e += 256) {
    const int i = e / kPW, j = e % kPW;
    float v = 0.f;
    if (i < w && j < w) v = j <= i ? A[(long long)i * d.ld + j] : 0.f;
    else if (i == j) v = 1.f;
    Ls[i * kInvLD + j] = v;
    Ys[i * kInvLD + j] = 0.f;
  }
  __syncthreads();
  if (warp < 4) {  // diagonal block b = warp: lane = column j, forward substitution down the rows
    const int b0 = 32 * warp;
    float y[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float sacc = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < i; ++k) sacc -= Ls[(b0 + i) * kInvLD + b0 + k] * y[k];
      y[i] = sacc / Ls[(b0 + i) * kInvLD + b0 + i];
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) Ys[(b0 + i) * kInvLD + b0 + lane] = i >= lane ? y[i] : 0.f;
  }
  __syncthreads();
  for (int dist = 1; dist < nbk; ++dist) {
    const int nblk = nbk - dist;  // output blocks (j + dist, j), j < nblk
    for (int e = tid; e < nblk * 1024; e += 256) {
      const int j = e / 1024, r = (e % 1024) / 32, c = e % 32, i = j + dist;
      float t = 0.f;
      for (int k = j; k < i; ++k)
#pragma unroll 8
        for (int q = 0; q < 32; ++q) t += Ls[(32 * i + r) * kInvLD + 32 * k + q] * Ys[(32 * k + q) * kInvLD + 32 * j + c];
      Tm[(j * 32 + r) * 33 + c] = t;
    }
    __syncthreads();
    for (int e = tid; e < nblk * 1024; e += 256) {
      const int j = e / 1024, r = (e % 1024) / 32, c = e % 32, i = j + dist;
      float t = 0.f;
#pragma unroll 8
      for (int q = 0; q < 32; ++q) t += Ys[(32 * i + r) * kInvLD + 32 * i + q] * Tm[(j * 32 + q) * 33 + c];
      Ys[(32 * i + r) * kInvLD + 32 * j + c] = -t;
    }
    __syncthreads();
  }
  float *out = pinv + (long long)blockIdx.y * kPW * kPW;
  for (int e = tid; e < kPW * kPW; e += 256) {
    const int i = e / kPW, j = e % kPW;
    out[e] = (i < w && j < w && j <= i) ? Ys[i * kInvLD + j] : 0.f;
  }
}

// ---- rank-k update of lower tiles --------------------------------------------
// Two-level right-looking blocking: inner panels of kNB columns inside outer
// panels [K0, K1) of kOB columns.
// mode 0 (inner): rows [k0+w, m), cols [k0+w, min(K1, e)), K = [k0, k0+w), w = one engine panel
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
    const int w = min(kEnginePanel, d.e - k0);
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
  const BandRows br = band_rows(d, row0, ke);  // rows past the band hold zeros in K = [kb, ke)
  if (mode != 1) colend = min(colend, band_limit(d, ke));
  const int ti = blockIdx.x / nct, tj = blockIdx.x % nct;
  if (tj > ti) return;
  const int v0 = ti * kTB, c0 = row0 + tj * kTB;
  if (mode == 1 && d.ifirst && v0 < br.nv) kb = max(kb, d.ifirst[v0] & ~3);  // rows' L starts there
  if (v0 >= br.nv || c0 >= colend || ke <= kb) return;
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
      const bool va = v0 + lr < br.nv;
      const int ra = va ? br.row(v0 + lr) : 0, rb = c0 + lr;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = kk + lk + q;
        As[lk + q][lr] = (va && k < ke) ? A[(long long)ra * d.ld + k] : T(0);
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
    const int v = v0 + ty + 16 * i;
    if (v >= br.nv) continue;
    const int r = br.row(v);
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
    const int w = min(kEnginePanel, d.e - k0);
    row0 = k0 + w; colend = min(K1, d.e); kb = k0; ke = k0 + w;
  } else if (mode == 2) {
    if (K1 >= d.e) return;
    row0 = K1; colend = d.e; kb = K0; ke = K1;
  } else {
    row0 = d.e; colend = d.m; kb = 0; ke = d.e;
  }
  const BandRows br = band_rows(d, row0, ke);  // rows past the band hold zeros in K = [kb, ke)
  if (mode != 1) colend = min(colend, band_limit(d, ke));
  const int ti = blockIdx.x / nct, tj = blockIdx.x % nct;
  if (tj > ti) return;
  const int v0 = ti * kTB2, c0 = row0 + tj * kTB2;
  if (mode == 1 && d.ifirst && v0 < br.nv) kb = max(kb, d.ifirst[v0] & ~3);  // rows' L starts there
  if (v0 >= br.nv || c0 >= colend || ke <= kb) return;
  float *A = base + d.off;
  __shared__ __align__(16) float As[2][kKC2][kTB2 + 4];
  __shared__ __align__(16) float Bs[2][kKC2][kTB2 + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // loader: thread -> (row lr, k offset lk): 128 rows x 16 k = 2 x 4 floats per thread per operand
  const int lr = tid >> 1, lk = (tid & 1) * 8;
  const bool va = v0 + lr < br.nv;
  const int ra = va ? br.row(v0 + lr) : 0, rb = c0 + lr;
  const bool vb = rb < colend;
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
    const int v = v0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (v >= br.nv) continue;
    float *crow = A + (long long)br.row(v) * d.ld;
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

// Lower-triangle entries that a band-limited update of rows band_rows(hd, t0, ke) x columns
// [t0, cend) touches: the interior rows up to the band (a trapezoid), then every column of
// the rows from e on (for a dense matrix: rows [t0, m) x columns [t0, cend), c <= r).
static double band_entries(const MatDesc &hd, int t0, int ke, int cend) {
  const long long k = cend - t0;
  if (k <= 0) return 0.0;
  const BandRows br = band_rows(hd, t0, ke);
  const long long iend = t0 + br.ni;
  const long long a = std::max(0LL, std::min(iend, (long long)cend) - t0);
  const long long b = std::max(0LL, iend - cend);
  return (double)(a * (a + 1) / 2 + b * k + (long long)(br.nv - br.ni) * k);
}

template <typename T>
void engine_partial_cholesky(const EngineShape &sh, const MatDesc *d_desc, T *base, int *d_err, cudaStream_t s,
                             T *store, ProfHook *prof, bool tc, float *pinv) {
  if (sh.count == 0) return;
  constexpr int RB = PanelRows<T>::RB;
  const int ob = std::max(kPW, (sh.ob / kPW) * kPW);  // outer block: columns per long-K trailing update
  // host copies of the descriptors' sizes and bands: the grids cover the rows and columns
  // the band lets an update reach (the kernels apply the same limits per matrix)
  std::vector<MatDesc> hd(sh.count);
  for (int b = 0; b < sh.count; ++b) {
    hd[b].m = sh.m[b];
    hd[b].e = sh.e[b];
    if (!sh.band.empty()) hd[b].band = sh.band[b];
    if (!sh.id0.empty()) hd[b].id0 = sh.id0[b];
    if (!sh.ifirst.empty()) hd[b].ifirst = sh.ifirst[b];
  }
  for (int K0 = 0; K0 < sh.max_e; K0 += ob) {
    const int K1 = K0 + ob;
    for (int k0 = K0; k0 < std::min(K1, sh.max_e); k0 += kPW) {
      int max_below = 0, max_cols = 0;
      double fl_panel = 0.0, fl_in = 0.0;
      for (int b = 0; b < sh.count; ++b) {
        if (k0 >= sh.e[b]) continue;
        const int w = std::min(kPW, sh.e[b] - k0);
        const int below = band_rows(hd[b], k0 + w, k0 + w).nv;
        const int cend = std::min({K1, sh.e[b], band_limit(hd[b], k0 + w)});
        max_below = std::max(max_below, below);
        max_cols = std::max(max_cols, cend - k0 - w);
        fl_panel += (double)w * w * w / 3.0 + (double)below * w * w;
        fl_in += 2.0 * w * band_entries(hd[b], k0 + w, k0 + w, cend);
      }
      if (prof) prof->begin(PROF_PANEL, s);
      k_bigpanel<T, false><<<dim3(1, sh.count), 256, bigpanel_smem<T, false>(), s>>>(d_desc, base, k0, d_err, store);
      count_launch();
      if (max_below > 0) {
        bool done_rows = false;
        if constexpr (std::is_same<T, float>::value) {
          if (tc && pinv) {  // L_21 = A_21 L_11^-T as one tensor-core product with the block's inverse
            k_diag_inverse<<<dim3(1, sh.count), 256, kInvSmem, s>>>(d_desc, base, k0, pinv);
            count_launch();
            launch_rankk_tc(d_desc, base, 3, k0, 0, max_below, kPW, sh.count, d_err, s, pinv);
            done_rows = true;
          }
        }
        if (!done_rows) {
          k_bigpanel<T, true><<<dim3(ceil_div(max_below, RB), sh.count), 256, bigpanel_smem<T, true>(), s>>>(
              d_desc, base, k0, d_err, store);
          count_launch();
        }
      }
      if (prof) prof->end(PROF_PANEL, s, fl_panel, 0.0);
      // the rest of the outer block: rows [k0 + w, m), columns [k0 + w, min(K1, e)); timed
      // with the panels (the long-K class holds only the trailing updates)
      if (max_below > 0 && max_cols > 0) {
        if (prof) prof->begin(PROF_PANEL, s);
        if constexpr (std::is_same<T, float>::value) {
          static_assert(kPW == 128, "the tensor-core in-block update takes 128-column panels");
          if (tc) launch_rankk_tc(d_desc, base, 0, k0, K1, max_below, max_cols, sh.count, d_err, s);
          else launch_rankk<T>(d_desc, base, 0, k0, K0, K1, max_below, max_cols, sh.count, s);
        } else {
          launch_rankk<T>(d_desc, base, 0, k0, K0, K1, max_below, max_cols, sh.count, s);
        }
        if (prof) prof->end(PROF_PANEL, s, fl_in, 0.0);
      }
    }
    // outer update of the trailing columns [K1, e) with the finished outer panel
    int max_rows = 0, max_cols = 0;
    double fl = 0.0, by = 0.0;
    for (int b = 0; b < sh.count; ++b) {
      if (K1 >= sh.e[b]) continue;
      const int rows = band_rows(hd[b], K1, K1).nv, cend = band_limit(hd[b], K1);
      max_rows = std::max(max_rows, rows);
      max_cols = std::max(max_cols, cend - K1);
      const double ent = band_entries(hd[b], K1, K1, cend);
      fl += 2.0 * ob * ent;
      by += sizeof(T) * (2.0 * ent + (double)ob * rows);
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
    const int rows = band_rows(hd[b], sh.e[b], sh.e[b]).nv;  // rows whose L row is not zero
    max_t = std::max(max_t, rows);
    const double n2 = sh.m[b] - sh.e[b];
    if (hd[b].ifirst) {  // row g of the trailing block needs K from ifirst[g] on
      for (int g = 0; g < rows; ++g) {
        const double k = sh.e[b] - (hd[b].ifirst[g] & ~3);
        fl += 2.0 * k * (g + 1);
        by += sizeof(T) * (2.0 * (g + 1) + k);
      }
    } else {
      const double ent = n2 * (n2 + 1) / 2.0;
      fl += 2.0 * sh.e[b] * ent;
      by += sizeof(T) * (2.0 * ent + n2 * sh.e[b]);
    }
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
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

// ---- batched symmetric GEMV: S CTAs (8 warps each) per matrix ---------------
// The matrix is read as 32 x 32 tiles of its lower block triangle, each once: tile (I, J),
// J < I, serves both y_I += A_IJ x_J and y_J += A_IJ^T x_I; a diagonal tile serves
// y_I += A_II x_I.  CTA s of a matrix takes the s-th of S contiguous runs of the row-major
// tile order and splits it over its warps the same way; a warp holds the next tile in
// registers (16-byte loads, a 128-byte row segment per 32 / VN lanes) while it multiplies
// the current one from its shared-memory copy (row sums: lane = tile row; column sums:
// lane = tile column) and adds both into its own partial vector, so no two warps write the
// same word.  The CTA adds its warps' vectors in warp order; with S > 1 it stores the sum in
// `scratch` and the last CTA of the matrix to finish (counter per matrix, reset by that CTA)
// adds the S sums in order s = 0 .. S-1.  Deterministic; half the bytes of a full GEMV.
// Plain rows of B go to the CTAs round-robin.
template <typename T>
__global__ void __launch_bounds__(256) k_symv_batched(const SymvTask *__restrict__ tasks, const T *__restrict__ A,
                                                      const double *__restrict__ x, const int *__restrict__ xidx,
                                                      double *__restrict__ y, double alpha, const int *__restrict__ done,
                                                      T *__restrict__ scratch, int *__restrict__ counter, int ld_scr) {
  if (done && *done) return;
  using VT = typename Vec16<T>::V;
  constexpr int VN = Vec16<T>::N;
  constexpr int LPR = 32 / VN;       // lanes per 32-wide tile row
  constexpr int RPI = 32 / LPR;      // tile rows per warp instruction
  constexpr int TPL = 32 / RPI;      // vectors per lane per tile
  const SymvTask t = tasks[blockIdx.y];
  const int S = gridDim.x, sidx = blockIdx.x;
  const int n = t.n, nb = (n + 31) >> 5, np = nb * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);  // [np]
  T *part = xs + np;                         // [8][np]
  T *tiles = part + 8 * np;                  // [8][32][33]
  __shared__ int last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c = tid; c < np; c += 256)
    xs[c] = c < n ? (T)((t.flags & 1) ? x[xidx[t.x_off + c]] : x[t.x_off + c]) : T(0);
  for (int c = tid; c < 8 * np; c += 256) part[c] = T(0);
  __syncthreads();
  const T *a = A + t.a_off;
  T *tile = tiles + warp * 32 * 33;
  T *mine = part + warp * np;
  const long long ntiles = (long long)nb * (nb + 1) / 2;
  const long long c0 = ntiles * sidx / S, c1 = ntiles * (sidx + 1) / S;  // this CTA's run
  const int s0 = (int)(c0 + (c1 - c0) * warp / 8), s1 = (int)(c0 + (c1 - c0) * (warp + 1) / 8);
  // tile index s = I (I + 1) / 2 + J  ->  (I, J)
  int I = 0;
  while ((I + 1) * (I + 2) / 2 <= s0) ++I;
  int J = s0 - I * (I + 1) / 2;
  const int lr = lane / LPR, lc = (lane % LPR) * VN;  // this lane's row in a group and column
  VT buf[TPL];
  auto load = [&](int ti, int tj) {
#pragma unroll
    for (int i = 0; i < TPL; ++i) {
      const int r = 32 * ti + i * RPI + lr, c = 32 * tj + lc;
      VT v = (r < n && c < n) ? *reinterpret_cast<const VT *>(a + (long long)r * t.ld + c) : VT{};
#pragma unroll
      for (int q = 0; q < VN; ++q)
        if (c + q >= n) Vec16<T>::set(v, q, T(0));
      buf[i] = v;
    }
  };
  if (s0 < s1) load(I, J);
  for (int s = s0; s < s1; ++s) {
#pragma unroll
    for (int i = 0; i < TPL; ++i)
#pragma unroll
      for (int q = 0; q < VN; ++q) tile[(i * RPI + lr) * 33 + lc + q] = Vec16<T>::get(buf[i], q);
    __syncwarp();
    const int ci = I, cj = J;
    if (++J > I) { ++I; J = 0; }
    if (s + 1 < s1) load(I, J);  // in flight while this tile is multiplied
    T rsum = T(0);
#pragma unroll 8
    for (int c = 0; c < 32; ++c) rsum += tile[lane * 33 + c] * xs[32 * cj + c];
    mine[32 * ci + lane] += rsum;
    if (cj < ci) {
      T csum = T(0);
#pragma unroll 8
      for (int r = 0; r < 32; ++r) csum += tile[r * 33 + lane] * xs[32 * ci + r];
      mine[32 * cj + lane] += csum;
    }
    __syncwarp();
  }
  // plain rows of B: one warp per row, rows dealt to the CTAs round-robin
  for (int r = sidx + S * warp; r < t.nb; r += 8 * S) {
    const T *brow = A + t.b_off + (long long)r * t.ld;
    T acc = T(0);
    for (int c = lane; c < n; c += 32) acc += brow[c] * xs[c];
    acc = warp_sum(acc);
    if (lane == 0) {
      const double v = alpha * (double)acc;
      y[t.yb_off + r] = (t.flags & 2) ? y[t.yb_off + r] + v : v;
    }
  }
  __syncthreads();
  if (S == 1) {
    for (int r = tid; r < n; r += 256) {
      T v = part[r];
#pragma unroll
      for (int w = 1; w < 8; ++w) v += part[w * np + r];
      const double o = alpha * (double)v;
      y[t.y_off + r] = (t.flags & 2) ? y[t.y_off + r] + o : o;
    }
    return;
  }
  T *mysum = scratch + ((long long)blockIdx.y * S + sidx) * ld_scr;
  for (int r = tid; r < n; r += 256) {
    T v = part[r];
#pragma unroll
    for (int w = 1; w < 8; ++w) v += part[w * np + r];
    mysum[r] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(&counter[blockIdx.y], 1) == S - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const T *sums = scratch + (long long)blockIdx.y * S * ld_scr;
  for (int r = tid; r < n; r += 256) {
    T v = __ldcg(sums + r);
    for (int q = 1; q < S; ++q) v += __ldcg(sums + (long long)q * ld_scr + r);
    const double o = alpha * (double)v;
    y[t.y_off + r] = (t.flags & 2) ? y[t.y_off + r] + o : o;
  }
  if (tid == 0) counter[blockIdx.y] = 0;  // ready for the next launch
}

template <typename T>
size_t symv_smem(int max_n) {
  const size_t np = (size_t)((max_n + 31) / 32) * 32;
  return sizeof(T) * (9 * np + 8 * 32 * 33);
}

// CTAs per matrix: one while the matrices alone fill the resident slots (a split costs a
// partial-sum round trip and shorter prefetch runs), else enough to fill one wave, with at
// least 8 tiles per CTA (one per warp) and at most 16.  slots = 0: one CTA per matrix.
int symv_split(int ntasks, int max_n, int slots) {
  if (slots <= 0 || ntasks <= 0 || ntasks >= slots) return 1;
  const long long nb = (max_n + 31) / 32, ntiles = nb * (nb + 1) / 2;
  const int smax = (int)std::max<long long>(1, std::min<long long>(16, ntiles / 8));
  return std::max(1, std::min(smax, (slots + ntasks - 1) / ntasks));
}

template <typename T>
int symv_occupancy(int max_n) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_symv_batched<T>, 256, symv_smem<T>(max_n)) != cudaSuccess)
    return 0;
  return occ;
}

template <typename T>
void launch_symv_batched(int ntasks, int max_n, int split, const SymvTask *d_tasks, const T *A, const double *x,
                         const int *xidx, double *y, double alpha, const int *done, T *scratch, int *counter,
                         int ld_scr, cudaStream_t s) {
  if (ntasks == 0 || max_n == 0) return;
  k_symv_batched<T><<<dim3(split, ntasks), 256, symv_smem<T>(max_n), s>>>(d_tasks, A, x, xidx, y, alpha, done,
                                                                          scratch, counter, ld_scr);
  count_launch();
}

// y[a] = (acc ? y[a] : 0) + alpha sum_p A[p][a] x[p]: one CTA per (task, 32 columns);
// x may instead be a sparse product evaluated while staging (csr.ptr set).
// lane = column (coalesced rows), the 8 warps split the rows with 4 loads in flight
// each and add up their partial sums in shared memory in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv_t(const GemvDesc *__restrict__ tasks, const T *__restrict__ A,
                                                const double *__restrict__ x, const int *__restrict__ xidx,
                                                double *__restrict__ y, double alpha, const int *__restrict__ done,
                                                const CsrIn csr) {
  if (done && *done) return;
  const GemvDesc t = tasks[blockIdx.y];
  const int c0 = blockIdx.x * 32;
  if (c0 >= t.cols) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  __shared__ T part[8][33];
  for (int p = threadIdx.x; p < t.rows; p += blockDim.x)
    xs[p] = (T)(csr.ptr ? csr_row(csr, t.x_off + p) : (t.flags & 1) ? x[xidx[t.x_off + p]] : x[t.x_off + p]);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int a = c0 + lane;
  const bool va = a < t.cols;
  const T *col = A + t.a_off + (va ? a : c0);
  const long long ld = t.ld;
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int p = wid;
  for (; p + 24 < t.rows; p += 32) {
    a0 += col[p * ld] * xs[p];
    a1 += col[(p + 8) * ld] * xs[p + 8];
    a2 += col[(p + 16) * ld] * xs[p + 16];
    a3 += col[(p + 24) * ld] * xs[p + 24];
  }
  for (; p < t.rows; p += 8) a0 += col[p * ld] * xs[p];
  part[wid][lane] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (wid == 0 && va) {
    T sum = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += part[k][lane];
    const double v = alpha * (double)sum;
    y[t.y_off + a] = (t.flags & 2) ? y[t.y_off + a] + v : v;
  }
}

// Batched GEMVs of many small matrices (deluxe blocks, Psi): one CTA per task covering all of
// its rows / columns, so the staging of x and the task descriptor are paid once per matrix.
// y = alpha A x (+ y): 8 warps over the rows, two rows at a time per warp, lanes over the
// columns (coalesced rows).
template <typename T>
__global__ void __launch_bounds__(256) k_gemv_task(const GemvDesc *__restrict__ tasks, const T *__restrict__ A,
                                                   const double *__restrict__ x, const int *__restrict__ xidx,
                                                   double *__restrict__ y, double alpha,
                                                   const int *__restrict__ done) {
  if (done && *done) return;
  const GemvDesc t = tasks[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  for (int c = threadIdx.x; c < t.cols; c += blockDim.x)
    xs[c] = (T)((t.flags & 1) ? x[xidx[t.x_off + c]] : x[t.x_off + c]);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r0 = 2 * wid; r0 < t.rows; r0 += 16) {
    const int r1 = r0 + 1;
    const bool v1 = r1 < t.rows;
    const T *row0 = A + t.a_off + (long long)r0 * t.ld;
    const T *row1 = A + t.a_off + (long long)(v1 ? r1 : r0) * t.ld;
    T a0 = T(0), b0 = T(0);
    for (int c = lane; c < t.cols; c += 32) {
      const T xv = xs[c];
      a0 += row0[c] * xv;
      b0 += row1[c] * xv;
    }
    const T s0 = warp_sum(a0), s1 = warp_sum(b0);
    if (lane == 0) {
      const double v = alpha * (double)s0;
      y[t.y_off + r0] = (t.flags & 2) ? y[t.y_off + r0] + v : v;
      if (v1) {
        const double w = alpha * (double)s1;
        y[t.y_off + r1] = (t.flags & 2) ? y[t.y_off + r1] + w : w;
      }
    }
  }
}

// y[a] = (acc ? y[a] : 0) + alpha sum_p A[p][a] x[p]: one CTA per task, one thread per column
// (coalesced rows), x staged (gathered, or a sparse product when csr.ptr is set).
template <typename T>
__global__ void __launch_bounds__(256) k_gemv_t_task(const GemvDesc *__restrict__ tasks, const T *__restrict__ A,
                                                     const double *__restrict__ x, const int *__restrict__ xidx,
                                                     double *__restrict__ y, double alpha,
                                                     const int *__restrict__ done, const CsrIn csr) {
  if (done && *done) return;
  const GemvDesc t = tasks[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  for (int p = threadIdx.x; p < t.rows; p += blockDim.x)
    xs[p] = (T)(csr.ptr ? csr_row(csr, t.x_off + p) : (t.flags & 1) ? x[xidx[t.x_off + p]] : x[t.x_off + p]);
  __syncthreads();
  const T *base = A + t.a_off;
  const long long ld = t.ld;
  for (int a = threadIdx.x; a < t.cols; a += blockDim.x) {
    T a0 = T(0), a1 = T(0);
    int p = 0;
    for (; p + 1 < t.rows; p += 2) {
      a0 += base[p * ld + a] * xs[p];
      a1 += base[(p + 1) * ld + a] * xs[p + 1];
    }
    if (p < t.rows) a0 += base[p * ld + a] * xs[p];
    const double v = alpha * (double)(a0 + a1);
    y[t.y_off + a] = (t.flags & 2) ? y[t.y_off + a] + v : v;
  }
}

template <typename T>
void launch_gemv_task(int ntasks, int max_rows, int max_cols, const GemvDesc *d_tasks, const T *A, const double *x,
                      const int *xidx, double *y, double alpha, const int *done, cudaStream_t s) {
  if (ntasks == 0 || max_rows == 0) return;
  k_gemv_task<T><<<ntasks, 256, sizeof(T) * (size_t)std::max(1, max_cols), s>>>(d_tasks, A, x, xidx, y, alpha, done);
  count_launch();
}

template <typename T>
void launch_gemv_t_task(int ntasks, int max_rows, int max_cols, const GemvDesc *d_tasks, const T *A,
                        const double *x, const int *xidx, double *y, double alpha, const int *done, cudaStream_t s,
                        const CsrIn *csr) {
  if (ntasks == 0 || max_cols == 0) return;
  const int threads = max_cols <= 128 ? 128 : 256;
  k_gemv_t_task<T><<<ntasks, threads, sizeof(T) * (size_t)std::max(1, max_rows), s>>>(
      d_tasks, A, x, xidx, y, alpha, done, csr ? *csr : CsrIn{});
  count_launch();
}

// y (+)= A x for one large symmetric matrix stored in full (n x n, row-major, ld a multiple
// of 8, zero padding columns), reading only its lower block triangle.  The CTA of rows
// [I0, I0 + 8) takes
//   the row strip     A[I0 .. I0+8)[0 .. I0+8)   (diagonal 8 x 8 block included; one warp
//                     per row, 16-byte loads, four in flight per lane), and
//   the column strip  A[I0+8 .. n)[I0 .. I0+8)   (the symmetric images of the same rows'
//                     entries right of the diagonal block; 16-byte loads, 32 / (8 / VN) rows
//                     per warp instruction, four instructions in flight),
// so every CTA reads n x 8 values and the kernel touches half the matrix: the repeated
// products of an iterative refinement find it in L2.  x staged in shared memory in T,
// accumulation in T, partial sums added in a fixed order.  The coarse solve of large
// coarse problems.
template <typename T>
__global__ void __launch_bounds__(256) k_symv_rows(int n, const T *__restrict__ A, int ld,
                                                   const double *__restrict__ x, double *__restrict__ y,
                                                   int accumulate, const int *__restrict__ done) {
  if (done && *done) return;
  using VT = typename Vec16<T>::V;
  constexpr int VN = Vec16<T>::N;
  constexpr int LPR = 8 / VN;    // lanes per 8-wide row segment of the column strip
  constexpr int RPI = 32 / LPR;  // column-strip rows per warp instruction
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  __shared__ T part[8][8];  // [warp][column of the block]: column-strip sums
  const int npad = (n + 7) & ~7;
  for (int c = threadIdx.x; c < npad; c += blockDim.x) xs[c] = c < n ? (T)x[c] : T(0);
  __syncthreads();
  const int I0 = blockIdx.x * 8, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = I0 + warp;
  // row strip: columns [0, I0 + 8) (I0 + 8 <= npad; padding columns are zero)
  T rs = T(0);
  if (row < n) {
    const VT *a = reinterpret_cast<const VT *>(A + (long long)row * ld);
    const VT *xv = reinterpret_cast<const VT *>(xs);
    const int nv = (I0 + 8) / VN;
    T acc0 = T(0), acc1 = T(0), acc2 = T(0), acc3 = T(0);
    int v = lane;
    for (; v + 96 < nv; v += 128) {
      const VT a0 = a[v], a1 = a[v + 32], a2 = a[v + 64], a3 = a[v + 96];
      acc0 += Vec16<T>::dot(a0, xv[v]);
      acc1 += Vec16<T>::dot(a1, xv[v + 32]);
      acc2 += Vec16<T>::dot(a2, xv[v + 64]);
      acc3 += Vec16<T>::dot(a3, xv[v + 96]);
    }
    for (; v < nv; v += 32) acc0 += Vec16<T>::dot(a[v], xv[v]);
    rs = warp_sum((acc0 + acc1) + (acc2 + acc3));
  }
  // column strip: rows [I0 + 8, n), columns [I0, I0 + 8); lane -> (row in the group, vector)
  T cs[VN];
#pragma unroll
  for (int q = 0; q < VN; ++q) cs[q] = T(0);
  {
    const int sub = lane / LPR, seg = lane % LPR;
    const T *col = A + I0 + seg * VN;
    constexpr int kStride = 8 * RPI;  // rows between a warp's consecutive instructions
    for (int j = I0 + 8 + warp * RPI + sub; j < n; j += 4 * kStride) {
      VT v[4];
      T xj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int jj = j + u * kStride;
        v[u] = jj < n ? *reinterpret_cast<const VT *>(col + (long long)jj * ld) : VT{};
        xj[u] = jj < n ? xs[jj] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) Vec16<T>::axpy(cs, v[u], xj[u]);
    }
#pragma unroll
    for (int q = 0; q < VN; ++q)
#pragma unroll
      for (int off = LPR; off < 32; off <<= 1) cs[q] += __shfl_xor_sync(0xffffffffu, cs[q], off);
    if (sub == 0) {
#pragma unroll
      for (int q = 0; q < VN; ++q) part[warp][seg * VN + q] = cs[q];
    }
  }
  __syncthreads();
  if (lane == 0 && row < n) {
    T t = rs;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += part[w][warp];
    y[row] = accumulate ? y[row] + (double)t : (double)t;
  }
}

template <typename T>
void launch_symv_rows(int n, const T *A, int ld, const double *x, double *y, int accumulate, const int *done,
                      cudaStream_t s) {
  if (n == 0) return;
  k_symv_rows<T><<<ceil_div(n, 8), 256, sizeof(T) * (size_t)((n + 7) & ~7), s>>>(n, A, ld, x, y, accumulate, done);
  count_launch();
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
                   const int *xidx, double *y, double alpha, const int *done, cudaStream_t s, const CsrIn *csr) {
  if (ntasks == 0 || max_cols == 0) return;
  dim3 g(ceil_div(max_cols, 32), ntasks);
  const size_t sm = sizeof(T) * (size_t)std::max(1, max_rows);
  k_gemv_t<T><<<g, 256, sm, s>>>(d_tasks, A, x, xidx, y, alpha, done, csr ? *csr : CsrIn{});
  count_launch();
}

// ---- batched triangular solves (one CTA of 32 warps per matrix) ---------------
// y = L^-1 b (lower, blocks in increasing order) or y = L^-T b (upper, decreasing),
// 32-row blocks, one barrier per block.  While warp 0 finishes block k (adds the
// contributions gathered for it, then substitutes with the factored diagonal block
// from the engine's store), warps 1..31 gather everything the next block needs
// that is already final: its diagonal block, the sums over the solved blocks before
// k (16-byte vector loads, several in flight per lane) and the 32 x 32 tile that
// couples it to block k.  Buffers alternate between blocks; the vector lives in
// shared memory.
template <typename T>
__global__ void __launch_bounds__(1024) k_trsv(const MatDesc *__restrict__ desc, const int *__restrict__ vec_off,
                                               const T *__restrict__ base, const T *__restrict__ store,
                                               const double *__restrict__ b, double *__restrict__ y, int transpose) {
  using VT = typename Vec16<T>::V;
  constexpr int VN = Vec16<T>::N, VPR = kNB / VN, RPW = 32 / VPR;
  const MatDesc d = desc[blockIdx.x];
  const int n = d.e;
  const T *L = base + d.off;
  // dynamic shared memory: six 32 x 33 tiles, then the vector
  typedef T Tile[32][33];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tile *Lb = reinterpret_cast<Tile *>(smem_raw);  // [2] diagonal block
  Tile *Lt = Lb + 2;    // [2] coupling tile: lower Lt[j][c] = L[r0n + j][r0 + c]; upper Lt[c][j] = L[r0 + c][r0n + j]
  Tile *part = Lb + 4;  // [2] lower: part[0][j] = prefix sums; upper: part[w][j] per warp
  T *v = reinterpret_cast<T *>(Lb + 6);
  const int off = vec_off[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nblk = ceil_div(n, 32);
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = (T)b[off + i];
  if (nblk > 0) {
    const int b0 = transpose ? nblk - 1 : 0;
    Lb[0][wid][lane] = store[((long long)d.dblk + b0) * kNB * kNB + wid * kNB + lane];
  }
  __syncthreads();
  for (int q = 0; q < nblk; ++q) {
    const int buf = q & 1, nb = buf ^ 1;
    const int bk = transpose ? nblk - 1 - q : q;
    const int r0 = bk * 32, r1 = min(n, r0 + 32);
    if (wid == 0) {
      const int r = r0 + lane;
      T vr = (r < r1) ? v[r] : T(0);
      if (q > 0) {
        if (!transpose) {  // previous block [r0 - 32, r0)
          T s = part[buf][0][lane];
#pragma unroll 8
          for (int c = 0; c < 32; ++c) s += Lt[buf][lane][c] * v[r0 - 32 + c];
          vr -= s;
        } else {  // previous block [r1, min(n, r1 + 32))
          T s = T(0);
#pragma unroll 8
          for (int k = 1; k < 32; ++k) s += part[buf][k][lane];
          const int cnt = min(32, n - r1);
          for (int c = 0; c < cnt; ++c) s += Lt[buf][c][lane] * v[r1 + c];
          vr -= s;
        }
      }
      const T rdl = T(1) / Lb[buf][lane][lane];
      if (!transpose) {
        for (int c = 0; c < r1 - r0; ++c) {
          const T xc = __shfl_sync(0xffffffffu, vr * rdl, c);
          if (lane == c) vr = xc;
          else if (lane > c) vr -= Lb[buf][lane][c] * xc;
        }
      } else {
        for (int c = r1 - r0 - 1; c >= 0; --c) {
          const T xc = __shfl_sync(0xffffffffu, vr * rdl, c);
          if (lane == c) vr = xc;
          else if (lane < c) vr -= Lb[buf][c][lane] * xc;
        }
      }
      if (r < r1) v[r] = vr;
    } else {
      const int bn = transpose ? bk - 1 : bk + 1;  // next block
      if (bn >= 0 && bn < nblk) {
        const int r0n = bn * 32;
        for (int j = wid - 1; j < 32; j += 31)
          Lb[nb][j][lane] = store[((long long)d.dblk + bn) * kNB * kNB + j * kNB + lane];
        if (!transpose) {
          // rows r0n + j: prefix over the columns [0, r0) and the tile against [r0, r1)
          for (int j = wid - 1; j < 32; j += 31) {
            const int rn = r0n + j;
            T s = T(0), tv = T(0);
            if (rn < n) {
              const T *Lr = L + (long long)rn * d.ld;
              tv = Lr[r0 + lane];  // r1 - r0 = 32 here: block k is not the last one
              const VT *Lv = reinterpret_cast<const VT *>(Lr);
              const VT *vv = reinterpret_cast<const VT *>(v);
              const int nv = r0 / VN;
              // columns left of rn - band hold zeros (banded factor): start at the band
              const int i0 = d.band >= n ? 0 : max(0, rn - d.band) / VN;
              T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
              int i = i0 + lane;
              for (; i + 96 < nv; i += 128) {
                const VT l0 = Lv[i], l1 = Lv[i + 32], l2 = Lv[i + 64], l3 = Lv[i + 96];
                a0 += Vec16<T>::dot(l0, vv[i]);
                a1 += Vec16<T>::dot(l1, vv[i + 32]);
                a2 += Vec16<T>::dot(l2, vv[i + 64]);
                a3 += Vec16<T>::dot(l3, vv[i + 96]);
              }
              for (; i < nv; i += 32) a0 += Vec16<T>::dot(Lv[i], vv[i]);
              s = warp_sum((a0 + a1) + (a2 + a3));
            }
            Lt[nb][j][lane] = tv;
            if (lane == 0) part[nb][0][j] = s;
          }
        } else {
          // columns r0n + j (the next block): sums over the rows [r1, n), tile against the rows [r0, r1)
          const int cq = lane % VPR, rq = lane / VPR;
          T acc[VN];
#pragma unroll
          for (int u = 0; u < VN; ++u) acc[u] = T(0);
          const T *Lc = L + r0n + VN * cq;
          constexpr int kStep = 31 * RPW;
          // rows past the band of the block's last column hold zeros there (banded factor)
          const int cend = d.band >= n ? n : min(n, r0n + 32 + d.band);
          int c = r1 + RPW * (wid - 1) + rq;
          for (; c + 3 * kStep < cend; c += 4 * kStep) {
            const VT l0 = *reinterpret_cast<const VT *>(Lc + (long long)c * d.ld);
            const VT l1 = *reinterpret_cast<const VT *>(Lc + (long long)(c + kStep) * d.ld);
            const VT l2 = *reinterpret_cast<const VT *>(Lc + (long long)(c + 2 * kStep) * d.ld);
            const VT l3 = *reinterpret_cast<const VT *>(Lc + (long long)(c + 3 * kStep) * d.ld);
            Vec16<T>::axpy(acc, l0, v[c]);
            Vec16<T>::axpy(acc, l1, v[c + kStep]);
            Vec16<T>::axpy(acc, l2, v[c + 2 * kStep]);
            Vec16<T>::axpy(acc, l3, v[c + 3 * kStep]);
          }
          for (; c < cend; c += kStep)
            Vec16<T>::axpy(acc, *reinterpret_cast<const VT *>(Lc + (long long)c * d.ld), v[c]);
#pragma unroll
          for (int u = 0; u < VN; ++u)
#pragma unroll
            for (int o = VPR; o < 32; o <<= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
          if (rq == 0)
#pragma unroll
            for (int u = 0; u < VN; ++u) part[nb][wid][VN * cq + u] = acc[u];
          for (int j = wid - 1; j < 32; j += 31)
            Lt[nb][j][lane] = (r0 + j < r1) ? L[(long long)(r0 + j) * d.ld + r0n + lane] : T(0);
        }
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[off + i] = (double)v[i];
}

template <typename T>
void launch_trsv(int count, int max_n, const MatDesc *d_desc, const int *vec_off, const T *base, const T *store,
                 const double *b, double *y, bool transpose, cudaStream_t s) {
  if (count == 0) return;
  const size_t sm = sizeof(T) * (6 * 32 * 33 + (size_t)std::max(4, max_n + 4));
  k_trsv<T><<<count, 1024, sm, s>>>(d_desc, vec_off, base, store, b, y, transpose ? 1 : 0);
  count_launch();
}

// Large local problems stage vectors of up to ~25k entries in shared memory.
size_t dense_smem_limit() { return 200 * 1024; }
bool dense_configure() {
  const int lim = (int)dense_smem_limit();
  bool ok = true;
  ok &= cudaFuncSetAttribute(k_diag_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvSmem) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_bigpanel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bigpanel_smem<float, false>()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_bigpanel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bigpanel_smem<float, true>()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_bigpanel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bigpanel_smem<double, false>()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_bigpanel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bigpanel_smem<double, true>()) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_trsv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_trsv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv_t<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv_t<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_symv_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_symv_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_symv_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) ==
        cudaSuccess;
  ok &= cudaFuncSetAttribute(k_symv_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv_task<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv_task<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv_t_task<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  ok &= cudaFuncSetAttribute(k_gemv_t_task<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
  return ok;
}

#define BD_INST(T)                                                                                              \
  template void engine_partial_cholesky<T>(const EngineShape &, const MatDesc *, T *, int *, cudaStream_t,    \
                                           T *, ProfHook *, bool, float *);                                    \
  template void launch_gemv<T>(int, int, int, const GemvDesc *, const T *, const double *, const int *,        \
                               double *, double, const int *, cudaStream_t);                                   \
  template void launch_symv_rows<T>(int, const T *, int, const double *, double *, int, const int *,           \
                                    cudaStream_t);                                                             \
  template size_t symv_smem<T>(int);                                                                           \
  template int symv_occupancy<T>(int);                                                                         \
  template void launch_symv_batched<T>(int, int, int, const SymvTask *, const T *, const double *, const int *,\
                                       double *, double, const int *, T *, int *, int, cudaStream_t);          \
  template void launch_gemv_task<T>(int, int, int, const GemvDesc *, const T *, const double *, const int *,   \
                                    double *, double, const int *, cudaStream_t);                              \
  template void launch_gemv_t_task<T>(int, int, int, const GemvDesc *, const T *, const double *, const int *, \
                                      double *, double, const int *, cudaStream_t, const CsrIn *);             \
  template void launch_gemv_t<T>(int, int, int, const GemvDesc *, const T *, const double *, const int *,      \
                                 double *, double, const int *, cudaStream_t, const CsrIn *);                  \
  template void launch_trsv<T>(int, int, const MatDesc *, const int *, const T *, const T *, const double *,   \
                               double *, bool, cudaStream_t);
BD_INST(float)
BD_INST(double)

}  // namespace bd
