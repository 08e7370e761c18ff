// Shared device helpers for the Bidomain GB300 library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace bd {

// device error flag bits (reported by the host as BD_ERR_*)
enum : int { DEV_ERR_NOT_SPD = 1, DEV_ERR_NAN = 2, DEV_ERR_TIMEOUT = 4 };

constexpr int kWarp = 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block reduction of one value per thread (fixed tree order).
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) v = warp_sum(v);
  __syncthreads();
  return v;  // valid in thread 0
}

// Batched dense matrix descriptor (row-major, leading dimension ld).
struct MatDesc {
  long long off;  // element offset of entry (0,0)
  int ld;         // leading dimension (elements)
  int m;          // order
  int e;          // columns to eliminate (partial Cholesky) / rows used
  int dblk;       // first slot of this matrix in the block store of factored kNB x kNB diagonal blocks
  // half-bandwidth of the eliminated block: entries (i, k), i, k < e, with |i - k| > band are
  // structurally zero, so the partial Cholesky leaves them zero (no fill outside the band) and
  // its updates skip the rows and columns past the band (band >= e: dense)
  int band = 1 << 30;
  // first row of an identity block below the eliminated columns (row id0 + i holds a single 1
  // in column i, as in the augmented matrices [[A, I], [I, 0]] whose partial Cholesky leaves
  // -A^-1): row id0 + i of L is zero left of column i, so an update whose K range ends at ke
  // reaches only the rows id0 .. id0 + ke - 1 of that block (id0 >= m: none)
  int id0 = 1 << 30;
  // first column of the eliminated block that each later row [e, m) reaches in L, as a
  // non-decreasing bound (suffix minimum): row e + g of L is zero left of ifirst[g], so an
  // update whose K range ends at ke reaches only the rows e .. e + #{g: ifirst[g] < ke} - 1 of
  // them, and the final update of rows [e + g, ...) needs K from ifirst[g] on (nullptr: dense;
  // a device pointer in the kernels' descriptors, a host pointer in the engine's host copies)
  const int *ifirst = nullptr;
};

// Rows [row0, m) that an update of the partial Cholesky with K range ending at ke reaches:
// the interior rows up to ke + band (the L entries of later interior rows vanish in that K
// range), then the dense rows from max(row0, e) up to the identity block, then the first ke
// rows of the identity block.  Virtual row v in [0, nv) -> matrix row.
struct BandRows {
  int row0, ni, mid0, nmid, idr, nv;
  __host__ __device__ int row(int v) const {
    return v < ni ? row0 + v : (v - ni < nmid ? mid0 + (v - ni) : idr + (v - ni - nmid));
  }
};
__host__ __device__ inline int band_limit(const MatDesc &d, int ke) {
  return d.band >= d.e ? d.e : (ke + d.band < d.e ? ke + d.band : d.e);
}
// rows e .. e + result - 1 of the later block are the ones whose L row reaches a K range
// ending at ke (binary search over the non-decreasing ifirst; m - e when there is no profile)
__host__ __device__ inline int profile_rows(const MatDesc &d, int ke) {
  const int n = d.m - d.e;
  if (!d.ifirst || n <= 0) return n > 0 ? n : 0;
  int lo = 0, hi = n;  // first g with ifirst[g] >= ke
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (d.ifirst[mid] < ke) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__host__ __device__ inline BandRows band_rows(const MatDesc &d, int row0, int ke) {
  BandRows b;
  b.row0 = row0;
  const int lim = band_limit(d, ke);
  b.ni = lim > row0 ? lim - row0 : 0;
  b.mid0 = row0 > d.e ? row0 : d.e;
  const int idb = d.id0 < d.m ? d.id0 : d.m;  // start of the identity block (m: none)
  int midend = idb;
  if (d.ifirst && row0 <= d.e) {  // the later rows whose L row the K range does not reach yet
    const int pend = d.e + profile_rows(d, ke);
    midend = pend < midend ? pend : midend;
  }
  b.nmid = midend > b.mid0 ? midend - b.mid0 : 0;
  b.idr = idb > b.mid0 ? idb : b.mid0;
  const long long idend = (long long)idb + ke;  // rows of the block reached so far
  const int iend = idend < d.m ? (int)idend : d.m;
  const int nid = iend > b.idr ? iend - b.idr : 0;
  b.nv = b.ni + b.nmid + nid;
  return b;
}

// Batched symmetric GEMV task: y = alpha A x for a symmetric n x n matrix stored in full
// (row-major, ld a multiple of 8, 16-byte aligned), plus optional plain rows yb = alpha B x
// (B: nb x n at b_off, same ld).  flags bit0: x gathered through xidx; bit1: accumulate.
struct SymvTask {
  long long a_off, b_off;
  int ld, n, nb, x_off, y_off, yb_off, flags;
};

// Generic batched GEMV task: y[y_idx?] = alpha * op(A) x + beta * y.
struct GemvDesc {
  long long a_off;  // matrix offset
  int ld, rows, cols;
  int x_off;        // offset into x (or into the x gather list)
  int y_off;        // offset into y
  int flags;        // bit0: x gathered via xidx, bit1: accumulate into y
};

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// A sparse product used as a kernel operand: entry i = sum_k val[k] v[col[k]] over
// k in [ptr[i], ptr[i + 1]); ptr == nullptr means "not used".
struct CsrIn {
  const int *ptr, *col;
  const double *val, *v;
};
__device__ __forceinline__ double csr_row(const CsrIn &c, int i) {
  double a = 0.0;
  for (int k = c.ptr[i]; k < c.ptr[i + 1]; ++k) a += c.val[k] * c.v[c.col[k]];
  return a;
}

}  // namespace bd
