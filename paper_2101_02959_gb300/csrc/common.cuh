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
