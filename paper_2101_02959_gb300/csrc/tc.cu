// Rank-k Schur updates on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// C[r][c] -= sum_k A[r][k] A[c][k] over one 128 x 128 lower tile per CTA, for
// the long-K updates of the partial Cholesky (outer panels and the final Schur
// complement S = K_GG - L_GI L_GI^T, Section 4.1).  FP32 operands are split as
// a = a_hi + a_lo with a_hi, a_lo TF32, and a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// (three MMAs per K step, FP32 accumulation in tensor memory), which keeps the
// Schur complement at FP32 accuracy.
//
// Per K chunk of 32: 128 threads load the two 128 x 32 tiles (cp.async, two
// chunks ahead), split them and store hi / lo copies in shared memory in the
// K-major layout with the 128-byte swizzle; one thread issues the MMAs and
// commits them to an mbarrier; the CTA waits on it (bounded) before reusing the
// buffers.  The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
// lanes 32w .. 32w+31 = tile rows), stages it in shared memory and subtracts it
// from C row by row (coalesced).
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace bd {

namespace {

constexpr int kTM = 128;          // tile rows (MMA M) and columns (MMA N)
constexpr int kKc = 32;           // fp32 K elements per chunk = one 128-byte swizzle row
constexpr int kTileBytes = kTM * kKc * 4;  // 16 KB per operand copy
constexpr int kRawStages = 3;              // FP32 load stages (prefetch distance 2 chunks)
constexpr uint32_t kTmemCols = 128;
constexpr long long kWaitLimit = 1LL << 22;

__device__ inline uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ inline uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)(16 >> 4) << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                         // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

// Instruction descriptor: D f32, A and B tf32, both K-major, M = N = 128.
__device__ inline uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTM >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ inline float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ inline void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// Bounded wait on an mbarrier phase; false on timeout.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase));
    if (ok) return true;
  }
  return false;
}

}  // namespace

__device__ inline void cp_async16(uint32_t dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes));
}

// mode 1: rows/cols [e, m), K = [0, e); mode 2: rows [K1, m), cols [K1, e), K = [K0, K1).
// Pipeline per K chunk i (raw stage i % 3, operand buffer b = i % 2):
//   raw (FP32 A and B tiles, cp.async, swizzled) -> split into hi/lo[b] -> 12 MMAs on hi/lo[b]
// with the loads of chunks i+1 and i+2 in flight during the split of chunk i and the
// MMAs of chunk i running while chunk i+1 is split (mbar[b] guards hi/lo[b] against reuse).
__global__ void __launch_bounds__(128, 1) k_rankk_tc(const MatDesc *__restrict__ desc, float *__restrict__ base,
                                                     int mode, int K0, int K1, int nct, int *__restrict__ err) {
  const MatDesc d = desc[blockIdx.y];
  int row0, colend, kb, ke;
  if (mode == 2) {
    if (K1 >= d.e) return;
    row0 = K1; colend = d.e; kb = K0; ke = K1;
  } else {
    row0 = d.e; colend = d.m; kb = 0; ke = d.e;
  }
  const int ti = blockIdx.x / nct, tj = blockIdx.x % nct;
  if (tj > ti) return;
  const int r0 = row0 + ti * kTM, c0 = row0 + tj * kTM;
  if (r0 >= d.m || c0 >= colend || ke <= kb) return;
  float *A = base + d.off;

  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const uint32_t raw0 = smem_addr(smem_raw);
  const uint32_t tiles = (raw0 + 1023u) & ~1023u;
  unsigned char *tp = smem_raw + (tiles - raw0);
  // layout: raw A/B per stage (kRawStages x 2 x 16 KB), then hi/lo A/B per buffer (2 x 4 x 16 KB)
  auto raw_off = [](int b, int op) { return (uint32_t)((b * 2 + op) * kTileBytes); };
  auto op_off = [](int b, int q) { return (uint32_t)(2 * kRawStages * kTileBytes + (b * 4 + q) * kTileBytes); };
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32();
  const int j = tid & 7, rr = tid >> 3;

  // asynchronous load of chunk starting at kk into raw buffer b (zero fill outside the matrix / K range)
  auto load = [&](int kk, int b) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = rr + 16 * i;
      const int k = kk + 4 * j;
      const uint32_t off = (uint32_t)r * 128u + (uint32_t)((j ^ (r & 7)) * 16);
      const int kv = max(0, min(4, ke - k));
      const int ra = r0 + r, rb = c0 + r;
      const uint32_t na = (ra < d.m) ? 4u * kv : 0u, nb = (rb < colend) ? 4u * kv : 0u;
      const float *sa = na ? A + (long long)ra * d.ld + k : A;
      const float *sb = nb ? A + (long long)rb * d.ld + k : A;
      cp_async16(tiles + raw_off(b, 0) + off, sa, na);
      cp_async16(tiles + raw_off(b, 1) + off, sb, nb);
    }
    asm volatile("cp.async.commit_group;");
  };

  const int nchunk = (ke - kb + kKc - 1) / kKc;
  uint32_t phase[2] = {0u, 0u};
  int pending[2] = {0, 0};  // an MMA batch is in flight on hi/lo[b]
  bool ok = true;
  // raw stages: chunk i lands in stage i % kRawStages, loaded kRawStages - 1 chunks ahead
  load(kb, 0);
  if (nchunk > 1) load(kb + kKc, 1);
  for (int i = 0; i < nchunk && ok; ++i) {
    const int b = i & 1, rs = i % kRawStages;
    // stage (i + 2) % 3 was last read by the split of chunk i - 1 (before its barrier)
    if (i + 2 < nchunk) {
      load(kb + (i + 2) * kKc, (i + 2) % kRawStages);
      asm volatile("cp.async.wait_group 2;");
    } else if (i + 1 < nchunk) {
      asm volatile("cp.async.wait_group 1;");
    } else {
      asm volatile("cp.async.wait_group 0;");
    }
    // hi/lo[b] was last read by the MMAs of chunk i - 2; a batch that has not completed
    // within the wait budget stays pending, and the drain below waits for it once more
    bool late = false;
    if (pending[b]) {
      late = !mbar_wait(smem_addr(&mbar[b]), phase[b]);
      if (!late) {
        phase[b] ^= 1u;
        pending[b] = 0;
      }
    }
    if (__syncthreads_or(late ? 1 : 0)) {
      ok = false;
      break;
    }
    // split raw[b] into TF32 hi and lo parts (same swizzled offsets)
#pragma unroll
    for (int i2 = 0; i2 < 8; ++i2) {
      const int r = rr + 16 * i2;
      const uint32_t off = (uint32_t)r * 128u + (uint32_t)((j ^ (r & 7)) * 16);
#pragma unroll
      for (int op = 0; op < 2; ++op) {
        const float4 x = *reinterpret_cast<const float4 *>(tp + raw_off(rs, op) + off);
        const float4 hi = make_float4(tf32_round(x.x), tf32_round(x.y), tf32_round(x.z), tf32_round(x.w));
        const float4 lo = make_float4(tf32_round(x.x - hi.x), tf32_round(x.y - hi.y), tf32_round(x.z - hi.z),
                                      tf32_round(x.w - hi.w));
        *reinterpret_cast<float4 *>(tp + op_off(b, 2 * op) + off) = hi;
        *reinterpret_cast<float4 *>(tp + op_off(b, 2 * op + 1) + off) = lo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = tiles + op_off(b, 0), al = tiles + op_off(b, 1);
      const uint32_t bh = tiles + op_off(b, 2), bl = tiles + op_off(b, 3);
#pragma unroll
      for (int t = 0; t < kKc / 8; ++t) {  // K = 8 tf32 = 32 bytes per MMA
        const uint32_t adv = (uint32_t)t * 32u;
        const uint32_t first = (i == 0 && t == 0) ? 0u : 1u;
        mma_tf32(tmem, sw128_desc(ah + adv), sw128_desc(bh + adv), idesc, first);
        mma_tf32(tmem, sw128_desc(ah + adv), sw128_desc(bl + adv), idesc, 1u);
        mma_tf32(tmem, sw128_desc(al + adv), sw128_desc(bh + adv), idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&mbar[b])));
    }
    pending[b] = 1;
  }
  asm volatile("cp.async.wait_group 0;");
  // drain: wait for every MMA batch still in flight (also one that timed out above), so
  // that no MMA still reads this CTA's shared memory or writes its tensor memory when the
  // CTA releases them.  A batch that misses this bounded wait too is reported
  // (DEV_ERR_TIMEOUT, skipped epilogue); the caller must then treat the whole handle as
  // lost (bidomain_destroy), since the tensor pipe may still be running on it.
  bool late = false;
  for (int b = 0; b < 2; ++b)
    if (pending[b]) {
      late |= !mbar_wait(smem_addr(&mbar[b]), phase[b]);
      phase[b] ^= 1u;
    }
  if (__syncthreads_or(late ? 1 : 0) || !ok) {
    ok = false;
    if (tid == 0) atomicOr(err, DEV_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // epilogue: warp w reads TMEM lanes 32w + lane (tile rows), 32 columns per load,
    // stages them in shared memory (the operand buffers are free now) and updates C
    // one row per instruction (coalesced 128-byte rows)
    __syncthreads();
    float *stage = reinterpret_cast<float *>(tp) + warp * 32 * 33;
    const int lane = tid & 31;
    for (int cc = 0; cc < kTM; cc += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
            "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int q = 0; q < 32; ++q) stage[lane * 33 + q] = __uint_as_float(v[q]);
      __syncwarp();
      const int c = c0 + cc + lane;
      const bool vc = c < colend;
      {  // all 32 rows' loads in flight, then their stores
        float cv[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int r = r0 + warp * 32 + u;
          cv[u] = (vc && r < d.m) ? A[(long long)r * d.ld + c] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int r = r0 + warp * 32 + u;
          if (vc && r < d.m) A[(long long)r * d.ld + c] = cv[u] - stage[u * 33 + lane];
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

static constexpr int kTcSmem = (2 * kRawStages + 8) * kTileBytes + 1024;  // raw stages + 2 x hi/lo A/B + alignment

bool tc_configure() {
  return cudaFuncSetAttribute(k_rankk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) == cudaSuccess;
}

void launch_rankk_tc(const MatDesc *d_desc, float *base, int mode, int K0, int K1, int max_rows, int max_cols,
                     int count, int *err, cudaStream_t s) {
  const int nrt = ceil_div(max_rows, kTM), nct = ceil_div(max_cols, kTM);
  if (nrt == 0 || nct == 0) return;
  k_rankk_tc<<<dim3(nrt * nct, count), 128, kTcSmem, s>>>(d_desc, base, mode, K0, K1, nct, err);
  count_launch();
}

}  // namespace bd
