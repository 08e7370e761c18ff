// Rank-k Schur updates on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// C[r][c] -= sum_k A[r][k] A[c][k] over one 128 x 128 lower tile per CTA, for
// the long-K updates of the partial Cholesky (outer panels and the final Schur
// complement S = K_GG - L_GI L_GI^T, Section 4.1).  FP32 operands are split as
// a = a_hi + a_lo with a_hi, a_lo TF32, and a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// (three MMAs per K step, FP32 accumulation in tensor memory), which keeps the
// Schur complement at FP32 accuracy.
//
// Per K chunk of 32: the 128 threads hold the two 128 x 32 FP32 tiles in registers
// (loaded while the previous chunk's MMAs ran), split them and store hi / lo copies
// in shared memory in the K-major layout with the 128-byte swizzle; one thread issues
// the MMAs and commits them to an mbarrier, which the CTA waits on (bounded) before
// the next split reuses the buffer.  Three CTAs share an SM.  The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
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

// mode 3: the panel solve L_21 = A_21 Linv^T below the factored diagonal block [K0, K0 + w)
// (w = min(128, e - K0)): rows as the band lets them reach, output columns K0 .. K0 + w - 1,
// the B operand from pinv (128 x 128 per matrix, the inverse of L_11), result stored;
// mode 0: the update of an outer block by its finished 128-column panel [K0, K0 + 128):
// rows [K0 + 128, m), cols [K0 + 128, min(K1, e)), K = [K0, min(K0 + 128, e));
// mode 1: rows/cols [e, m), K = [0, e); mode 2: rows [K1, m), cols [K1, e), K = [K0, K1).
// Per K chunk i of 32 FP32 columns: every thread holds its share of chunk i in registers
// (loaded while the MMAs of chunk i - 1 ran), waits (bounded) for those MMAs to release the
// single hi/lo operand buffer, splits its values into TF32 hi and lo parts there (128-byte
// swizzled K-major layout), and thread 0 issues the 12 MMAs of the chunk; then the loads of
// chunk i + 1 go out while they run.  65 KB of shared memory per CTA let three CTAs share an
// SM, so one CTA's split, epilogue or pipeline fill overlaps the others' MMAs.
__global__ void __launch_bounds__(128, 3) k_rankk_tc(const MatDesc *__restrict__ desc, float *__restrict__ base,
                                                     int mode, int K0, int K1, int nct, int *__restrict__ err,
                                                     const float *__restrict__ pinv) {
  const MatDesc d = desc[blockIdx.y];
  int row0, colend, kb, ke;
  if (mode == 3) {
    if (K0 >= d.e) return;
    const int w = min(kTM, d.e - K0);
    row0 = K0 + w; colend = w; kb = K0; ke = K0 + w;  // colend, c0: columns of the panel (relative)
  } else if (mode == 0) {
    if (K0 + kTM >= d.e) return;
    row0 = K0 + kTM; colend = min(K1, d.e); kb = K0; ke = K0 + kTM;
  } else if (mode == 2) {
    if (K1 >= d.e) return;
    row0 = K1; colend = d.e; kb = K0; ke = K1;
  } else {
    row0 = d.e; colend = d.m; kb = 0; ke = d.e;
  }
  const BandRows br = band_rows(d, row0, ke);  // rows past the band hold zeros in K = [kb, ke)
  if (mode == 0 || mode == 2) colend = min(colend, band_limit(d, ke));
  const int ti = blockIdx.x / nct, tj = blockIdx.x % nct;
  if (tj > ti) return;
  const int v0 = ti * kTM, c0 = (mode == 3 ? 0 : row0) + tj * kTM;
  if (mode == 1 && d.ifirst && v0 < br.nv) kb = max(kb, d.ifirst[v0] & ~3);  // rows' L starts there
  const float *B = mode == 3 ? pinv + (long long)blockIdx.y * kTM * kTM : nullptr;  // rows c, K from kb
  if (v0 >= br.nv || c0 >= colend || ke <= kb) return;
  const float *A = base + d.off;

  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const uint32_t raw0 = smem_addr(smem_raw);
  const uint32_t tiles = (raw0 + 1023u) & ~1023u;
  unsigned char *tp = smem_raw + (tiles - raw0);
  auto op_off = [](int q) { return (uint32_t)(q * kTileBytes); };  // q: A hi, A lo, B hi, B lo
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32();
  const int j = tid & 7, rr = tid >> 3;

  // this thread's share of a chunk: rows rr + 16 i (i < 8) of the A and B tiles, columns
  // kk + 4 j .. + 3; zero outside the matrix and past the K range
  float4 ra[8], rb[8];
  auto load = [&](int kk) {
    const int k = kk + 4 * j;
    const int kv = max(0, min(4, ke - k));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = rr + 16 * i;
      const bool va = v0 + r < br.nv, vb = c0 + r < colend;
      const float *pa = A + (long long)(va ? br.row(v0 + r) : 0) * d.ld + k;
      const float *pb = B ? B + (long long)(c0 + r) * kTM + (k - kb) : A + (long long)(c0 + r) * d.ld + k;
      if (kv == 4) {
        ra[i] = va ? __ldg(reinterpret_cast<const float4 *>(pa)) : make_float4(0.f, 0.f, 0.f, 0.f);
        rb[i] = vb ? __ldg(reinterpret_cast<const float4 *>(pb)) : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        float ta[4] = {0.f, 0.f, 0.f, 0.f}, tb[4] = {0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < kv; ++q) {
          if (va) ta[q] = pa[q];
          if (vb) tb[q] = pb[q];
        }
        ra[i] = make_float4(ta[0], ta[1], ta[2], ta[3]);
        rb[i] = make_float4(tb[0], tb[1], tb[2], tb[3]);
      }
    }
  };
  auto split_store = [&](const float4 &x, uint32_t hi_off, uint32_t lo_off, uint32_t off) {
    const float4 hi = make_float4(tf32_round(x.x), tf32_round(x.y), tf32_round(x.z), tf32_round(x.w));
    const float4 lo = make_float4(tf32_round(x.x - hi.x), tf32_round(x.y - hi.y), tf32_round(x.z - hi.z),
                                  tf32_round(x.w - hi.w));
    *reinterpret_cast<float4 *>(tp + hi_off + off) = hi;
    *reinterpret_cast<float4 *>(tp + lo_off + off) = lo;
  };

  const int nchunk = (ke - kb + kKc - 1) / kKc;
  uint32_t phase = 0u;
  bool pending = false, ok = true;
  load(kb);
  for (int i = 0; i < nchunk; ++i) {
    // the MMAs of chunk i - 1 read the operand buffer: wait for them (bounded); a batch that
    // has not completed stays pending for the drain below
    bool late = false;
    if (pending) {
      late = !mbar_wait(smem_addr(&mbar), phase);
      if (!late) {
        phase ^= 1u;
        pending = false;
      }
    }
    if (__syncthreads_or(late ? 1 : 0)) {
      ok = false;
      break;
    }
#pragma unroll
    for (int i2 = 0; i2 < 8; ++i2) {
      const int r = rr + 16 * i2;
      const uint32_t off = (uint32_t)r * 128u + (uint32_t)((j ^ (r & 7)) * 16);
      split_store(ra[i2], op_off(0), op_off(1), off);
      split_store(rb[i2], op_off(2), op_off(3), off);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = tiles + op_off(0), al = tiles + op_off(1);
      const uint32_t bh = tiles + op_off(2), bl = tiles + op_off(3);
#pragma unroll
      for (int t = 0; t < kKc / 8; ++t) {  // K = 8 tf32 = 32 bytes per MMA
        const uint32_t adv = (uint32_t)t * 32u;
        const uint32_t first = (i == 0 && t == 0) ? 0u : 1u;
        mma_tf32(tmem, sw128_desc(ah + adv), sw128_desc(bh + adv), idesc, first);
        mma_tf32(tmem, sw128_desc(ah + adv), sw128_desc(bl + adv), idesc, 1u);
        mma_tf32(tmem, sw128_desc(al + adv), sw128_desc(bh + adv), idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&mbar)));
    }
    pending = true;
    if (i + 1 < nchunk) load(kb + (i + 1) * kKc);  // in flight while the MMAs of chunk i run
  }
  // drain: wait for the MMA batch still in flight (also one a bounded wait above gave up on),
  // so that no MMA still reads this CTA's shared memory or writes its tensor memory when the
  // CTA releases them.  A batch that misses this bounded wait too is reported
  // (DEV_ERR_TIMEOUT, skipped epilogue); the caller must then treat the whole handle as lost
  // (bidomain_destroy), since the tensor pipe may still be running on it.
  bool late = false;
  if (pending) {
    late = !mbar_wait(smem_addr(&mbar), phase);
    phase ^= 1u;
  }
  if (__syncthreads_or(late ? 1 : 0) || !ok) {
    ok = false;
    if (tid == 0) atomicOr(err, DEV_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // epilogue: warp w reads TMEM lanes 32w + lane (tile rows), 32 columns per load,
    // stages them in shared memory (the operand buffer is free now) and updates C
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
      if (mode == 3) {  // the panel solve stores its product
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int v = v0 + warp * 32 + u;
          if (vc && v < br.nv) base[d.off + (long long)br.row(v) * d.ld + K0 + c] = stage[u * 33 + lane];
        }
      } else {  // all 32 rows' loads in flight, then their stores
        float cv[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int v = v0 + warp * 32 + u;
          cv[u] = (vc && v < br.nv) ? A[(long long)br.row(v) * d.ld + c] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int v = v0 + warp * 32 + u;
          if (vc && v < br.nv) base[d.off + (long long)br.row(v) * d.ld + c] = cv[u] - stage[u * 33 + lane];
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

static constexpr int kTcSmem = 4 * kTileBytes + 1024;  // hi/lo A/B + alignment

bool tc_configure() {
  return cudaFuncSetAttribute(k_rankk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) == cudaSuccess;
}

void launch_rankk_tc(const MatDesc *d_desc, float *base, int mode, int K0, int K1, int max_rows, int max_cols,
                     int count, int *err, cudaStream_t s, const float *pinv) {
  const int nrt = ceil_div(max_rows, kTM), nct = ceil_div(max_cols, kTM);
  if (nrt == 0 || nct == 0) return;
  k_rankk_tc<<<dim3(nrt * nct, count), 128, kTcSmem, s>>>(d_desc, base, mode, K0, K1, nct, err, pinv);
  count_launch();
}

}  // namespace bd
