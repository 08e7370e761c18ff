// Dense bf16 GEMMs of the learned-guess network on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, bf16 operands, FP32 accumulation in tensor memory).
//
// C (M x N) = A (M x K) B (N x K)^T with A and B K-major (row-major, leading
// dimensions multiples of 8, K padded with zeros to a multiple of 64).  One CTA of 128
// threads per 128 x 128 output tile.  Per K chunk of 64 bf16 (one 128-byte swizzle
// row per tile row) the 128 threads load both tiles with cp.async straight into the
// 128-byte-swizzled K-major layout the MMA reads (four stages, two chunks in flight
// ahead of the MMAs); one thread issues four MMAs (K = 16 each) per chunk and commits
// them to the stage's mbarrier, which the loads wait on (bounded) before reusing it.
// The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w ..
// 32w + 31 = tile rows) and applies the layer's operation:
//   forward:  z = acc + bias; Z = z; Hb = bf16(relu(z)) and its transpose HbT
//   backward: d = acc * (Zprev > 0); Z = d; Hb = bf16(d) and its transpose HbT
//   weights:  Z = acc
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp.cuh"

namespace bd {

namespace {

constexpr int kGM = 128, kGN = 128;     // output tile (MMA M and N)
constexpr int kGK = 64;                 // bf16 K elements per chunk = 128 bytes
constexpr int kGStages = 4;
constexpr int kGTile = kGM * kGK * 2;   // 16 KB per operand tile
constexpr uint32_t kGTmemCols = 128;
constexpr long long kGWaitLimit = 1LL << 22;

__device__ inline uint32_t g_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ inline uint64_t g_sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: D f32, A and B bf16, both K-major, M = kGM, N = kGN.
__device__ inline uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGN >> 3) << 17) | ((uint32_t)(kGM >> 4) << 24);
}

__device__ inline void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ inline bool g_mbar_wait(uint32_t bar, uint32_t phase) {
  for (long long it = 0; it < kGWaitLimit; ++it) {
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

__device__ inline void g_cp_async16(uint32_t dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes));
}

}  // namespace

__global__ void __launch_bounds__(128, 1) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A,
                                                      int lda, const __nv_bfloat16 *__restrict__ B, int ldb,
                                                      GemmEpi ep, int *__restrict__ err) {
  const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t mbar[kGStages];
  __shared__ uint32_t tmem_slot;
  const uint32_t raw0 = g_smem_addr(smem_raw);
  const uint32_t tiles = (raw0 + 1023u) & ~1023u;
  unsigned char *tp = smem_raw + (tiles - raw0);
  auto st_off = [](int s, int op) { return (uint32_t)((s * 2 + op) * kGTile); };
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(g_smem_addr(&tmem_slot)),
                 "r"(kGTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kGStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(g_smem_addr(&mbar[s])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16();
  const int seg = tid & 7, rr = tid >> 3;  // 16-byte segment of a 128-byte row, first row

  // chunk c (K elements [64c, 64c + 64)) into stage s; rows outside M / N read nothing (zero fill)
  auto load = [&](int c, int s) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = rr + 16 * i;
      const uint32_t off = (uint32_t)r * 128u + (uint32_t)((seg ^ (r & 7)) * 16);
      const long long k = (long long)c * kGK + seg * 8;
      const bool va = m0 + r < M, vb = n0 + r < N;
      const __nv_bfloat16 *sa = va ? A + (long long)(m0 + r) * lda + k : A;
      const __nv_bfloat16 *sb = vb ? B + (long long)(n0 + r) * ldb + k : B;
      g_cp_async16(tiles + st_off(s, 0) + off, sa, va ? 16u : 0u);
      g_cp_async16(tiles + st_off(s, 1) + off, sb, vb ? 16u : 0u);
    }
    asm volatile("cp.async.commit_group;");
  };

  const int nchunk = K / kGK;
  uint32_t phase[kGStages] = {0u, 0u, 0u, 0u};
  int pending[kGStages] = {0, 0, 0, 0};
  bool ok = true;
  load(0, 0);
  if (nchunk > 1) load(1, 1);
  for (int i = 0; i < nchunk; ++i) {
    const int s = i % kGStages;
    if (i + 2 < nchunk) {
      // stage (i + 2) % 4 was last read by the MMAs of chunk i - 2
      const int s2 = (i + 2) % kGStages;
      bool late = false;
      if (pending[s2]) {
        late = !g_mbar_wait(g_smem_addr(&mbar[s2]), phase[s2]);
        if (!late) {
          phase[s2] ^= 1u;
          pending[s2] = 0;
        }
      }
      if (__syncthreads_or(late ? 1 : 0)) {
        ok = false;
        break;
      }
      load(i + 2, s2);
      asm volatile("cp.async.wait_group 2;");
    } else if (i + 1 < nchunk) {
      asm volatile("cp.async.wait_group 1;");
    } else {
      asm volatile("cp.async.wait_group 0;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a = tiles + st_off(s, 0), b = tiles + st_off(s, 1);
#pragma unroll
      for (int t = 0; t < kGK / 16; ++t)  // K = 16 bf16 = 32 bytes per MMA
        mma_bf16(tmem, g_sw128_desc(a + 32u * t), g_sw128_desc(b + 32u * t), idesc, (i == 0 && t == 0) ? 0u : 1u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          g_smem_addr(&mbar[s])));
    }
    pending[s] = 1;
  }
  asm volatile("cp.async.wait_group 0;");
  // drain every MMA batch still in flight (also one a bounded wait above gave up on) before
  // the epilogue reads TMEM or the CTA releases its shared and tensor memory; a batch that
  // misses this wait too is reported and the epilogue skipped
  bool late = false;
  for (int s = 0; s < kGStages; ++s)
    if (pending[s]) {
      late |= !g_mbar_wait(g_smem_addr(&mbar[s]), phase[s]);
      phase[s] ^= 1u;
    }
  if (__syncthreads_or(late ? 1 : 0) || !ok) {
    ok = false;
    if (tid == 0) atomicOr(err, DEV_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    __syncthreads();
    float *stage = reinterpret_cast<float *>(tp) + warp * 32 * 33;
    const int lane = tid & 31;
    for (int cc = 0; cc < kGN; cc += 32) {
      if (n0 + cc >= N) break;
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
      // this thread holds row m = m0 + 32 warp + lane, columns n0 + cc + q
      const int m = m0 + warp * 32 + lane;
#pragma unroll
      for (int q = 0; q < 32; ++q) stage[lane * 33 + q] = __uint_as_float(v[q]);
      __syncwarp();
      // now lane = column: rows m0 + 32 warp + u, column n = n0 + cc + lane (coalesced rows)
      const int n = n0 + cc + lane;
      const bool vn = n < N;
      float bias = 0.f;
      if (ep.mode == 0 && ep.bias && vn) bias = ep.bias[n];
#pragma unroll 4
      for (int u = 0; u < 32; ++u) {
        const int mm = m0 + warp * 32 + u;
        if (!vn || mm >= M) continue;
        float x = stage[u * 33 + lane];
        if (ep.mode == 0) x += bias;
        if (ep.mode == 1) x = (ep.Zprev[(long long)mm * ep.ldzp + n] > 0.f) ? x : 0.f;
        if (ep.Z) ep.Z[(long long)mm * ep.ldz + n] = x;
        if (ep.mode != 2) {
          const float h = (ep.mode == 0 && ep.relu) ? fmaxf(x, 0.f) : x;
          if (ep.Hb) ep.Hb[(long long)mm * ep.ldh + n] = __float2bfloat16(h);
          stage[u * 33 + lane] = h;  // for the transposed copy below
        }
      }
      __syncwarp();
      if (ep.mode != 2 && ep.HbT && m < M) {
        // transposed copy: row n of HbT, column m (lane = row m: coalesced over the warp)
#pragma unroll 4
        for (int q = 0; q < 32; ++q) {
          const int nn = n0 + cc + q;
          if (nn < N) ep.HbT[(long long)nn * ep.ldht + m] = __float2bfloat16(stage[lane * 33 + q]);
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGTmemCols));
  }
}

static constexpr int kGemmSmem = 2 * kGStages * kGTile + 1024;

bool gemm_tc_configure() {
  return cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem) == cudaSuccess;
}

void launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                      const GemmEpi &ep, int *err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  k_gemm_bf16<<<dim3(ceil_div(M, kGM), ceil_div(N, kGN)), 128, kGemmSmem, s>>>(M, N, K, A, lda, B, ldb, ep, err);
  count_launch();
}

}  // namespace bd
