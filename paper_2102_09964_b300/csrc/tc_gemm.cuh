// tc_gemm.cuh -- BF16 GEMM with FP32 accumulation on the 5th-generation
// tensor cores of sm_103a: C[M x N] = A[M x K] B[N x K]^T, both operands
// K-contiguous (row-major with K innermost), an epilogue functor per element.
//
// One CTA of 128 threads computes a 128 x 64 tile of C:
//   - TMA (cp.async.bulk.tensor.2d) loads 64-wide K slices of A (128 rows) and
//     B (64 rows) into shared memory in the 128-byte swizzled layout, STAGES
//     slices in flight, each completing an mbarrier (expect-tx bytes);
//     rows or columns outside the matrices are zero-filled by the TMA unit;
//   - one thread issues tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 64,
//     K = 16: four per slice) with the FP32 accumulator in tensor memory, and
//     tcgen05.commit returns each slice's buffer to the loads once the
//     multiplies that read it are done;
//   - after the last slice the four warps read the accumulator back with
//     tcgen05.ld (warp w: TMEM lanes = tile rows 32w .. 32w+31) and apply the
//     epilogue to every element inside C.
// Every wait on an mbarrier gives up after about a second of clock cycles and
// sets *err; the tensor-memory columns are freed on every path.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace pssgp {
namespace tc {

constexpr int BM = 128;          // tile rows (UMMA M)
constexpr int BN = 64;           // tile columns (UMMA N)
constexpr int BK = 64;           // K slice: 64 bf16 = one 128-byte swizzle row
constexpr int UK = 16;           // K of one tcgen05.mma (kind::f16)
constexpr int STAGES = 3;
constexpr int A_BYTES = BM * BK * 2;          // 16 KB
constexpr int B_BYTES = BN * BK * 2;          // 8 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 64;                 // FP32 accumulator: 128 lanes x 64 columns
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;   // + alignment slack (tiles on 1024 B)
constexpr long long WAIT_CYCLES = 2000000000LL;           // about 1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarriers ------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed; false after
// WAIT_CYCLES without it
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

// ---- TMA ------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// ---- tensor memory and the MMA ---------------------------------------------
// shared-memory matrix descriptor: K-major operand in the 128-byte swizzled
// layout written by the TMA (rows of 128 bytes, 8-row atoms of 1024 bytes):
// start address >> 4 (bits 0-13), leading offset 1 (unused for this layout,
// bits 16-29), stride offset 1024 >> 4 between 8-row atoms (bits 32-45),
// descriptor version 1 (bits 46-47), swizzle mode 2 = 128 B (bits 61-63)
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3
// (bits 17-22), M >> 4 (bits 24-28)
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(taddr), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the mbarrier once every tcgen05.mma issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <class Epi>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(const __grid_constant__ CUtensorMap mapA,
                                                   const __grid_constant__ CUtensorMap mapB, int M, int N, int K,
                                                   Epi epi, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ int issue_ok;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;   // tiles on 1024-byte boundaries
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int KT = (K + BK - 1) / BK;
  constexpr uint32_t IDESC = idesc_bf16_f32(BM, BN);
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    issue_ok = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tmem_base;
  if (tid == 0) {
    bool ok = true;
    const int pro = KT < STAGES ? KT : STAGES;
    for (int kt = 0; kt < pro; ++kt) {
      const uint32_t a = base + kt * STAGE_BYTES;
      mbar_expect_tx(smem_u32(&full[kt]), STAGE_BYTES);
      tma_load_2d(a, &mapA, kt * BK, m0, smem_u32(&full[kt]));
      tma_load_2d(a + A_BYTES, &mapB, kt * BK, n0, smem_u32(&full[kt]));
    }
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait(smem_u32(&full[s]), ph)) { ok = false; break; }
      tc_fence_after();
      const uint32_t a = base + s * STAGE_BYTES, b = a + A_BYTES;
      // K steps of 16 that hold data (the TMA zero-fills past K)
      const int rem = K - kt * BK;
      const int nkk = rem >= BK ? BK / UK : (rem + UK - 1) / UK;
      for (int kk = 0; kk < nkk; ++kk)
        mma_bf16(taddr, smem_desc_sw128(a + kk * UK * 2), smem_desc_sw128(b + kk * UK * 2), IDESC,
                 (kt | kk) != 0 ? 1u : 0u);
      mma_commit(smem_u32(&empty[s]));
      const int nk = kt + STAGES;
      if (nk < KT) {
        // the buffer is free once the multiplies that read it are done
        if (!mbar_wait(smem_u32(&empty[s]), ph)) { ok = false; break; }
        mbar_expect_tx(smem_u32(&full[s]), STAGE_BYTES);
        tma_load_2d(a, &mapA, nk * BK, m0, smem_u32(&full[s]));
        tma_load_2d(b, &mapB, nk * BK, n0, smem_u32(&full[s]));
      }
    }
    // arrives once every multiply issued above is done (also after a timeout,
    // so that the accumulator is not freed under running multiplies)
    mma_commit(smem_u32(&done));
    if (!ok) issue_ok = 0;
  }
  const bool fin = mbar_wait(smem_u32(&done), 0);
  __syncthreads();
  tc_fence_after();
  const bool good = fin && issue_ok;
  if (good) {
    const int row = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
      if (row < M) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (n0 + c + i < N) epi(row, n0 + c + i, v[i]);
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, TMEM_COLS);
}

}  // namespace tc
}  // namespace pssgp
