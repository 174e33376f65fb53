// Fifth-generation tensor-core primitives (tcgen05, sm_100a / sm_103a) in inline PTX:
// shared-memory matrix descriptors, the instruction descriptor of a bf16 x bf16 -> FP32 MMA,
// tensor-memory (TMEM) allocation, MMA issue and completion through an mbarrier, and loads of
// the FP32 accumulator from TMEM.  Layout conventions (PTX ISA, tcgen05 chapter):
//   * operands are K-major tiles in shared memory in the 64-byte swizzled layout: rows of 64 B
//     (32 bf16 along K), 8-row groups 512 B apart, the 16-byte chunk q of row r stored at chunk
//     q ^ ((r >> 1) & 3) of that row; tiles start on a 512-byte boundary;
//   * the accumulator of an M = 128 MMA (cta_group::1) holds row i in TMEM lane i and column j
//     in TMEM column (base + j); warp w of a warpgroup reads lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once
#include <cuda.h>
#include <stdint.h>

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand tile in the 64-byte swizzled layout:
// start address (bits 0-13, >> 4), leading-dimension offset (bits 16-29, unused for swizzled
// K-major tiles), stride between 8-row groups (bits 32-45, 512 B >> 4), descriptor version 1
// (bits 46-48), swizzle mode 64B = 4 (bits 61-63).  A K offset inside the 64-byte row is added
// to the start address (the hardware applies the swizzle to the generated addresses).
__device__ __forceinline__ uint64_t tc_desc_k_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Instruction descriptor of tcgen05.mma.kind::f16: D FP32 (bits 4-5 = 1), A and B bf16 (bits
// 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A B^T for one K = 16 step, issued by a single thread.
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive (once) on the mbarrier when every tcgen05 operation issued so far by this thread is done.
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tc_smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void tc_mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Non-blocking test of the phase of the given parity.
__device__ __forceinline__ bool tc_mbar_test_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(tc_smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete, giving up after `budget` clock cycles
// (a spin on the non-blocking test, so that a small budget runs out deterministically).
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* mbar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (!tc_mbar_test_wait(mbar, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}

// TMEM allocation (one whole warp); the column base is written to shared memory.
__device__ __forceinline__ void tc_alloc(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(holder)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Eight consecutive FP32 columns of this thread's TMEM lane (32x32b shape), waited on in the
// same statement so that no use of the registers can move ahead of the load.
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Arrive once on the mbarrier and add `bytes` to the transaction count it waits for.
__device__ __forceinline__ void tc_mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem_u32(mbar)), "r"(bytes)
               : "memory");
}

// Bulk tensor copy (TMA) of the box at (x, y) of a 2-D tensor map into shared memory; completion is
// counted in bytes on the mbarrier.  The map is a __grid_constant__ kernel parameter.
__device__ __forceinline__ void tc_tma_load_2d(uint32_t sdst, const CUtensorMap* map, int x, int y, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          sdst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(tc_smem_u32(mbar))
      : "memory");
}
