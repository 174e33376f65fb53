// Sliced FP64 products on the fifth-generation tensor cores: the block-wide main loop shared by
// the Krylov-chain kernel (k_chain_tc.cu) and the adjoint pair-matrix kernel (k_pair_tc.cu).
//
// One CTA of 256 threads owns a 128 x NB output tile.  A (128 rows) and B (NB rows) are given
// as S digit planes of signed 7-bit integers stored as bf16 (ozaki.cuh), K-major.  The loop
//   * stages K slices of 32 of every plane of A and B into a three-deep ring of 64-byte-swizzled
//     shared-memory tiles with cp.async (16-byte chunks; rows past `rows` and K past `K` are
//     zero-filled);
//   * keeps one FP32 accumulator per digit order g in tensor memory, NB columns each, order g
//     at columns [g NB, g NB + NB).  The B planes of a slot are consecutive in shared memory, so
//     planes l0 .. l0 + n - 1 form one taller B operand, and the product of A plane k with it,
//     written at column (k + l0) NB, lands each pair (k, l) in the accumulator of order k + l:
//     one tcgen05.mma (M = 128, N = n NB <= 256, K = 16, bf16 -> FP32) per A plane covers all
//     its digit pairs with k + l <= S - 1;
//   * issues each slot's MMAs from one thread as soon as its copies have landed and commits
//     them to the slot's mbarrier; the slot is refilled once those MMAs are done, while the
//     next slot's MMAs are already queued;
//   * at the end of every K chunk of OZ_KCHUNK (every partial sum of the low digit orders is an
//     integer below 2^24 and therefore exact in FP32) hands the accumulators to `consume`, which
//     reads them with tcgen05.ld and adds them up as integers; the next chunk restarts them.
// Every mbarrier wait is bounded (TCS_WAIT_CYCLES); if one runs out the loop stops, and the
// teardown lets the block's copies and MMAs drain (bounded again), frees tensor memory and sets
// LMBD_FLAG_TIMEOUT.
#pragma once
#include "lmbd_internal.cuh"
#include "ozaki.cuh"
#include "tc05.cuh"

#define TCS_M 128
#define TCS_KS 32                    // K elements per ring slot: one 64-byte swizzled row
#define TCS_NBUF 3                   // ring depth
#define TCS_TMEM_COLS 512            // tensor-memory allocation per CTA
#define TCS_WAIT_CYCLES (1LL << 32)  // about two seconds at 2 GHz

template <int S, int NB>
struct TcsShape {
  static constexpr int kAPlane = TCS_M * TCS_KS * 2;
  static constexpr int kBPlane = NB * TCS_KS * 2;
  static constexpr int kSlot = S * (kAPlane + kBPlane);
  static constexpr int kBytes = TCS_NBUF * kSlot + 1024;  // + slack to align the ring to 1024 B
  static constexpr int kGroupCols = NB;                    // TMEM columns per digit order
  static constexpr int kPlanesPerMma = 256 / NB;           // B planes per MMA (N <= 256)
  static_assert(S * kGroupCols <= TCS_TMEM_COLS, "accumulators exceed the tensor-memory allocation");
  static_assert(NB % 16 == 0 && NB >= 16 && NB <= 256, "N of an M = 128 tcgen05.mma");
  static_assert(kBPlane % 512 == 0, "swizzled tiles start on 512-byte boundaries");
};

// One operand: digit plane k, row r, element j at g[k plane + r ld + j]; rows >= `rows` are zero.
struct TcsOperand {
  const unsigned short* g;
  long long plane;
  long long ld;
  int rows;
};

// Block-wide set-up: tensor memory (warp 0) and the ring's mbarriers.  Returns the TMEM base.
__device__ __forceinline__ uint32_t tcs_setup(uint32_t* holder, uint64_t* mbar) {
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    tc_alloc(holder, TCS_TMEM_COLS);
    tc_relinquish();
  }
  if (threadIdx.x == 32) {
#pragma unroll
    for (int b = 0; b < TCS_NBUF; ++b) tc_mbar_init(&mbar[b], 1);
    tc_mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *holder;
}

// Block-wide tear-down: drain copies (and, after an abort, the last committed MMAs), free TMEM.
__device__ __forceinline__ void tcs_teardown(uint32_t tmem, bool abort, int committed, uint64_t* mbar, int* status) {
  tc_cp_wait_all();
  if (abort) {
    if (threadIdx.x == 0) atomicOr(status, LMBD_FLAG_TIMEOUT);
    if (committed >= 0) tc_mbar_wait(&mbar[committed % TCS_NBUF], (committed / TCS_NBUF) & 1, TCS_WAIT_CYCLES);
  }
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tc_dealloc(tmem, TCS_TMEM_COLS);
  }
}

// TMEM address of lane quarter (warp % 4), column `col`.
__device__ __forceinline__ uint32_t tcs_lane_addr(uint32_t tmem, int col) {
  return tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + (uint32_t)col;
}

// The main loop (all 256 threads).  consume() runs block-wide at the end of every K chunk with
// the accumulators complete in TMEM; returns false if a wait ran out.
template <int S, int NB, class Consume>
__device__ __forceinline__ bool tcs_mainloop(const TcsOperand& A, const TcsOperand& B, int K, uint32_t sbase,
                                             uint32_t tmem, uint64_t* mbar, int& committed, Consume&& consume) {
  using Sh = TcsShape<S, NB>;
  const int tid = threadIdx.x;
  const int nst = (K + TCS_KS - 1) / TCS_KS;
  auto load = [&](int stage, int slot) {
    const int k0 = stage * TCS_KS;
    const uint32_t sA = sbase + slot * Sh::kSlot;
    const uint32_t sB = sA + S * Sh::kAPlane;
    for (int e = tid; e < S * TCS_M * 4 + S * NB * 4; e += blockDim.x) {
      const unsigned short* src = A.g;
      uint32_t dst;
      bool ok;
      if (e < S * TCS_M * 4) {
        const int k = e / (TCS_M * 4), r = (e >> 2) & (TCS_M - 1), q = e & 3;
        ok = r < A.rows && k0 + 8 * q < K;
        if (ok) src = A.g + k * A.plane + r * A.ld + k0 + 8 * q;
        dst = sA + k * Sh::kAPlane + r * 64 + ((q ^ ((r >> 1) & 3)) << 4);
      } else {
        const int e2 = e - S * TCS_M * 4, k = e2 / (NB * 4), r = (e2 >> 2) % NB, q = e2 & 3;
        ok = r < B.rows && k0 + 8 * q < K;
        if (ok) src = B.g + k * B.plane + r * B.ld + k0 + 8 * q;
        dst = sB + k * Sh::kBPlane + r * 64 + ((q ^ ((r >> 1) & 3)) << 4);
      }
      tc_cp_async16(dst, src, ok ? 16 : 0);
    }
    tc_cp_commit();
  };
  load(0, 0);
  if (nst > 1) load(1, 1);
  else tc_cp_commit();
  for (int s = 0; s < nst; ++s) {
    // the copies of stage s have landed (those of stage s + 1 may still be in flight)
    tc_cp_wait<1>();
    tc_fence_proxy_async();
    __syncthreads();
    const bool chunk_first = (s * TCS_KS) % OZ_KCHUNK == 0;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sA = sbase + (s % TCS_NBUF) * Sh::kSlot;
      const uint32_t sB = sA + S * Sh::kAPlane;
#pragma unroll
      for (int kk = 0; kk < TCS_KS / 16; ++kk)
#pragma unroll
        for (int k = 0; k < S; ++k) {
          const uint64_t ad = tc_desc_k_sw64(sA + k * Sh::kAPlane + kk * 32);
#pragma unroll
          for (int l0 = 0; l0 < S - k; l0 += Sh::kPlanesPerMma) {
            const int n = (S - k - l0) < Sh::kPlanesPerMma ? (S - k - l0) : Sh::kPlanesPerMma;
            const uint64_t bd = tc_desc_k_sw64(sB + l0 * Sh::kBPlane + kk * 32);
            // at the start of a chunk the products of A plane 0 (every order) restart the sums
            tc_mma_bf16(tmem + (uint32_t)((k + l0) * Sh::kGroupCols), ad, bd, tc_idesc_bf16(TCS_M, n * NB),
                        (chunk_first && kk == 0 && k == 0) ? 0u : 1u);
          }
        }
      tc_commit(&mbar[s % TCS_NBUF]);
    }
    committed = s;
    // refill the slot that the MMAs of stage s - 1 read, once they are done
    bool to = false;
    if (s + 2 < nst) {
      if (s >= 1) to = !tc_mbar_wait(&mbar[(s - 1) % TCS_NBUF], ((s - 1) / TCS_NBUF) & 1, TCS_WAIT_CYCLES);
      if (!to) load(s + 2, (s + 2) % TCS_NBUF);
      else tc_cp_commit();
    } else {
      tc_cp_commit();
    }
    if (((s + 1) * TCS_KS) % OZ_KCHUNK == 0 || s + 1 == nst) {
      to = to || !tc_mbar_wait(&mbar[s % TCS_NBUF], (s / TCS_NBUF) & 1, TCS_WAIT_CYCLES);
      if (__syncthreads_or(to)) return false;
      tc_fence_after();
      consume();
      tc_fence_before();
      __syncthreads();
    } else if (__syncthreads_or(to)) {
      return false;
    }
  }
  return true;
}
