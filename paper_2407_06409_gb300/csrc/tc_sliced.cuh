// Sliced FP64 products on the fifth-generation tensor cores: the block-wide main loop shared by
// the Krylov-chain kernel (k_chain_tc.cu) and the adjoint pair-matrix kernel (k_pair_tc.cu).
//
// One CTA of 256 threads owns a 128 x NB output tile.  A (128 rows) and B (NB rows) are S digit
// planes of signed 7-bit integers stored as bf16 (ozaki.cuh), K-major, addressed through 2-D
// tensor maps (inner dimension K, one row per matrix row, 64-byte swizzle).  The loop
//   * stages K slices of 32 of every plane of A and B into a three-deep ring of 64-byte-swizzled
//     shared-memory tiles with bulk tensor copies (TMA, cp.async.bulk.tensor) issued by one
//     thread; each slot has a "full" mbarrier counting the bytes in flight (K past the tensor's
//     extent is zero-filled by the copy engine);
//   * keeps one FP32 accumulator per digit order g in tensor memory, NB columns each, order g
//     at columns [g NB, g NB + NB).  The B planes of a slot are consecutive in shared memory, so
//     planes l0 .. l0 + n - 1 form one taller B operand, and the product of A plane k with it,
//     written at column (k + l0) NB, lands each pair (k, l) in the accumulator of order k + l:
//     one tcgen05.mma (M = 128, N = n NB <= 256, K = 16, bf16 -> FP32) per A plane covers all
//     its digit pairs with k + l <= S - 1;
//   * the same thread issues each slot's MMAs once its copies have landed, commits them to the
//     slot's "empty" mbarrier, and refills the slot of the previous stage (whose MMAs are done by
//     then) with the stage three ahead, so copies and MMAs overlap;
//   * at the end of every K chunk of OZ_KCHUNK (every partial sum of the low digit orders is an
//     integer below 2^24 and therefore exact in FP32) the thread commits an "accumulators"
//     mbarrier and waits for it, a block barrier publishes the result, and all 256 threads hand
//     the accumulators to `consume`, which reads them with tcgen05.ld and adds them up as
//     integers; the next chunk restarts them.
// Rows of a box past a plane's end read the next plane or centre: they only reach output rows
// (A) or columns (B) that the callers discard.  Every mbarrier wait of the loop is bounded (a
// cycle budget, 2^32 by default); if one runs out the loop stops, and the teardown waits for the
// block's copies and MMAs in flight (bounded by TCS_WAIT_CYCLES), frees tensor memory and sets
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

// Host: 2-D tensor map over bf16 digit planes (`inner` elements per row, row pitch `pitch`
// elements, `rows` rows), boxes of 32 x box_rows, 64-byte swizzle, zero fill outside the tensor.
bool tc_encode_map(CUtensorMap* map, const void* base, long long inner, long long pitch, long long rows,
                   int box_rows);

// One operand tile: digit plane k starts at row y0 + k plane_rows of the tensor map.
struct TcsTile {
  const CUtensorMap* map;
  int y0;
  int plane_rows;
};

// Shared-memory state of the loop.
struct TcsBarriers {
  uint64_t full[TCS_NBUF];   // copies of a slot landed
  uint64_t empty[TCS_NBUF];  // MMAs reading a slot done
  uint64_t acc;              // accumulators of a K chunk complete
  uint32_t tmem;             // tensor-memory base of the CTA
};

// Block-wide set-up: tensor memory (warp 0) and the mbarriers.  Returns the TMEM base.
__device__ __forceinline__ uint32_t tcs_setup(TcsBarriers& bar) {
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    tc_alloc(&bar.tmem, TCS_TMEM_COLS);
    tc_relinquish();
  }
  if (threadIdx.x == 32) {
#pragma unroll
    for (int b = 0; b < TCS_NBUF; ++b) {
      tc_mbar_init(&bar.full[b], 1);
      tc_mbar_init(&bar.empty[b], 1);
    }
    tc_mbar_init(&bar.acc, 1);
    tc_mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return bar.tmem;
}

// What thread 0 has in flight: the last stage copied, the last stage whose MMAs were committed,
// and the K chunk whose accumulator commit was not yet seen complete (-1: none).
struct TcsProgress {
  int issued = -1, committed = -1, acc = -1;
};

// Block-wide tear-down.  After an abort, thread 0 waits (bounded) for the copies it issued, the
// MMAs it committed and their commits' arrivals, so nothing lands in shared or tensor memory
// after the block is gone; then tensor memory is freed.
__device__ __forceinline__ void tcs_teardown(TcsBarriers& bar, bool abort, const TcsProgress& pr, int* status) {
  if (abort && threadIdx.x == 0) {
    atomicOr(status, LMBD_FLAG_TIMEOUT);
    for (int s = pr.committed + 1; s <= pr.issued; ++s)
      tc_mbar_wait(&bar.full[s % TCS_NBUF], (s / TCS_NBUF) & 1, TCS_WAIT_CYCLES);
    if (pr.committed >= 0)
      tc_mbar_wait(&bar.empty[pr.committed % TCS_NBUF], (pr.committed / TCS_NBUF) & 1, TCS_WAIT_CYCLES);
    if (pr.acc >= 0) tc_mbar_wait(&bar.acc, pr.acc & 1, TCS_WAIT_CYCLES);
  }
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tc_dealloc(bar.tmem, TCS_TMEM_COLS);
  }
}

// TMEM address of lane quarter (warp % 4), column `col`.
__device__ __forceinline__ uint32_t tcs_lane_addr(uint32_t tmem, int col) {
  return tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + (uint32_t)col;
}

// The main loop (all 256 threads; thread 0 issues copies and MMAs and waits for them).
// consume() runs block-wide at the end of every K chunk with the accumulators complete in TMEM.
// Every wait is bounded by `budget` cycles; returns false if one ran out.  `pr` (thread 0) keeps
// what is in flight, for the tear-down.
template <int S, int NB, class Consume>
__device__ __forceinline__ bool tcs_mainloop(const TcsTile& A, const TcsTile& B, int K, uint32_t sbase,
                                             TcsBarriers& bar, long long budget, TcsProgress& pr, Consume&& consume) {
  using Sh = TcsShape<S, NB>;
  const int tid = threadIdx.x;
  const int nst = (K + TCS_KS - 1) / TCS_KS;
  constexpr int kPerChunk = OZ_KCHUNK / TCS_KS;
  const uint32_t tmem = bar.tmem;
  auto load = [&](int s) {
    const int slot = s % TCS_NBUF;
    const uint32_t sA = sbase + slot * Sh::kSlot;
    const uint32_t sB = sA + S * Sh::kAPlane;
    tc_mbar_expect_tx(&bar.full[slot], (uint32_t)Sh::kSlot);
#pragma unroll
    for (int k = 0; k < S; ++k) tc_tma_load_2d(sA + k * Sh::kAPlane, A.map, s * TCS_KS, A.y0 + k * A.plane_rows, &bar.full[slot]);
#pragma unroll
    for (int k = 0; k < S; ++k) tc_tma_load_2d(sB + k * Sh::kBPlane, B.map, s * TCS_KS, B.y0 + k * B.plane_rows, &bar.full[slot]);
    pr.issued = s;
  };
  if (tid == 0)
    for (int s = 0; s < TCS_NBUF && s < nst; ++s) load(s);
  const int nchunk = (nst + kPerChunk - 1) / kPerChunk;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int s0 = ch * kPerChunk, s1 = min(nst, s0 + kPerChunk);
    bool to = false;
    if (tid == 0) {
      for (int s = s0; s < s1; ++s) {
        const int slot = s % TCS_NBUF;
        if (!tc_mbar_wait(&bar.full[slot], (s / TCS_NBUF) & 1, budget)) {
          to = true;
          break;
        }
        tc_fence_after();
        const uint32_t sA = sbase + slot * Sh::kSlot;
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
                          (s == s0 && kk == 0 && k == 0) ? 0u : 1u);
            }
          }
        tc_commit(&bar.empty[slot]);
        pr.committed = s;
        // refill the slot of stage s - 1 with stage s - 1 + TCS_NBUF once its MMAs are done
        const int r = s - 1 + TCS_NBUF;
        if (s >= 1 && r < nst) {
          if (!tc_mbar_wait(&bar.empty[(s - 1) % TCS_NBUF], ((s - 1) / TCS_NBUF) & 1, budget)) {
            to = true;
            break;
          }
          load(r);
        }
      }
      if (!to) {
        // accumulators of this chunk complete: seen by thread 0, published by the barrier
        tc_commit(&bar.acc);
        pr.acc = ch;
        if (tc_mbar_wait(&bar.acc, ch & 1, budget)) pr.acc = -1;
        else to = true;
      }
    }
    if (__syncthreads_or(to)) return false;
    tc_fence_after();
    consume();
    tc_fence_before();
    __syncthreads();
  }
  return true;
}
