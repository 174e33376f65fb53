// FP64 matrix products on the bf16 tensor cores by exact integer slicing.
//
// GB300 runs FP64 at 1/70 of FP32, while its bf16 tensor cores are two orders of magnitude
// faster still.  A product C = A B of FP64 matrices is evaluated from integer digit planes (the
// slicing scheme of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", and its tensor-core use by
// Mukunoki et al.):
//   * every row of A (column of B) is scaled by a power of two 2^e so that |a| < 2^e;
//   * the scaled value is truncated to 7 S bits and split into S signed 7-bit digits,
//       a = 2^e sum_k d_k 2^{-7k},  |d_k| <= 127  (exact in bf16);
//   * digit planes are multiplied on the tensor cores (tcgen05.mma, tc_sliced.cuh, or the
//     warp-level mma.sync below) with FP32 accumulation; every product d_k d_l is an integer
//     below 2^14, and the K dimension is accumulated in chunks of at most OZ_KCHUNK = 256
//     terms, so one digit pair sums to less than 2^22;
//   * products with the same digit order m = k + l share one FP32 accumulator: with at most
//     four pairs per order below m = 6 every partial sum stays below 2^24 and is exact;
//     higher orders can round, at a level below 2^-52 of the leading term.  Pairs with
//     m > S - 1 are dropped; after each K chunk the orders are recombined exactly as 64-bit
//     integers, Y += sum_m acc_m 2^{7 (S - 1 - m)}, and the result is scaled once in FP64:
//       c = 2^{e_row + e_col - 7 (S + 1)} Y.
// The result differs from the FP64 product by at most ~S 2^{-7S} sum |a||b| (normwise);
// the digit count S is chosen per product from the accuracy its consumer needs.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

// Exponent e with |v| < 2^e for the largest |v| (biased exponent of v, 0 for zero).
__device__ __forceinline__ int oz_biased_exp(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}

// Scale exponent from the largest biased exponent of a row/column: |v| < 2^(ex - 1022).
__device__ __forceinline__ int oz_scale_exp(int max_biased) { return max_biased == 0 ? -1022 : max_biased - 1022; }

// K chunk over which one digit order is accumulated in FP32 before the exact integer
// recombination (every partial sum of the low orders stays an integer below 2^24).
#define OZ_KCHUNK 256

__device__ __forceinline__ unsigned short oz_bf16_bits(int d) {
  __nv_bfloat16 h = __float2bfloat16_rn((float)d);
  return *reinterpret_cast<unsigned short*>(&h);
}

// Signed 7-bit digits of v relative to 2^e (|v| < 2^e): v ~= 2^e sum_{k=1..S} d_k 2^{-7k},
// truncated toward zero (integer operations only), stored as bf16 bits at dst[(k - 1) plane].
// S is a compile-time constant so the digits stay in registers.
template <int S>
__device__ __forceinline__ void oz_store_digits(unsigned short* dst, long long plane, double v, int e) {
  const long long bits = __double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7ff);
  unsigned long long U = 0;
  if (ex != 0) {
    const unsigned long long mant = (unsigned long long)(bits & 0xFFFFFFFFFFFFFLL) | (1ULL << 52);
    const int sh = (ex - 1075) + 7 * S - e;
    if (sh >= 0) U = mant << sh;
    else if (sh > -64) U = mant >> (-sh);
  }
  const int sg = bits < 0 ? -1 : 1;
#pragma unroll
  for (int k = 0; k < S; ++k) dst[k * plane] = oz_bf16_bits(sg * (int)((U >> (7 * (S - 1 - k))) & 127ULL));
}

// 2^E as a double (E clamped to the normal range; tiny scales flush to zero).
__device__ __forceinline__ double oz_pow2(int E) {
  if (E < -1022) return 0.0;
  if (E > 1023) E = 1023;
  return __longlong_as_double((long long)(E + 1023) << 52);
}

// d += a b for one m16n8k16 bf16 tile (row-major A, column-major B, FP32 accumulate).
__device__ __forceinline__ void oz_mma(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t oz_ld32(const unsigned short* p) { return *reinterpret_cast<const uint32_t*>(p); }

// ---------------------------------------------------------------------------------------
// shared-memory staged variant
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void oz_cp_async16(void* smem_dst, const void* gsrc, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(bytes));
}
__device__ __forceinline__ void oz_cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void oz_cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ uint32_t oz_lds32(const unsigned short* p) { return *reinterpret_cast<const uint32_t*>(p); }

// One warp, one k16 step from shared-memory tiles: A digit planes [S][*][lda] at rows ar..ar+15,
// B digit planes [S][*][ldb] at rows br..br+15 (two n8 tiles).
template <int S>
__device__ __forceinline__ void oz_warp_k16_smem(const unsigned short* sA, int pa, int lda, int ar,
                                                 const unsigned short* sB, int pb, int ldb, int br, int kk,
                                                 float (&acc)[S][2][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t b[S][2][2];
#pragma unroll
  for (int l = 0; l < S; ++l)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const unsigned short* q = sB + l * pb + (br + nt * 8 + g) * ldb + kk + 2 * t;
      b[l][nt][0] = oz_lds32(q);
      b[l][nt][1] = oz_lds32(q + 8);
    }
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const unsigned short* q = sA + k * pa + (ar + g) * lda + kk + 2 * t;
    uint32_t a[4];
    a[0] = oz_lds32(q);
    a[1] = oz_lds32(q + 8 * lda);
    a[2] = oz_lds32(q + 8);
    a[3] = oz_lds32(q + 8 * lda + 8);
#pragma unroll
    for (int l = 0; l < S - k; ++l)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) oz_mma(acc[k + l][nt], a, b[l][nt]);
  }
}

// Exact integer recombination of the digit-order groups: Y += sum_m acc_m 2^{7 (S - 1 - m)}
// (every group value is an integer held exactly by the FP32 accumulator or rounded to one).
template <int S>
__device__ __forceinline__ void oz_int_combine(float (&acc)[S][2][4], long long (&Y)[2][4]) {
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      long long s = 0;
#pragma unroll
      for (int m = 0; m < S; ++m) s += (long long)__float2int_rn(acc[m][nt][v]) << (7 * (S - 1 - m));
      Y[nt][v] += s;
#pragma unroll
      for (int m = 0; m < S; ++m) acc[m][nt][v] = 0.f;
    }
}
