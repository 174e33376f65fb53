// Krylov chain step v_{m+1} = D (T_LR W) of Eq. E_k on the fifth-generation tensor cores.
//
// Same sliced arithmetic as the warp-level kernel (ozaki.cuh): T_LR and W = D v_m are cut into
// S signed 7-bit digit planes, digit pairs (k, l) with k + l <= S - 1 are multiplied on the
// tensor cores with FP32 accumulation, one accumulator per digit order, K chunks of at most
// 256, and the orders are recombined exactly in 64-bit integers.  One CTA owns a 128-row tile of
// one central atom's T_LR and all 48 columns of W; the tcgen05 main loop (tc_sliced.cuh,
// M = 128, N = 48) accumulates in tensor memory, the 8 warps read the accumulators at the end of
// each K chunk (warp w: rows 32 (w % 4) .., columns 24 (w / 4) ..), and the epilogue scales by
// the row and column exponents and by D.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_sliced.cuh"

#define CTC_NB 48

namespace {

__device__ __forceinline__ int ctc_mpad(int n) { return (n + 63) / 64 * 64; }
__device__ __forceinline__ int ctc_kpad(int n) { return (n + 15) / 16 * 16; }

template <int S>
__global__ void __launch_bounds__(256, 1)
    k_chain_tc(Work w, DevParams p, int m, int c0, int tiles_per_c, int st, const __grid_constant__ CUtensorMap tmT,
               const __grid_constant__ CUtensorMap tmW) {
  using Sh = TcsShape<S, CTC_NB>;
  extern __shared__ unsigned char tc_dyn[];
  __shared__ TcsBarriers bar;
  const int c = c0 + blockIdx.x / tiles_per_c;
  const int tile = blockIdx.x % tiles_per_c;
  if (c >= w.n_atoms) return;
  const int N = 3 * w.counts[c].ns, Mpad = ctc_mpad(N), Kpad = ctc_kpad(N);
  const int row0 = tile * TCS_M;
  if (row0 >= N) return;
  // T digit planes: rows off_tr[c] st + k Mpad + r of the wave's T map (row pitch w.tk);
  // W digit planes: rows ((c - wc0) S + k) 48 + r of the wave's W map
  const TcsTile A{&tmT, (int)(w.off_tr[c] * st - w.trow0) + row0, Mpad};
  const TcsTile B{&tmW, (c - w.wc0) * S * CTC_NB, CTC_NB};
  const uint32_t sbase = (tc_smem_u32(tc_dyn) + 1023u) & ~1023u;
  const uint32_t tmem = tcs_setup(bar);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cb = (warp >> 2) * 24;
  long long Y[24];
#pragma unroll
  for (int j = 0; j < 24; ++j) Y[j] = 0;
  TcsProgress pr;
  const bool ok = tcs_mainloop<S, CTC_NB>(A, B, Kpad, sbase, bar, p.tc_wait, pr, [&]() {
#pragma unroll
    for (int g = 0; g < S; ++g)
#pragma unroll
      for (int j8 = 0; j8 < 3; ++j8) {
        float v[8];
        tc_ld8(tcs_lane_addr(tmem, g * Sh::kGroupCols + cb + j8 * 8), v);
#pragma unroll
        for (int i = 0; i < 8; ++i) Y[j8 * 8 + i] += (long long)__float2int_rn(v[i]) << (7 * (S - 1 - g));
      }
  });
  tcs_teardown(bar, !ok, pr, w.status);
  if (!ok) return;

  const int row = row0 + 32 * (warp & 3) + lane;
  if (row >= N) return;
  const long long offs = w.off_s[c];
  const int ncv = 3 * p.n_freq;
  double* Vout = w.vkr + (long long)m * w.vstride + (offs * 3) * ncv + (long long)row * ncv;
  const double* dsq = w.dsq + offs * p.nq + (row / 3) * p.nq;
  const int er = w.texp[w.off_tr[c] + row];
#pragma unroll
  for (int j = 0; j < 24; ++j) {
    const int col = cb + j;
    if (col < ncv) {
      const int ec = w.wexp[(long long)c * 48 + col];
      Vout[col] = dsq[col / 3 + 1] * ((double)Y[j] * oz_pow2(er + ec - 7 * (S + 1)));
    }
  }
}

static_assert(TcsShape<6, CTC_NB>::kBytes <= 232448, "staging ring exceeds the shared memory of a CTA");

}  // namespace

size_t chain_tc_smem(int digits) { return digits == 6 ? TcsShape<6, CTC_NB>::kBytes : TcsShape<5, CTC_NB>::kBytes; }

// 2-D tensor map over bf16 digit planes: `inner` elements per row (row pitch `pitch` elements),
// `rows` rows, boxes of 32 x box_rows, 64-byte swizzle, zero fill outside the tensor.
bool tc_encode_map(CUtensorMap* map, const void* base, long long inner, long long pitch, long long rows,
                   int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!encode || rows <= 0 || inner <= 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TCS_KS, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool launch_chain_tc(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, int digits, int st,
                     cudaStream_t s) {
  if (c1 <= c0) return true;
  if (digits != 5 && digits != 6) return false;
  launch_slice_w(w, p, m, c0, c1, digits, s);
  const int tiles = (3 * max_ns + TCS_M - 1) / TCS_M;
  // the wave's T planes start at row trow0 of the rebased pointer; its W planes at centre wc0
  CUtensorMap tmT, tmW;
  const unsigned short* traw = w.tdig + w.trow0 * w.tk;
  const unsigned short* wraw = w.wdig + (long long)w.wc0 * 48 * digits * w.tk;
  if (!tc_encode_map(&tmT, traw, w.tk, w.tk, w.trows, TCS_M) ||
      !tc_encode_map(&tmW, wraw, w.tk, w.tk, (long long)w.wcn * 48 * digits, CTC_NB))
    return false;
  if (digits == 6) {
    raise_smem_limit((const void*)k_chain_tc<6>, TcsShape<6, CTC_NB>::kBytes);
    k_chain_tc<6><<<(c1 - c0) * tiles, 256, TcsShape<6, CTC_NB>::kBytes, s>>>(w, p, m, c0, tiles, st, tmT, tmW);
  } else {
    raise_smem_limit((const void*)k_chain_tc<5>, TcsShape<5, CTC_NB>::kBytes);
    k_chain_tc<5><<<(c1 - c0) * tiles, 256, TcsShape<5, CTC_NB>::kBytes, s>>>(w, p, m, c0, tiles, st, tmT, tmW);
  }
  return true;
}
