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
#include "tc_sliced.cuh"

#define CTC_NB 48

namespace {

__device__ __forceinline__ int ctc_mpad(int n) { return (n + 63) / 64 * 64; }
__device__ __forceinline__ int ctc_kpad(int n) { return (n + 15) / 16 * 16; }

template <int S>
__global__ void __launch_bounds__(256, 1) k_chain_tc(Work w, DevParams p, int m, int c0, int tiles_per_c, int st) {
  using Sh = TcsShape<S, CTC_NB>;
  extern __shared__ unsigned char tc_dyn[];
  __shared__ uint64_t mbar[TCS_NBUF];
  __shared__ uint32_t tmem_holder;
  const int c = c0 + blockIdx.x / tiles_per_c;
  const int tile = blockIdx.x % tiles_per_c;
  if (c >= w.n_atoms) return;
  const int N = 3 * w.counts[c].ns, Mpad = ctc_mpad(N), Kpad = ctc_kpad(N);
  const int row0 = tile * TCS_M;
  if (row0 >= N) return;
  // T digit planes [st][Mpad][Kpad] (rows N..Mpad are zero), W digit planes [S][48][Kpad]
  const TcsOperand A{w.tdig + w.off_tq[c] * st + (long long)row0 * Kpad, (long long)Mpad * Kpad, Kpad, Mpad - row0};
  const TcsOperand B{w.wdig + w.off_kp[c] * 48 * S, 48LL * Kpad, Kpad, CTC_NB};
  const uint32_t sbase = (tc_smem_u32(tc_dyn) + 1023u) & ~1023u;
  const uint32_t tmem = tcs_setup(&tmem_holder, mbar);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cb = (warp >> 2) * 24;
  long long Y[24];
#pragma unroll
  for (int j = 0; j < 24; ++j) Y[j] = 0;
  int committed = -1;
  const bool ok = tcs_mainloop<S, CTC_NB>(A, B, Kpad, sbase, tmem, mbar, committed, [&]() {
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
  tcs_teardown(tmem, !ok, committed, mbar, w.status);
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

void launch_chain_tc(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, int digits, int st,
                     cudaStream_t s) {
  if (c1 <= c0) return;
  launch_slice_w(w, p, m, c0, c1, digits, s);
  const int tiles = (3 * max_ns + TCS_M - 1) / TCS_M;
  if (digits == 6) {
    raise_smem_limit((const void*)k_chain_tc<6>, TcsShape<6, CTC_NB>::kBytes);
    k_chain_tc<6><<<(c1 - c0) * tiles, 256, TcsShape<6, CTC_NB>::kBytes, s>>>(w, p, m, c0, tiles, st);
  } else {
    raise_smem_limit((const void*)k_chain_tc<5>, TcsShape<5, CTC_NB>::kBytes);
    k_chain_tc<5><<<(c1 - c0) * tiles, 256, TcsShape<5, CTC_NB>::kBytes, s>>>(w, p, m, c0, tiles, st);
  }
}
