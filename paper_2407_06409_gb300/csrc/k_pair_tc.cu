// Adjoint pair matrix M' = P Q^T on the fifth-generation tensor cores, with the per-pair
// contraction against dT_LR/dr and dT_LR/dS~ (the derivative pieces of Sec. III.D, exact).
//
// P and Q (3 n_s rows, 3 n_freq (n_max - 2) columns per central atom) are cut into 5 digit
// planes by k_slice_pq.  One CTA owns a tile of 42 row sites (126 rows of P) by 32 column sites
// (96 rows of Q): the tcgen05 main loop (tc_sliced.cuh, M = 128, N = 96) accumulates the digit
// orders in tensor memory, the 8 warps recombine them as integers (warp w: rows 32 (w % 4) ..,
// columns 48 (w / 4) ..), scale them by the row and column exponents into an FP64 tile in
// shared memory, and every thread then runs the pair epilogue on site pairs s > t of the tile;
// per-site sums go to the force accumulator and the SCS-radius seed with one atomic per site.
#include "pair_epilogue.cuh"
#include "tc_sliced.cuh"

#define PTC_SA 42   // row sites per tile (126 of the 128 MMA rows)
#define PTC_SB 32   // column sites per tile (N = 96)
#define PTC_NB 96
#define PTC_LD 97   // row stride of the FP64 tile in shared memory

namespace {

__device__ __forceinline__ int ptc_kpad(int n) { return (n + 15) / 16 * 16; }
inline long long ptc_kpad_host(int n) { return (n + 15) / 16 * 16; }

template <int S>
__global__ void __launch_bounds__(256, 1)
    k_pair_tc(Work w, DevParams p, int c0, int nb_max, int tiles_per_c, const __grid_constant__ CUtensorMap tmP,
              const __grid_constant__ CUtensorMap tmQ) {
  using Sh = TcsShape<S, PTC_NB>;
  extern __shared__ unsigned char tc_dyn[];
  __shared__ TcsBarriers bar;
  const int c = c0 + blockIdx.x / tiles_per_c;
  const int tile = blockIdx.x % tiles_per_c;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns;
  const int s0 = PTC_SA * (tile / nb_max), t0 = PTC_SB * (tile % nb_max);
  // tiles without a site pair s > t inside the sphere have nothing to do
  if (s0 >= ns || t0 >= ns || min(s0 + PTC_SA, ns) - 1 <= t0) return;
  const int R = 3 * ((ns + 15) / 16 * 16), Kp = ptc_kpad(w.ncol);
  // P and Q digit planes of this centre: rows off_sp[c] 3 S + k R + r of the wave's maps (pitch Kp)
  const int prow = (int)(w.off_sp[c] * 3 * S - w.prow0);
  const TcsTile A{&tmP, prow + 3 * s0, R};
  const TcsTile B{&tmQ, prow + 3 * t0, R};
  const uint32_t sraw = tc_smem_u32(tc_dyn);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  const uint32_t tmem = tcs_setup(bar);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cb = (warp >> 2) * 48;
  long long Y[48];
#pragma unroll
  for (int j = 0; j < 48; ++j) Y[j] = 0;
  TcsProgress pr;
  const bool ok = tcs_mainloop<S, PTC_NB>(A, B, Kp, sbase, bar, p.tc_wait, pr, [&]() {
#pragma unroll
    for (int g = 0; g < S; ++g)
#pragma unroll
      for (int j8 = 0; j8 < 6; ++j8) {
        float v[8];
        tc_ld8(tcs_lane_addr(tmem, g * Sh::kGroupCols + cb + j8 * 8), v);
#pragma unroll
        for (int i = 0; i < 8; ++i) Y[j8 * 8 + i] += (long long)__float2int_rn(v[i]) << (7 * (S - 1 - g));
      }
  });
  tcs_teardown(bar, !ok, pr, w.status);
  if (!ok) return;

  // FP64 tile (126 x 96) and per-pair results (42 x 32 x 4) in the drained staging ring
  double* Ms = reinterpret_cast<double*>(tc_dyn + (sbase - sraw));
  double* gp = Ms + 3 * PTC_SA * PTC_LD;
  const int row = 32 * (warp & 3) + lane;
  const int* pe = w.pexp + w.off_sp[c] * 3;
  const int* qe = w.qexp + w.off_sp[c] * 3;
  if (row < 3 * PTC_SA) {
    const bool rv = 3 * s0 + row < R;
    const int er = rv ? pe[3 * s0 + row] : 0;
#pragma unroll
    for (int j = 0; j < 48; ++j) {
      const int col = cb + j;
      double v = 0.0;
      if (rv && 3 * t0 + col < R) v = (double)Y[j] * oz_pow2(er + qe[3 * t0 + col] - 7 * (S + 1));
      Ms[row * PTC_LD + col] = v;
    }
  }
  __syncthreads();
  const long long offs = w.off_s[c];
  const long long offt = w.off_t[c];
  for (int e = tid; e < PTC_SA * PTC_SB; e += blockDim.x) {
    const int sl = e / PTC_SB, tl = e % PTC_SB;
    double a3[3][3];
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
      for (int be = 0; be < 3; ++be) a3[al][be] = Ms[(3 * sl + al) * PTC_LD + 3 * tl + be];
    pair_epilogue(w, offs, offt, s0 + sl, t0 + tl, ns, a3, gp + 4 * e);
  }
  __syncthreads();
  // deterministic per-site sums: row sites get -g, column sites +g; one atomic per site
  if (tid < PTC_SA + PTC_SB) {
    const bool rs = tid < PTC_SA;
    const int l = rs ? tid : tid - PTC_SA;
    const int ss = (rs ? s0 : t0) + l;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0, sb = 0.0;
    const int n = rs ? PTC_SB : PTC_SA;
    for (int o = 0; o < n; ++o) {
      const double* v = gp + 4 * (rs ? l * PTC_SB + o : o * PTC_SB + l);
      g0 += v[0];
      g1 += v[1];
      g2 += v[2];
      sb += v[3];
    }
    if (ss < ns) {
      const double sgn = rs ? -1.0 : 1.0;
      const int a = w.site_atom[(long long)c * w.site_cap + ss];
      if (g0 != 0.0 || g1 != 0.0 || g2 != 0.0) atomic_add3(w.gacc + 3 * a, sgn * g0, sgn * g1, sgn * g2);
      if (sb != 0.0) atomicAdd(&w.rbar[offs + ss], sb);
    }
  }
}

static_assert(TcsShape<5, PTC_NB>::kBytes <= 232448, "staging ring exceeds the shared memory of a CTA");
static_assert((3 * PTC_SA * PTC_LD + 4 * PTC_SA * PTC_SB) * 8 <= TcsShape<5, PTC_NB>::kBytes - 1024,
              "FP64 tile and pair results must fit in the staging ring");

}  // namespace

// Digit planes of P and Q (k_slice_pq), then the tcgen05 pair kernel; digits must be 5.
bool launch_pair_tc(const Work& w, const DevParams& p, int c0, int c1, int max_ns, int digits, cudaStream_t s) {
  if (c1 <= c0) return true;
  if (digits != 5) return false;
  launch_slice_pq(w, c0, c1, digits, s);
  const int na = (max_ns + PTC_SA - 1) / PTC_SA, nb = (max_ns + PTC_SB - 1) / PTC_SB;
  const long long Kp = ptc_kpad_host(w.ncol);
  CUtensorMap tmP, tmQ;
  if (!tc_encode_map(&tmP, w.pdig + w.prow0 * Kp, Kp, Kp, w.prows, TCS_M) ||
      !tc_encode_map(&tmQ, w.qdig + w.prow0 * Kp, Kp, Kp, w.prows, PTC_NB))
    return false;
  using Sh = TcsShape<5, PTC_NB>;
  raise_smem_limit((const void*)k_pair_tc<5>, Sh::kBytes);
  k_pair_tc<5><<<(c1 - c0) * na * nb, 256, Sh::kBytes, s>>>(w, p, c0, nb, na * nb, tmP, tmQ);
  return true;
}
