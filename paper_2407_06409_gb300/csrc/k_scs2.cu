// Stage 1, mixed precision: local SCS solves (Sec. III.B, Eq. local_pol) for every
// central atom k and frequency omega_q, FP64 results.
//
//   B_K = diag(1/alpha_bar_i) + T_SR,K,ij (i, j in K1),  d_K,i = 1 - sum_{j in K2} T_SR,K,ij alpha_bar_j
//   X = B_K^-1 d_K,  alpha_K,i = Tr(X_i)/3,  alpha_I,k = alpha_K,k
//   T_SR,K,ij = F(r) [A0(r) I + B0(r) r r^T],  F = f_inner f_SR (1 - f(r, S_ij)),
//   A0 = g/r^3, B0 = (h~ - 3 g)/r^5 (Eqs. T_SR, g-func, h-func, written out in lmbd_internal.cuh)
//
// Design for GB300, whose FP64 pipe runs at 1/70 of FP32:
//  * the pairs (i in K1, j in K1 u K2) with r_ij < r_SCS are listed once per central atom
//    with their frequency-independent geometry and damping F, dF/dr (k_scs_count/k_scs_fill);
//  * erf and exp of r/sigma_ij are evaluated once per atom pair and frequency (k_pair_radial,
//    FP64), not once per local system holding the pair; the local systems read the table;
//  * B_K is factorised in FP32 (Cholesky, packed lower triangle in shared memory) and the
//    FP64 solution is recovered by iterative refinement: the residual d - B X is formed in
//    FP64 from the sparse pair list, corrections come from the FP32 factor (classical mixed-
//    precision refinement, Wilkinson/Moler; converges when cond(B) * eps_fp32 << 1);
//  * the adjoint solve B lambda = dL/dX reuses the stored FP32 factor with the same refinement,
//    and contracts dB/dr, dd/dr pair by pair from the stored radial terms.
#include "lmbd_internal.cuh"
#include "ff.cuh"

// pair predicate shared by the counting and filling kernels (identical FP64 arithmetic)
__device__ __forceinline__ bool scs_pair_in(const double* xs, int ld, int i, int j, double rc2, double& rx,
                                            double& ry, double& rz, double& r2) {
  rx = xs[j] - xs[i];
  ry = xs[ld + j] - xs[ld + i];
  rz = xs[2 * ld + j] - xs[2 * ld + i];
  r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
  return r2 < rc2;
}

// FP32 screen of the same predicate: pairs farther than a relative 1e-4 from the radius are
// decided in FP32 (the FP32 error of r^2 is below 1e-5 r_SCS^2 for sites within 27 r_SCS of
// the centre); the others take the FP64 test, so the decision is always the FP64 one.
__device__ __forceinline__ bool scs_pair_in_screened(const float* xf, const double* xs, int ld, int i, int j,
                                                     float lo2, float hi2, double rc2) {
  const float dx = xf[j] - xf[i], dy = xf[ld + j] - xf[ld + i], dz = xf[2 * ld + j] - xf[2 * ld + i];
  const float r2f = dx * dx + dy * dy + dz * dz;
  if (r2f < lo2) return true;
  if (r2f > hi2) return false;
  double rx, ry, rz, r2;
  return scs_pair_in(xs, ld, i, j, rc2, rx, ry, rz, r2);
}

__device__ __forceinline__ long long packed_idx(int i, int k) { return (long long)i * (i + 1) / 2 + k; }

// ---------------------------------------------------------------------------------------
// pair lists: count (before the workspace is sized) and fill
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scs_count(Work w, DevParams p, int max_n12) {
  extern __shared__ double smem_d[];
  double* xs = smem_d;                 // 3 x max_n12
  float* xf = (float*)(xs + 3 * max_n12);   // 3 x max_n12, FP32 copies
  __shared__ int cnt_k1k1, cnt_k2;
  const int c = blockIdx.x;
  if (c >= w.n_atoms) return;
  const Counts cn = w.counts[c];
  const int n1 = cn.n1, n12 = cn.n12;
  const long long sbase = (long long)c * w.site_cap;
  const int tid = threadIdx.x;
  for (int s = tid; s < n12; s += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      const double v = w.site_x[3 * (sbase + s) + d];
      xs[d * max_n12 + s] = v;
      xf[d * max_n12 + s] = (float)v;
    }
  if (tid == 0) { cnt_k1k1 = 0; cnt_k2 = 0; }
  __syncthreads();
  const double rc2 = p.r_scs * p.r_scs;
  const float lo2 = (float)(rc2 * (1.0 - 1e-4)), hi2 = (float)(rc2 * (1.0 + 1e-4));
  int a = 0, b = 0;
  const int nkk = n1 * (n1 - 1) / 2;
  for (int e = tid; e < nkk; e += blockDim.x) {
    int i = (int)((sqrtf(8.0f * e + 1.0f) + 1.0f) * 0.5f);
    while (i * (i - 1) / 2 > e) --i;
    while ((i + 1) * i / 2 <= e) ++i;
    int j = e - i * (i - 1) / 2;
    a += scs_pair_in_screened(xf, xs, max_n12, i, j, lo2, hi2, rc2);
  }
  const int n2 = n12 - n1;
  for (int e = tid; e < n1 * n2; e += blockDim.x) {
    int i = e / n2, j = n1 + e % n2;
    b += scs_pair_in_screened(xf, xs, max_n12, i, j, lo2, hi2, rc2);
  }
  atomicAdd(&cnt_k1k1, a);
  atomicAdd(&cnt_k2, b);
  __syncthreads();
  if (tid == 0) {
    w.pcount[2 * c] = cnt_k1k1 + cnt_k2;   // unique pairs
    w.pcount[2 * c + 1] = 2 * cnt_k1k1;    // adjacency entries (both directions of K1-K1 pairs)
  }
}

// One block per central atom.  Pairs are ordered by owner row i: first the K1 partners
// j < i (ascending), then the K2 partners (ascending); adjacency rows list every K1
// partner j != i (ascending) with the index of the shared pair.
__global__ void __launch_bounds__(256) k_scs_fill(Work w, DevParams p, int c0, int max_n12, int max_n1) {
  extern __shared__ double smem_d[];
  double* xs = smem_d;                             // 3 x max_n12
  int* pid = (int*)(xs + 3 * max_n12);             // max_n1 x max_n1 (pair index, -1 = none)
  int* rowk1 = pid + max_n1 * max_n1;              // max_n1
  int* rowcnt = rowk1 + max_n1;                    // max_n1
  int* rowstart = rowcnt + max_n1;                 // max_n1 + 1
  int* adjcnt = rowstart + max_n1 + 1;             // max_n1
  int* adjstart = adjcnt + max_n1;                 // max_n1 + 1
  int* k2cnt = adjstart + max_n1 + 1;              // max_n12
  int* klist = k2cnt + max_n12;                    // per warp max_n1: atoms of one K1 list
  float* xf = (float*)(klist + 8 * max_n1);        // 3 x max_n12, FP32 copies of xs
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const Counts cn = w.counts[c];
  const int n1 = cn.n1, n12 = cn.n12;
  const long long sbase = (long long)c * w.site_cap;
  const long long offp = w.off_p[c], offa = w.off_a[c], rbase = w.off_k1[c] + c;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32, nw = blockDim.x / 32;
  for (int s = tid; s < n12; s += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      const double v = w.site_x[3 * (sbase + s) + d];
      xs[d * max_n12 + s] = v;
      xf[d * max_n12 + s] = (float)v;
    }
  for (int e = tid; e < n1 * n1; e += blockDim.x) pid[(e / n1) * max_n1 + e % n1] = -1;
  __syncthreads();
  const double rc2 = p.r_scs * p.r_scs;
  const float lo2 = (float)(rc2 * (1.0 - 1e-4)), hi2 = (float)(rc2 * (1.0 + 1e-4));
  // phase 1: per-row counts
  for (int i = warp; i < n1; i += nw) {
    int k1 = 0, k2 = 0;
    for (int j0 = 0; j0 < i; j0 += 32) {
      int j = j0 + lane;
      bool in = j < i && scs_pair_in_screened(xf, xs, max_n12, i, j, lo2, hi2, rc2);
      k1 += __popc(__ballot_sync(0xffffffffu, in));
    }
    for (int j0 = n1; j0 < n12; j0 += 32) {
      int j = j0 + lane;
      bool in = j < n12 && scs_pair_in_screened(xf, xs, max_n12, i, j, lo2, hi2, rc2);
      k2 += __popc(__ballot_sync(0xffffffffu, in));
    }
    if (lane == 0) { rowk1[i] = k1; rowcnt[i] = k1 + k2; }
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int i = 0; i < n1; ++i) { rowstart[i] = run; run += rowcnt[i]; }
    rowstart[n1] = run;
  }
  __syncthreads();
  // phase 2a: pairs in order (row, partner) and their entry in the atom-pair radial table
  int* lst = klist + warp * max_n1;
  for (int i = warp; i < n1; i += nw) {
    int pos = rowstart[i];
    // atoms of the K1 list of site i's atom, for the radial-table lookup below
    const int ai = w.site_atom[sbase + i];
    const int na = w.counts[ai].n1;
    const long long ab = (long long)ai * w.site_cap;
    __syncwarp();
    for (int t = lane; t < na; t += 32) lst[t] = w.site_atom[ab + t];
    __syncwarp();
    for (int pass = 0; pass < 2; ++pass) {
      int jb = pass == 0 ? 0 : n1, je = pass == 0 ? i : n12;
      for (int j0 = jb; j0 < je; j0 += 32) {
        int j = j0 + lane;
        bool in = j < je && scs_pair_in_screened(xf, xs, max_n12, i, j, lo2, hi2, rc2);
        unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
          int slot = pos + __popc(m & ((1u << lane) - 1u));
          long long q = offp + slot;
          w.pr_ij[2 * q] = i;
          w.pr_ij[2 * q + 1] = j;
          // the same atom pair in the radial table: the site of atom aj at displacement
          // r = x_j - x_i in atom ai's own K1 list (periodic images of one atom are far apart,
          // so an FP32 match is unambiguous; none only if r ties r_SCS to rounding)
          const int aj = w.site_atom[sbase + j];
          const float rxf = xf[j] - xf[i], ryf = xf[max_n12 + j] - xf[max_n12 + i],
                      rzf = xf[2 * max_n12 + j] - xf[2 * max_n12 + i];
          int gi = -1;
          for (int t = 1; t < na; ++t) {
            if (lst[t] != aj) continue;
            const double* xt = w.site_x + 3 * (ab + t);
            const float dx = (float)xt[0] - rxf, dy = (float)xt[1] - ryf, dz = (float)xt[2] - rzf;
            if (dx * dx + dy * dy + dz * dz < 1e-4f) {
              gi = (int)(w.off_k1[ai] + t);
              break;
            }
          }
          w.pr_g[q] = gi;
          if (pass == 0) pid[i * max_n1 + j] = slot;
        }
        pos += __popc(m);
      }
    }
    if (lane == 0) {
      w.prow[rbase + i] = rowstart[i];
      w.prow_k2[rbase + i] = rowstart[i] + rowk1[i];
    }
  }
  if (tid == 0) w.prow[rbase + n1] = rowstart[n1];
  __syncthreads();
  // phase 2b: FP64 geometry and damping of every pair, one thread per pair
  for (int t = tid; t < rowstart[n1]; t += blockDim.x) {
    const long long q = offp + t;
    const int i = w.pr_ij[2 * q], j = w.pr_ij[2 * q + 1];
    double rx, ry, rz, r2;
    scs_pair_in(xs, max_n12, i, j, rc2, rx, ry, rz, r2);
    // 1/r from one reciprocal square root; the Fermi damping (Eq. damping-function) through
    // x = r / S_vdW, its r-derivative f (1 - f) d / S_vdW as f (1 - f) d x / r
    const double ir = rsqrt(r2);
    const double r = r2 * ir;
    const int ai = w.site_atom[sbase + i], aj = w.site_atom[sbase + j];
    double fsr, dfsr, fin = 1.0, dfin = 0.0;
    cutoff_buf(r, p.r_scs, p.r_buf, fsr, dfsr);
    if (j >= n1) finner(r, p.r_inner, fin, dfin);
    const double x = r / (p.beta * (w.rvdw[ai] + w.rvdw[aj]));
    const double f = 1.0 / (1.0 + exp(-p.d * (x - 1.0)));
    const double dfr = f * (1.0 - f) * p.d * x * ir;
    const double F = fin * fsr * (1.0 - f);
    const double dF = dfin * fsr * (1.0 - f) + fin * dfsr * (1.0 - f) - fin * fsr * dfr;
    double* g = w.pr_geo + 8 * q;
    g[0] = rx; g[1] = ry; g[2] = rz; g[3] = r; g[4] = F; g[5] = dF; g[6] = ir; g[7] = 0.0;
    float2* gf = w.pr_gff + 6 * q;
#pragma unroll
    for (int u = 0; u < 7; ++u) {
      if (u == 3) continue;
      const ff v = ff_from_double(g[u]);
      gf[u < 3 ? u : u - 1] = make_float2(v.hi, v.lo);
    }
  }
  __syncthreads();
  // phase 3: adjacency rows (K1 partners of every coupled site, both directions)
  for (int i = warp; i < n1; i += nw) {
    int k = 0;
    for (int j0 = 0; j0 < n1; j0 += 32) {
      int j = j0 + lane;
      bool in = j < n1 && j != i && (j < i ? pid[i * max_n1 + j] : pid[j * max_n1 + i]) >= 0;
      k += __popc(__ballot_sync(0xffffffffu, in));
    }
    if (lane == 0) adjcnt[i] = k;
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int i = 0; i < n1; ++i) { adjstart[i] = run; run += adjcnt[i]; }
    adjstart[n1] = run;
  }
  __syncthreads();
  for (int i = warp; i < n1; i += nw) {
    int pos = adjstart[i];
    for (int j0 = 0; j0 < n1; j0 += 32) {
      int j = j0 + lane;
      int pp = -1;
      if (j < n1 && j != i) pp = j < i ? pid[i * max_n1 + j] : pid[j * max_n1 + i];
      unsigned m = __ballot_sync(0xffffffffu, pp >= 0);
      if (pp >= 0) {
        long long q = offa + pos + __popc(m & ((1u << lane) - 1u));
        w.adj[2 * q] = j;
        w.adj[2 * q + 1] = pp;
      }
      pos += __popc(m);
    }
    if (lane == 0) w.arow[rbase + i] = adjstart[i];
  }
  if (tid == 0) w.arow[rbase + n1] = adjstart[n1];
  // phase 4: for every K2 site the pairs in which it is the partner (rows ascending)
  if (tid < 32) {
    for (int j = n1 + lane; j < n12; j += 32) k2cnt[j] = 0;
    __syncwarp();
    for (int i = 0; i < n1; ++i) {
      const int b = rowstart[i] + rowk1[i], e = rowstart[i + 1];
      for (int t = b + lane; t < e; t += 32) ++k2cnt[w.pr_ij[2 * (offp + t) + 1]];
      __syncwarp();
    }
    if (lane == 0) {
      int run = 0;
      for (int j = n1; j < n12; ++j) {
        int cj = k2cnt[j];
        w.k2ptr[sbase + j] = run;
        k2cnt[j] = run;
        run += cj;
      }
      w.k2ptr[sbase + n12] = run;
    }
    __syncwarp();
    for (int i = 0; i < n1; ++i) {
      const int b = rowstart[i] + rowk1[i], e = rowstart[i + 1];
      for (int t = b + lane; t < e; t += 32) {
        const int j = w.pr_ij[2 * (offp + t) + 1];
        w.k2rev[offp + k2cnt[j]] = t;
        ++k2cnt[j];
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------------------
// FP32 Cholesky and triangular solves on a packed lower triangle in shared memory
// (whole thread block of 256 threads; 16-wide blocks; 3 right-hand sides)
// ---------------------------------------------------------------------------------------
#define CB 16
#define CBP (CB * (CB + 1) / 2)   // packed lower triangle of one diagonal-block inverse
__device__ __forceinline__ int pidx16(int i, int j) { return i * (i + 1) / 2 + j; }

// The 16 x 16 diagonal block at k0, one warp: right-looking Cholesky in registers (one row per
// lane, rows beyond the block hold the identity; one reciprocal square root per pivot, so
// sinv[i] = 1/L_ii is that reciprocal), then the inverse of the factor block, one column per
// lane, into binv (packed lower triangle).  A non-positive pivot sets *bad.
__device__ void chol32_diag(float* A, int n, int k0, int* bad, float* sinv, float* binv) {
  const int lane = threadIdx.x & 31;
  const int kb = min(CB, n - k0);
  const bool act = lane < kb;
  float a[CB];
#pragma unroll
  for (int u = 0; u < CB; ++u)
    a[u] = act ? (u <= lane ? A[packed_idx(k0 + lane, k0 + u)] : 0.f) : (u == lane ? 1.f : 0.f);
  bool fail = false;
  float il_own = 1.f;
#pragma unroll
  for (int t = 0; t < CB; ++t) {
    float d = __shfl_sync(0xffffffffu, a[t], t);
    if (t < kb && !(d > 0.f)) {
      fail = true;
      d = 1.f;
    }
    const float il = rsqrtf(d), l = d * il;
    if (lane == t) {
      a[t] = l;
      il_own = il;
    } else if (lane > t) {
      a[t] *= il;
    }
#pragma unroll
    for (int j = 1; j < CB; ++j) {
      if (j > t) {
        const float ljt = __shfl_sync(0xffffffffu, a[t], j);
        if (lane >= j) a[j] -= a[t] * ljt;
      }
    }
  }
  if (fail && lane == 0) *bad = 1;
#pragma unroll
  for (int u = 0; u < CB; ++u)
    if (act && u <= lane) A[packed_idx(k0 + lane, k0 + u)] = a[u];
  if (act) sinv[k0 + lane] = il_own;
  __syncwarp();
  // inverse of the factor block: lane c solves L x = e_c, reading L from shared memory
  // (every lane reads the same element: broadcast)
  float* inv = binv + (k0 / CB) * CBP;
  float x[CB];
#pragma unroll
  for (int i = 0; i < CB; ++i) {
    float v = 0.f;
    if (i < kb) {
      const float* Li = A + packed_idx(k0 + i, k0);
      float s = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int u = 0; u < i; ++u) s -= Li[u] * x[u];
      v = (i >= lane && act) ? s * sinv[k0 + i] : 0.f;
    }
    x[i] = v;
    if (lane < CB && i >= lane) inv[pidx16(i, lane)] = v;
  }
  __syncwarp();
}

// named barrier 1 between warp 0 (waits) and warp 1 (arrives): 64 threads
__device__ __forceinline__ void nbar_sync_w01() { asm volatile("bar.sync 1, 64;" ::: "memory"); }
__device__ __forceinline__ void nbar_arrive_w01() { asm volatile("bar.arrive 1, 64;" ::: "memory"); }

// Right-looking blocked Cholesky of the packed lower triangle (16-wide blocks, 256 threads),
// with lookahead.  Per block column k: all threads form the panel rows below the diagonal block
// from the inverse diagonal block (L_ik = A_ik L_kk^-T, independent dot products); then warp 1
// updates the next diagonal block first and hands it to warp 0 through a named barrier, warp 0
// factors and inverts it while warps 1..7 update the trailing rows below it, two rows per warp
// at a time (each panel value a lane loads serves both rows).  Two block barriers per block
// column; the factor of the next diagonal block is off the path of the trailing update.
// sinv[i] = 1/L_ii; binv holds the inverses of the diagonal blocks (solve32_warp).
__device__ __noinline__ void chol32_packed(float* A, int n, int* bad, float* sinv, float* binv) {
  constexpr int RB = 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  if (warp == 0) chol32_diag(A, n, 0, bad, sinv, binv);
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += CB) {
    const int kb = min(CB, n - k0), r0 = k0 + kb;
    if (r0 >= n) break;
    const float* inv = binv + (k0 / CB) * CBP;
    for (int i = r0 + tid; i < n; i += blockDim.x) {
      float* row = A + packed_idx(i, k0);
      float v[CB], o[CB];
#pragma unroll
      for (int t = 0; t < CB; ++t) v[t] = t < kb ? row[t] : 0.f;
#pragma unroll
      for (int t = 0; t < CB; ++t) {
        float sum = 0.f;
#pragma unroll
        for (int u = 0; u <= t; ++u) sum += v[u] * inv[pidx16(t, u)];
        o[t] = sum;
      }
#pragma unroll
      for (int t = 0; t < CB; ++t)
        if (t < kb) row[t] = o[t];
    }
    __syncthreads();
    const int k1 = r0, kb1 = min(CB, n - k1), r1 = k1 + kb1;
    if (warp == 0) {
      nbar_sync_w01();
      chol32_diag(A, n, k1, bad, sinv, binv);
    } else {
      if (warp == 1) {
        // the next diagonal block: lane l takes row l % 16, the columns of parity l / 16
        const int i = lane & 15;
        if (i < kb1) {
          const float* li = A + packed_idx(k1 + i, k0);
          float a[CB];
#pragma unroll
          for (int t = 0; t < CB; ++t) a[t] = t < kb ? li[t] : 0.f;
          for (int j = lane >> 4; j <= i; j += 2) {
            const float* lj = A + packed_idx(k1 + j, k0);
            float sum = 0.f;
#pragma unroll
            for (int t = 0; t < CB; ++t)
              if (t < kb) sum += a[t] * lj[t];
            A[packed_idx(k1 + i, k1 + j)] -= sum;
          }
        }
        __threadfence_block();
        nbar_arrive_w01();
      }
      for (int i0 = r1 + RB * (warp - 1); i0 < n; i0 += RB * (nw - 1)) {
        float a[RB][CB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const float* li = A + packed_idx(min(i0 + r, n - 1), k0);
#pragma unroll
          for (int t = 0; t < CB; ++t) a[r][t] = t < kb ? li[t] : 0.f;
        }
        const int ilast = min(i0 + RB - 1, n - 1);
        for (int j = k1 + lane; j <= ilast; j += 32) {
          const float* lj = A + packed_idx(j, k0);
          float sum[RB];
#pragma unroll
          for (int r = 0; r < RB; ++r) sum[r] = 0.f;
#pragma unroll
          for (int t = 0; t < CB; ++t) {
            const float v = t < kb ? lj[t] : 0.f;
#pragma unroll
            for (int r = 0; r < RB; ++r) sum[r] += a[r][t] * v;
          }
#pragma unroll
          for (int r = 0; r < RB; ++r)
            if (j <= i0 + r && i0 + r < n) A[packed_idx(i0 + r, j)] -= sum[r];
        }
      }
    }
    __syncthreads();
  }
}

// y (n x 3, FP32, shared) <- (L L^T)^-1 y with binv the inverses of the 16 x 16 diagonal blocks,
// a blocked substitution with one warp per right-hand side column: warps 0..2 each solve their
// column with warp-level
// synchronisation only (a block row: half-warp partial sums of its 16 rows over the solved part,
// combined across the halves with a shuffle, then the product with the inverse diagonal block by
// shuffles), so the substitution needs no block barrier; z (n x 3) is scratch.  The caller's
// writes to y must be visible (a block barrier before); the result is visible after the final one.
__device__ void solve32_warp(const float* L, int n, const float* binv, float* y, float* z) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 3) {
    const int c = warp, r = lane & 15, h = lane >> 4;
    // forward: z = L^-1 y
    for (int b0 = 0; b0 < n; b0 += CB) {
      const int bb = min(CB, n - b0);
      const float* inv = binv + (b0 / CB) * CBP;
      float t = 0.f;
      if (r < bb) {
        const float* row = L + packed_idx(b0 + r, 0);
        for (int k = h; k < b0; k += 2) t += row[k] * z[3 * k + c];
      }
      t += __shfl_xor_sync(0xffffffffu, t, 16);
      const float v = r < bb ? y[3 * (b0 + r) + c] - t : 0.f;
      float acc = 0.f;
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const float vu = __shfl_sync(0xffffffffu, v, u);
        if (u <= r && r < bb) acc += inv[pidx16(r, u)] * vu;
      }
      if (h == 0 && r < bb) z[3 * (b0 + r) + c] = acc;
      __syncwarp();
    }
    // backward: y = L^-T z
    const int nblk = (n + CB - 1) / CB;
    for (int blk = nblk - 1; blk >= 0; --blk) {
      const int b0 = blk * CB, bb = min(CB, n - b0), b1 = b0 + bb;
      const float* inv = binv + blk * CBP;
      float t = 0.f;
      if (r < bb)
        for (int k = b1 + h; k < n; k += 2) t += L[packed_idx(k, b0 + r)] * y[3 * k + c];
      t += __shfl_xor_sync(0xffffffffu, t, 16);
      const float v = r < bb ? z[3 * (b0 + r) + c] - t : 0.f;
      float acc = 0.f;
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const float vu = __shfl_sync(0xffffffffu, v, u);
        if (u >= r && u < bb) acc += inv[pidx16(u, r)] * vu;
      }
      if (h == 0 && r < bb) y[3 * (b0 + r) + c] = acc;
      __syncwarp();
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// shared memory of the per-(atom, frequency) kernels
// ---------------------------------------------------------------------------------------
struct Scs2Smem {
  float* A;       // packed lower factor, N1 (N1 + 1) / 2
  float* sinv;    // N1
  float* binv;    // ceil(N1/16) x 136: inverses of the diagonal blocks (packed lower)
  float* y;       // N1 x 3 (FP32 right-hand side / correction)
  float* z;       // N1 x 3 (FP32 scratch of the triangular solves)
  double* rhs;    // N1 x 3 (FP64 right-hand side d or dL/dX)
  double* x;      // N1 x 3 (FP64 solution X or lambda)
  double* xs;     // N1 x 3 (adjoint: X of the forward solve)
  ff* abf;        // n12 (alpha_bar at this frequency, float-float)
  double* iab;    // n1 (1 / alpha_bar of the coupled sites)
  double* red;    // 64
};

__host__ __device__ inline size_t scs2_smem_bytes(int max_n1, int max_n12, bool adjoint) {
  size_t N1 = 3 * (size_t)max_n1;
  size_t fl = N1 * (N1 + 1) / 2 + N1 + 6 * N1 + (N1 + 15) / 16 * CBP;
  fl = (fl + 1) & ~size_t(1);
  size_t dd = 2 * 3 * N1 + (size_t)max_n12 + (size_t)max_n1 + 64;
  if (adjoint) dd += 3 * N1;
  return fl * sizeof(float) + dd * sizeof(double);
}

__device__ inline Scs2Smem scs2_carve(unsigned char* base, int max_n1, int max_n12, bool adjoint) {
  Scs2Smem s;
  size_t N1 = 3 * (size_t)max_n1;
  s.A = (float*)base;
  s.sinv = s.A + N1 * (N1 + 1) / 2;
  s.y = s.sinv + N1;
  s.z = s.y + 3 * N1;
  s.binv = s.z + 3 * N1;
  size_t fl = N1 * (N1 + 1) / 2 + N1 + 6 * N1 + (N1 + 15) / 16 * CBP;
  fl = (fl + 1) & ~size_t(1);
  double* d = (double*)(base + fl * sizeof(float));
  s.rhs = d;
  s.x = s.rhs + 3 * N1;
  s.abf = reinterpret_cast<ff*>(s.x + 3 * N1);      // one ff per site: 8 bytes, as a double
  s.iab = reinterpret_cast<double*>(s.abf + max_n12);
  s.red = s.iab + max_n1;
  s.xs = adjoint ? s.red + 64 : nullptr;
  return s;
}

// rhs <- rhs - B y for the FP32 vector y, in float-float arithmetic on the FP32 pipe (B from the
// float-float tables: 1/alpha_bar on the diagonal, F A0 delta + F B0 r r^T per K1 pair).  Called
// with the FP32 solution x0 = y it forms the residual d - B x0 (error ~2^-46 |B| |x0|, so the
// refined solution carries a relative error ~cond(B) 2^-46); called with a correction delta
// (~1e-7 of x) it updates the residual of x + delta to FP64 rounding.
__device__ void scs2_residual_update(const Work& w, const DevParams& p, int n1, long long offp, long long offa,
                                     long long rbase, int q, Scs2Smem& sm) {
  // two threads per (coupled site i, right-hand side c), neighbouring lanes, each summing half of
  // the adjacency row; the halves are combined with a shuffle in a fixed order
  const int items = 6 * n1;
  for (int base = 0; base < items; base += blockDim.x) {
    const int e = base + threadIdx.x;
    const bool act = e < items;
    const int i = act ? e / 6 : 0, c = act ? (e >> 1) % 3 : 0, half = e & 1;
    ff a0 = ff_make(0.f, 0.f), a1 = a0, a2 = a0;
    if (act) {
      if (half == 0) {
        const ff ia = ff_from_double(sm.iab[i]);
        a0 = ff_scale(ia, sm.y[9 * i + c]);
        a1 = ff_scale(ia, sm.y[9 * i + 3 + c]);
        a2 = ff_scale(ia, sm.y[9 * i + 6 + c]);
      }
      const int b0 = w.arow[rbase + i], en0 = w.arow[rbase + i + 1];
      const int mid = b0 + (en0 - b0 + 1) / 2;
      const int b = half == 0 ? b0 : mid, en = half == 0 ? mid : en0;
      for (int t = b; t < en; ++t) {
        const int j = w.adj[2 * (offa + t)];
        const long long pq = offp + w.adj[2 * (offa + t) + 1];
        const float2* gf = w.pr_gff + 6 * pq;
        const float2* rf = w.pr_rad_ff + 2 * (pq * p.nqs + q);
        const ff rx = ff_make(gf[0].x, gf[0].y), ry = ff_make(gf[1].x, gf[1].y), rz = ff_make(gf[2].x, gf[2].y);
        const ff fa = ff_make(rf[0].x, rf[0].y), fb = ff_make(rf[1].x, rf[1].y);
        const float d0 = sm.y[9 * j + c], d1 = sm.y[9 * j + 3 + c], d2 = sm.y[9 * j + 6 + c];
        const ff bu = ff_mul(fb, ff_add(ff_add(ff_scale(rx, d0), ff_scale(ry, d1)), ff_scale(rz, d2)));
        a0 = ff_add(a0, ff_add(ff_scale(fa, d0), ff_mul(bu, rx)));
        a1 = ff_add(a1, ff_add(ff_scale(fa, d1), ff_mul(bu, ry)));
        a2 = ff_add(a2, ff_add(ff_scale(fa, d2), ff_mul(bu, rz)));
      }
    }
    const ff o0 = ff_make(__shfl_xor_sync(0xffffffffu, a0.hi, 1), __shfl_xor_sync(0xffffffffu, a0.lo, 1));
    const ff o1 = ff_make(__shfl_xor_sync(0xffffffffu, a1.hi, 1), __shfl_xor_sync(0xffffffffu, a1.lo, 1));
    const ff o2 = ff_make(__shfl_xor_sync(0xffffffffu, a2.hi, 1), __shfl_xor_sync(0xffffffffu, a2.lo, 1));
    if (act && half == 0) {
      sm.rhs[9 * i + c] -= ff_to_double(ff_add(a0, o0));
      sm.rhs[9 * i + 3 + c] -= ff_to_double(ff_add(a1, o1));
      sm.rhs[9 * i + 6 + c] -= ff_to_double(ff_add(a2, o2));
    }
  }
}

// x = B^-1 rhs: FP32 solve, then FP64 refinement until the predicted error is below
// rel_tol |x|: the residual is formed once in FP64 and then updated by the corrections (rhs is
// overwritten).  Returns the number of corrections; *fail set if it does not converge.
// rel_tol = 2^-52 for the forward solve (alpha_K and alpha_I to FP64 accuracy); the adjoint
// solve, whose lambda only feeds the forces (1e-8 eV/A tolerance; a relative error of 1e-9 in
// lambda moves them by ~1e-11 eV/A), stops at 2^-30 and may stop after the first correction on
// an a-priori contraction estimate (below).
__device__ int scs2_refine(const Work& w, const DevParams& p, int n1, long long offp, long long offa,
                           long long rbase, int q, Scs2Smem& sm, int* fail, double rel_tol) {
  const int N1 = 3 * n1, tid = threadIdx.x;
  for (int e = tid; e < 3 * N1; e += blockDim.x) sm.y[e] = (float)sm.rhs[e];
  __syncthreads();
  solve32_warp(sm.A, N1, sm.binv, sm.y, sm.z);
  for (int e = tid; e < 3 * N1; e += blockDim.x) sm.x[e] = (double)sm.y[e];
  __syncthreads();
  // the residual d - B x0 of the FP32 solution x0 = y, in float-float arithmetic on the FP32
  // pipe (kept in rhs), then updated by -B delta per correction the same way
  scs2_residual_update(w, p, n1, offp, offa, rbase, q, sm);
  __syncthreads();
  for (int e = tid; e < 3 * N1; e += blockDim.x) sm.y[e] = (float)sm.rhs[e];
  __syncthreads();
  double prev = 0.0;
  int it = 0;
  for (; it < 12; ++it) {
    solve32_warp(sm.A, N1, sm.binv, sm.y, sm.z);
    double dmax = 0.0, xmax = 0.0;
    for (int e = tid; e < 3 * N1; e += blockDim.x) {
      double dlt = (double)sm.y[e];
      double xn = sm.x[e] + dlt;
      sm.x[e] = xn;
      dmax = fmax(dmax, fabs(dlt));
      xmax = fmax(xmax, fabs(xn));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if ((tid & 31) == 0) { sm.red[tid >> 5] = dmax; sm.red[32 + (tid >> 5)] = xmax; }
    __syncthreads();
    dmax = 0.0;
    xmax = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      dmax = fmax(dmax, sm.red[k]);
      xmax = fmax(xmax, sm.red[32 + k]);
    }
    __syncthreads();
    // contraction estimate rho = |delta_k| / |delta_{k-1}|; stop when rho |delta_k| is negligible.
    // With the looser adjoint tolerance the first correction already gives an estimate: the
    // FP32 solution's relative error, i.e. |delta_0| / |x|, is the contraction factor of the
    // iteration (error_0 = (M^-1 - B^-1) d with M = L L^T), so the error left after it is about
    // (|delta_0| / |x|) |delta_0|; a margin of 10 on that
    const double tol = rel_tol * xmax;
    if (dmax <= tol) { ++it; break; }
    if (it == 0 && rel_tol > 1e-15 && 10.0 * (dmax / xmax) * dmax <= tol) { ++it; break; }
    if (it >= 1) {
      double rho = prev > 0.0 ? dmax / prev : 1.0;
      if (rho < 0.5 && rho * dmax <= tol) { ++it; break; }
    }
    prev = dmax;
    if (it == 11 && tid == 0) *fail = 1;
    scs2_residual_update(w, p, n1, offp, offa, rbase, q, sm);
    __syncthreads();
    for (int e = tid; e < 3 * N1; e += blockDim.x) sm.y[e] = (float)sm.rhs[e];
    __syncthreads();
  }
  return it;
}

// Radial terms of T_SR (see lmbd_internal.cuh): A0 = g/r^3, B0 = (h~ - 3g)/r^5 and their
// r-derivatives, with x = r / sigma_ij.  For x >= 8, erf(x) = 1 and x^3 exp(-x^2) < 1e-25 in
// double precision, so g = 1 and h~ = 0 exactly; the transcendental calls are skipped there.
__device__ __forceinline__ void tsr_radial_fast(double r, double ir, double s2, double& A0, double& B0,
                                                double& dA0, double& dB0) {
  const double x = r * rsqrt(s2);
  double g = 1.0, ht = 0.0;
  if (x < 8.0) {
    const double two_over_sqrtpi = 1.1283791670955126;
    const double ex = exp(-x * x);
    g = erf(x) - two_over_sqrtpi * x * ex;
    ht = 2.0 * two_over_sqrtpi * x * x * x * ex;
  }
  const double ir2 = ir * ir, ir3 = ir2 * ir, ir4 = ir2 * ir2;
  A0 = g * ir3;
  B0 = (ht - 3.0 * g) * ir4 * ir;
  dA0 = (ht - 3.0 * g) * ir4;
  dB0 = (15.0 * g - 5.0 * ht - 2.0 * x * x * ht) * ir4 * ir2;
}

// Radial terms per atom pair and frequency: for atom a and every site s (1 <= s < n1) of its
// own K1 list, A0, B0 and their r-derivatives at sigma_ab(omega_q).  They depend on |r_ab|
// and sigma_a, sigma_b only, so every central atom whose local system holds the pair reads
// them instead of evaluating erf and exp again (about 50 local systems share each pair).
__global__ void __launch_bounds__(128) k_pair_radial(Work w, DevParams p) {
  const int a = blockIdx.x;
  if (a >= w.n_atoms) return;
  const int n1 = w.counts[a].n1;
  const long long ab = (long long)a * w.site_cap, base = w.off_k1[a];
  for (int e = threadIdx.x; e < n1 * p.nqs; e += blockDim.x) {
    const int s = e / p.nqs, q = e % p.nqs;
    if (s == 0) continue;
    const double* x = w.site_x + 3 * (ab + s);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x[0], x[0]), __dmul_rn(x[1], x[1])), __dmul_rn(x[2], x[2]));
    const double r = sqrt(r2);
    const int b = w.site_atom[ab + s];
    const double sa = w.sig[(long long)a * p.nqs + q], sb = w.sig[(long long)b * p.nqs + q];
    double A0, B0, dA0, dB0;
    tsr_radial_fast(r, 1.0 / r, sa * sa + sb * sb, A0, B0, dA0, dB0);
    const long long o = (base + s) * p.nqs + q;
    w.rad_ab[2 * o] = A0;
    w.rad_ab[2 * o + 1] = B0;
    const double v[4] = {A0, B0, dA0, dB0};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const ff t = ff_from_double(v[u]);
      w.rad_ff[4 * o + u] = make_float2(t.hi, t.lo);
    }
  }
}

// ---------------------------------------------------------------------------------------
// pieces shared by the Cholesky kernels and the LU fallback
// ---------------------------------------------------------------------------------------
// alpha_bar of every site at SCS frequency q, and 1/alpha_bar of the coupled sites
__device__ __forceinline__ void scs2_load_abar(const Work& w, const DevParams& p, int c, int q, int n1, int n12, Scs2Smem& sm) {
  const long long sbase = (long long)c * w.site_cap;
  for (int s = threadIdx.x; s < n12; s += blockDim.x) {
    int a = w.site_atom[sbase + s];
    const double ab = w.abar[(long long)a * p.nqs + q];
    sm.abf[s] = ff_from_double(ab);
    if (s < n1) sm.iab[s] = 1.0 / ab;
  }
}

// right-hand side d_i = 1 - sum_{j in K2} T_SR,ij alpha_bar_j (Eq. local_pol) in float-float
// arithmetic on the FP32 pipe (fixed order, ~2^-46 relative), rounded to FP64; one thread per
// (coupled site i, column c): column c of T_SR,ij is F A0 e_c + F B0 r r_c.  rhs is N1 x 3
// row-major (row 3 i + alpha).  Needs the float-float radial terms of this frequency.
__device__ __forceinline__ void scs2_build_rhs(const Work& w, const DevParams& p, int n1, long long offp,
                                               long long rbase, int q, const ff* abf, double* rhs) {
  for (int e = threadIdx.x; e < 3 * n1; e += blockDim.x) {
    const int i = e / 3, c = e % 3;
    ff a0 = ff_make(0.f, 0.f), a1 = a0, a2 = a0, ad = a0;
    const int b = w.prow_k2[rbase + i], en = w.prow[rbase + i + 1];
    for (int t = b; t < en; ++t) {
      const long long pq = offp + t;
      const int j = w.pr_ij[2 * pq + 1];
      const float2* gf = w.pr_gff + 6 * pq;
      const float2* rf = w.pr_rad_ff + 2 * (pq * p.nqs + q);
      const ff rx = ff_make(gf[0].x, gf[0].y), ry = ff_make(gf[1].x, gf[1].y), rz = ff_make(gf[2].x, gf[2].y);
      const ff rc = c == 0 ? rx : (c == 1 ? ry : rz);
      const ff abj = abf[j];
      ad = ff_fma(abj, ff_make(rf[0].x, rf[0].y), ad);
      const ff wb = ff_mul(ff_mul(abj, ff_make(rf[1].x, rf[1].y)), rc);
      a0 = ff_fma(wb, rx, a0);
      a1 = ff_fma(wb, ry, a1);
      a2 = ff_fma(wb, rz, a2);
    }
    if (c == 0) a0 = ff_add(a0, ad);
    if (c == 1) a1 = ff_add(a1, ad);
    if (c == 2) a2 = ff_add(a2, ad);
    double* y = rhs + 9 * i;
    y[c] = (c == 0 ? 1.0 : 0.0) - ff_to_double(a0);
    y[3 + c] = (c == 1 ? 1.0 : 0.0) - ff_to_double(a1);
    y[6 + c] = (c == 2 ? 1.0 : 0.0) - ff_to_double(a2);
  }
}

// FP64 damped radial terms F A0, F B0 of pair pq at SCS frequency q (LU fallback): from the
// atom-pair table, or evaluated when the pair has no table entry
__device__ __forceinline__ void pair_rad64(const Work& w, const DevParams& p, int c, int q, long long pq, double& fa,
                                           double& fb) {
  const double* g = w.pr_geo + 8 * pq;
  const int gi = w.pr_g[pq];
  double A0, B0;
  if (gi >= 0) {
    const double* ra = w.rad_ab + 2 * ((long long)gi * p.nqs + q);
    A0 = ra[0];
    B0 = ra[1];
  } else {
    const long long sbase = (long long)c * w.site_cap;
    const int i = w.pr_ij[2 * pq], j = w.pr_ij[2 * pq + 1];
    const double si = w.sig[(long long)w.site_atom[sbase + i] * p.nqs + q];
    const double sj = w.sig[(long long)w.site_atom[sbase + j] * p.nqs + q];
    double dA0, dB0;
    tsr_radial_fast(g[3], g[6], si * si + sj * sj, A0, B0, dA0, dB0);
  }
  fa = g[4] * A0;
  fb = g[4] * B0;
}

// the right-hand side of Eq. local_pol in FP64 (LU fallback), alpha_bar from global memory
__device__ void scs2_build_rhs64(const Work& w, const DevParams& p, int c, int n1, int q, double* rhs) {
  const long long offp = w.off_p[c], rbase = w.off_k1[c] + c, sbase = (long long)c * w.site_cap;
  for (int e = threadIdx.x; e < 3 * n1; e += blockDim.x) {
    const int i = e / 3, cc = e % 3;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, ad = 0.0;
    const int b = w.prow_k2[rbase + i], en = w.prow[rbase + i + 1];
    for (int t = b; t < en; ++t) {
      const long long pq = offp + t;
      const int j = w.pr_ij[2 * pq + 1];
      const double* g = w.pr_geo + 8 * pq;
      double fa, fb;
      pair_rad64(w, p, c, q, pq, fa, fb);
      const double abj = w.abar[(long long)w.site_atom[sbase + j] * p.nqs + q];
      ad += abj * fa;
      const double wb = abj * fb * g[cc];
      a0 += wb * g[0];
      a1 += wb * g[1];
      a2 += wb * g[2];
    }
    double* y = rhs + 9 * i;
    y[cc] = (cc == 0 ? 1.0 : 0.0) - a0 - (cc == 0 ? ad : 0.0);
    y[3 + cc] = (cc == 1 ? 1.0 : 0.0) - a1 - (cc == 1 ? ad : 0.0);
    y[6 + cc] = (cc == 2 ? 1.0 : 0.0) - a2 - (cc == 2 ? ad : 0.0);
  }
}

// X (N1 x 3), alpha_K,i = Tr(X_i)/3 and alpha_I,c = alpha_K,0 of one (centre, frequency)
__device__ __forceinline__ void scs2_store_solution(const Work& w, const DevParams& p, int c, int q, int n1, const double* x) {
  const int N1 = 3 * n1;
  const long long offk1 = w.off_k1[c];
  double* X = w.xsol + offk1 * p.nqs * 9 + (long long)q * N1 * 3;
  for (int e = threadIdx.x; e < N1 * 3; e += blockDim.x) X[e] = x[e];
  for (int i = threadIdx.x; i < n1; i += blockDim.x) {
    double a = (x[9 * i + 0] + x[9 * i + 4] + x[9 * i + 8]) / 3.0;
    w.alphaK[(offk1 + i) * p.nqs + q] = a;
    if (i == 0) w.alphaI[(long long)c * p.nqs + q] = a;
  }
}

// ---------------------------------------------------------------------------------------
// forward: one block per (central atom, frequency)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3) k_scs_factor(Work w, DevParams p, const int* order, int c0, int max_n1,
                                                  int max_n12) {
  extern __shared__ unsigned char smem_raw[];
  const int c = order ? order[c0 + blockIdx.x / p.nqs] : c0 + blockIdx.x / p.nqs;
  const int q = blockIdx.x % p.nqs;
  if (c >= w.n_atoms) return;
  const Counts cn = w.counts[c];
  const int n1 = cn.n1, n12 = cn.n12, N1 = 3 * n1;
  Scs2Smem sm = scs2_carve(smem_raw, max_n1, max_n12, false);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const long long sbase = (long long)c * w.site_cap;
  const long long offp = w.off_p[c], offa = w.off_a[c], rbase = w.off_k1[c] + c;
  const int np = w.prow[rbase + n1];
  __shared__ int bad, fail;
  if (tid == 0) { bad = 0; fail = 0; }
  scs2_load_abar(w, p, c, q, n1, n12, sm);
  const long long nA = (long long)N1 * (N1 + 1) / 2;
  for (long long e = tid; e < nA; e += blockDim.x) sm.A[e] = 0.f;
  __syncthreads();
  // damped radial terms F A0, F B0 of every pair at this frequency in float-float (F times the
  // atom-pair table entry, on the FP32 pipe), stored for the residuals and the adjoint, and the
  // K1 blocks of B in FP32 (the factor needs FP32 values only)
  for (int t = tid; t < np; t += blockDim.x) {
    const long long pq = offp + t;
    const int i = w.pr_ij[2 * pq], j = w.pr_ij[2 * pq + 1];
    const int gi = w.pr_g[pq];
    const float2* gf = w.pr_gff + 6 * pq;
    ff fa, fb;
    if (gi >= 0) {
      const float2* ra = w.rad_ff + 4 * ((long long)gi * p.nqs + q);
      const ff F = ff_make(gf[3].x, gf[3].y);
      fa = ff_mul(F, ff_make(ra[0].x, ra[0].y));
      fb = ff_mul(F, ff_make(ra[1].x, ra[1].y));
    } else {   // no table entry (a distance that ties r_SCS to rounding): evaluate in FP64
      double da, db;
      pair_rad64(w, p, c, q, pq, da, db);
      fa = ff_from_double(da);
      fb = ff_from_double(db);
    }
    float2* rf = w.pr_rad_ff + 2 * (pq * p.nqs + q);
    rf[0] = make_float2(fa.hi, fa.lo);
    rf[1] = make_float2(fb.hi, fb.lo);
    if (j < n1) {
      const float rr[3] = {gf[0].x, gf[1].x, gf[2].x};
#pragma unroll
      for (int al = 0; al < 3; ++al) {
        float* row = sm.A + packed_idx(3 * i + al, 3 * j);
#pragma unroll
        for (int be = 0; be < 3; ++be) row[be] = fb.hi * rr[al] * rr[be] + (al == be ? fa.hi : 0.f);
      }
    }
  }
  for (int i = tid; i < n1; i += blockDim.x)
#pragma unroll
    for (int al = 0; al < 3; ++al) sm.A[packed_idx(3 * i + al, 3 * i + al)] = (float)sm.iab[i];
  __threadfence_block();
  __syncthreads();
  scs2_build_rhs(w, p, n1, offp, rbase, q, sm.abf, sm.rhs);
  __syncthreads();
  chol32_packed(sm.A, N1, &bad, sm.sinv, sm.binv);
  // a non-positive pivot (B_K not positive definite: Sec. III.A, polarisation catastrophe) or
  // a refinement that does not converge sends the system to the LU fallback (k_scs_lu_forward)
  if (!bad) scs2_refine(w, p, n1, offp, offa, rbase, q, sm, &fail, 2.220446049250313e-16);
  __syncthreads();
  if (bad || fail) {
    if (tid == 0) {
      w.fb_flag[(long long)c * p.nqs + q] = 1;
      const int e = atomicAdd(w.fb, 1);
      w.fb[1 + e] = c * p.nqs + q;
    }
    return;
  }
  if (tid == 0) w.fb_flag[(long long)c * p.nqs + q] = 0;
  // outputs: X, alpha_K, alpha_I and the FP32 factor for the adjoint
  scs2_store_solution(w, p, c, q, n1, sm.x);
  float* Lg = w.lfac + w.off_b[c] + (long long)q * nA;
  for (long long e = tid; e < nA; e += blockDim.x) Lg[e] = sm.A[e];
  // the inverses of the diagonal blocks as well, so that the adjoint need not form them again
  float* Bg = w.binvg + ((long long)c * p.nqs + q) * w.binv_slot;
  for (int e = tid; e < (N1 + CB - 1) / CB * CBP; e += blockDim.x) Bg[e] = sm.binv[e];
}

// Adjoint right-hand side dL/dX of one (centre, frequency) into sm.rhs (dL/dX_i = delta/3 times
// dL/dalpha_K,i, plus dL/dalpha_I,c on the centre's block), and the forward solution X into sm.xs.
__device__ __forceinline__ void scs2_load_adjoint_rhs(const Work& w, const DevParams& p, int c, int q, int n1, Scs2Smem& sm) {
  const int N1 = 3 * n1;
  const long long offk1 = w.off_k1[c];
  const double* X = w.xsol + offk1 * p.nqs * 9 + (long long)q * N1 * 3;
  for (int e = threadIdx.x; e < N1 * 3; e += blockDim.x) {
    sm.xs[e] = X[e];
    int row = e / 3, col = e % 3, i = row / 3, al = row % 3;
    double gval = 0.0;
    if (al == col) {
      gval = w.alphaK_bar[(offk1 + i) * p.nqs + q];
      if (i == 0) gval += w.alphaI_bar[(long long)c * p.nqs + q];
      gval *= (1.0 / 3.0);
    }
    sm.rhs[e] = gval;
  }
}

// Adjoint contraction of one (centre, frequency) given lambda = B^-1 dL/dX in sm.x and the
// forward solution X in sm.xs (both N1 x 3, FP64): per pair <M, dT_SR/dr> with
// M = -(lambda_i X_j^T + lambda_j X_i^T) (K1 pairs) or M = -alpha_bar_j lambda_i (K2 pairs),
// symmetrised; g = dL/dr_j = -dL/dr_i per pair, staged in global scratch (L2-resident), then
// summed per site in a fixed order.  The contraction runs in float-float arithmetic (ff.cuh,
// ~2^-46 relative) on the FP32 pipe: lambda and X are converted once per site, geometry and
// radial terms come converted from the tables.  sm.rhs and sm.xs are overwritten.
__device__ __forceinline__ void scs2_adjoint_contract(const Work& w, const DevParams& p, int c, int q, int n1, int n12, Scs2Smem& sm) {
  const int N1 = 3 * n1, tid = threadIdx.x;
  const long long sbase = (long long)c * w.site_cap;
  const long long offp = w.off_p[c], offa = w.off_a[c], rbase = w.off_k1[c] + c;
  const int np = w.prow[rbase + n1];
  ff* lf = reinterpret_cast<ff*>(sm.rhs);   // lambda, 9 n1 (rhs is no longer needed)
  ff* xf = reinterpret_cast<ff*>(sm.xs);    // X, 9 n1 (in place: one element per thread)
  for (int e = tid; e < N1 * 3; e += blockDim.x) {
    const double xv = sm.xs[e];
    lf[e] = ff_from_double(sm.x[e]);
    xf[e] = ff_from_double(xv);
  }
  __syncthreads();
  // pair gradients as float-float (the per-site sums below stay on the FP32 pipe)
  float2* gst = reinterpret_cast<float2*>(w.gstage) + (offp * p.nqs + (long long)q * np) * 3;
  for (int t = tid; t < np; t += blockDim.x) {
    const long long pq = offp + t;
    const int i = w.pr_ij[2 * pq], j = w.pr_ij[2 * pq + 1];
    const int gi = w.pr_g[pq];
    const ff* li = lf + 9 * i;
    ff M[6];
    if (j < n1) {
      const ff* lj = lf + 9 * j;
      const ff* xi = xf + 9 * i;
      const ff* xj = xf + 9 * j;
      ff Mf[3][3];
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
          ff s = ff_mul(li[3 * al], xj[3 * be]);
          s = ff_fma(lj[3 * al], xi[3 * be], s);
#pragma unroll
          for (int ga = 1; ga < 3; ++ga) {
            s = ff_fma(li[3 * al + ga], xj[3 * be + ga], s);
            s = ff_fma(lj[3 * al + ga], xi[3 * be + ga], s);
          }
          Mf[al][be] = ff_neg(s);
        }
      M[0] = Mf[0][0]; M[1] = Mf[1][1]; M[2] = Mf[2][2];
      M[3] = ff_scale(ff_add(Mf[0][1], Mf[1][0]), 0.5f);
      M[4] = ff_scale(ff_add(Mf[0][2], Mf[2][0]), 0.5f);
      M[5] = ff_scale(ff_add(Mf[1][2], Mf[2][1]), 0.5f);
    } else {
      const ff aj = ff_neg(sm.abf[j]);
      M[0] = ff_mul(aj, li[0]); M[1] = ff_mul(aj, li[4]); M[2] = ff_mul(aj, li[8]);
      M[3] = ff_scale(ff_mul(aj, ff_add(li[1], li[3])), 0.5f);
      M[4] = ff_scale(ff_mul(aj, ff_add(li[2], li[6])), 0.5f);
      M[5] = ff_scale(ff_mul(aj, ff_add(li[5], li[7])), 0.5f);
    }
    const float2* gf = w.pr_gff + 6 * pq;
    const ff rr[3] = {ff_make(gf[0].x, gf[0].y), ff_make(gf[1].x, gf[1].y), ff_make(gf[2].x, gf[2].y)};
    const ff F = ff_make(gf[3].x, gf[3].y), dF = ff_make(gf[4].x, gf[4].y), ir = ff_make(gf[5].x, gf[5].y);
    ff A0, B0, dA0, dB0;
    if (gi >= 0) {
      const float2* ra = w.rad_ff + 4 * ((long long)gi * p.nqs + q);
      A0 = ff_make(ra[0].x, ra[0].y); B0 = ff_make(ra[1].x, ra[1].y);
      dA0 = ff_make(ra[2].x, ra[2].y); dB0 = ff_make(ra[3].x, ra[3].y);
    } else {
      const double* g = w.pr_geo + 8 * pq;
      const double si = w.sig[(long long)w.site_atom[sbase + i] * p.nqs + q];
      const double sj = w.sig[(long long)w.site_atom[sbase + j] * p.nqs + q];
      double a0d, b0d, da0d, db0d;
      tsr_radial_fast(g[3], g[6], si * si + sj * sj, a0d, b0d, da0d, db0d);
      A0 = ff_from_double(a0d); B0 = ff_from_double(b0d); dA0 = ff_from_double(da0d); dB0 = ff_from_double(db0d);
    }
    const ff Mr[3] = {ff_fma(M[4], rr[2], ff_fma(M[3], rr[1], ff_mul(M[0], rr[0]))),
                      ff_fma(M[5], rr[2], ff_fma(M[1], rr[1], ff_mul(M[3], rr[0]))),
                      ff_fma(M[2], rr[2], ff_fma(M[5], rr[1], ff_mul(M[4], rr[0])))};
    const ff trM = ff_add(ff_add(M[0], M[1]), M[2]);
    const ff rMr = ff_fma(rr[2], Mr[2], ff_fma(rr[1], Mr[1], ff_mul(rr[0], Mr[0])));
    const ff phi = ff_fma(B0, rMr, ff_mul(A0, trM));
    const ff inner = ff_fma(dB0, rMr, ff_mul(dA0, trM));
    const ff radial = ff_mul(ff_fma(F, inner, ff_mul(dF, phi)), ir);
    const ff tang = ff_scale(ff_mul(F, B0), 2.0f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const ff g = ff_fma(tang, Mr[d], ff_mul(radial, rr[d]));
      gst[3 * t + d] = make_float2(g.hi, g.lo);
    }
  }
  __syncthreads();
  // per site (fixed order): owner of its row's pairs (-g), partner of K1 pairs owned by later
  // rows (+g, from the adjacency row) and of K2 pairs (+g, from the reverse list)
  double* sgq = w.sgq + (sbase * p.nqs + q) * 3;
  auto gld = [&](long long k) { const float2 v = gst[k]; return ff_make(v.x, v.y); };
  for (int s = tid; s < n12; s += blockDim.x) {
    ff gx = ff_make(0.f, 0.f), gy = gx, gz = gx;
    if (s < n1) {
      for (int t = w.prow[rbase + s]; t < w.prow[rbase + s + 1]; ++t) {
        gx = ff_sub(gx, gld(3 * t)); gy = ff_sub(gy, gld(3 * t + 1)); gz = ff_sub(gz, gld(3 * t + 2));
      }
      for (int t = w.arow[rbase + s]; t < w.arow[rbase + s + 1]; ++t) {
        const int j = w.adj[2 * (offa + t)], pp = w.adj[2 * (offa + t) + 1];
        if (j > s) { gx = ff_add(gx, gld(3 * pp)); gy = ff_add(gy, gld(3 * pp + 1)); gz = ff_add(gz, gld(3 * pp + 2)); }
      }
    } else {
      for (int t = w.k2ptr[sbase + s]; t < w.k2ptr[sbase + s + 1]; ++t) {
        const int pp = w.k2rev[offp + t];
        gx = ff_add(gx, gld(3 * pp)); gy = ff_add(gy, gld(3 * pp + 1)); gz = ff_add(gz, gld(3 * pp + 2));
      }
    }
    sgq[(long long)s * p.nqs * 3] = ff_to_double(gx);
    sgq[(long long)s * p.nqs * 3 + 1] = ff_to_double(gy);
    sgq[(long long)s * p.nqs * 3 + 2] = ff_to_double(gz);
  }
}

// ---------------------------------------------------------------------------------------
// adjoint: one block per (central atom, frequency)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3) k_scs_adjoint2(Work w, DevParams p, const int* order, int c0, int max_n1,
                                                  int max_n12) {
  extern __shared__ unsigned char smem_raw[];
  const int c = order ? order[c0 + blockIdx.x / p.nqs] : c0 + blockIdx.x / p.nqs;
  const int q = blockIdx.x % p.nqs;
  if (c >= w.n_atoms) return;
  if (w.fb_flag[(long long)c * p.nqs + q]) return;   // solved by the LU fallback (k_scs_lu_adjoint)
  const Counts cn = w.counts[c];
  const int n1 = cn.n1, n12 = cn.n12, N1 = 3 * n1;
  Scs2Smem sm = scs2_carve(smem_raw, max_n1, max_n12, true);
  const int tid = threadIdx.x;
  const long long offp = w.off_p[c], offa = w.off_a[c], rbase = w.off_k1[c] + c;
  __shared__ int fail;
  if (tid == 0) fail = 0;
  scs2_load_abar(w, p, c, q, n1, n12, sm);
  const long long nA = (long long)N1 * (N1 + 1) / 2;
  const float* Lg = w.lfac + w.off_b[c] + (long long)q * nA;
  for (long long e = tid; e < nA; e += blockDim.x) sm.A[e] = Lg[e];
  // the inverses of the diagonal blocks, as the factor kernel formed them (the solves need no more)
  const float* Bg = w.binvg + ((long long)c * p.nqs + q) * w.binv_slot;
  for (int e = tid; e < (N1 + CB - 1) / CB * CBP; e += blockDim.x) sm.binv[e] = Bg[e];
  __syncthreads();
  scs2_load_adjoint_rhs(w, p, c, q, n1, sm);
  __syncthreads();
  scs2_refine(w, p, n1, offp, offa, rbase, q, sm, &fail, 9.313225746154785e-10);   // lambda, 2^-30
  __syncthreads();
  scs2_adjoint_contract(w, p, c, q, n1, n12, sm);
  if (tid == 0 && fail) atomicOr(w.status, LMBD_FLAG_NOT_CONVERGED);
}

// ---------------------------------------------------------------------------------------
// LU fallback for screening matrices that are not positive definite (Sec. III.A: the
// polarisation catastrophe makes B_K indefinite) or on which the FP32-factor refinement does
// not converge.  Such systems are rare; each is solved in FP64 by Gaussian elimination with
// partial pivoting (row interchanges), the same factorisation a library dense solve uses, on
// the dense B_K assembled from the pair list into a per-block slot of global memory.  A pivot
// that is exactly zero (B_K singular) sets LMBD_FLAG_NOT_SPD.
// ---------------------------------------------------------------------------------------
// dense B_K (N1 x N1 row-major, FP64) of one (centre, frequency): diag(1/alpha_bar) plus the
// T_SR blocks of the K1 pairs (symmetric 3 x 3 blocks, F A0 delta + F B0 r r^T)
__device__ void scs2_dense_b(const Work& w, const DevParams& p, int c, int q, int n1, const Scs2Smem& sm, double* A) {
  const int N1 = 3 * n1;
  const long long offp = w.off_p[c], rbase = w.off_k1[c] + c;
  const int np = w.prow[rbase + n1];
  for (long long e = threadIdx.x; e < (long long)N1 * N1; e += blockDim.x) A[e] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < n1; i += blockDim.x)
    for (int al = 0; al < 3; ++al) A[(long long)(3 * i + al) * N1 + 3 * i + al] = sm.iab[i];
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    const long long pq = offp + t;
    const int i = w.pr_ij[2 * pq], j = w.pr_ij[2 * pq + 1];
    if (j >= n1) continue;
    const double* g = w.pr_geo + 8 * pq;
    double fa, fb;
    pair_rad64(w, p, c, q, pq, fa, fb);
    for (int al = 0; al < 3; ++al)
      for (int be = 0; be < 3; ++be) {
        const double v = fb * g[al] * g[be] + (al == be ? fa : 0.0);
        A[(long long)(3 * i + al) * N1 + 3 * j + be] = v;
        A[(long long)(3 * j + be) * N1 + 3 * i + al] = v;
      }
  }
  __syncthreads();
}

// In-place LU with partial pivoting of the N1 x N1 matrix A (global memory), whole block:
// P A = L U, L unit lower (below the diagonal), U upper; piv[k] = row swapped with row k.
// Returns (uniformly) false if a pivot is zero or not finite.
__device__ bool lu_factor_dense(double* A, int n, int* piv, double* redv, int* redi) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  __shared__ int ok_s, p_s;
  if (tid == 0) ok_s = 1;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // pivot: the largest |A[i][k]|, i >= k (ties to the lowest row)
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += blockDim.x) {
      const double v = fabs(A[(long long)i * n + k]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { redv[warp] = best; redi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = redv[0];
      int ix = redi[0];
      for (int u = 1; u < nw; ++u)
        if (redv[u] > b || (redv[u] == b && redi[u] < ix)) { b = redv[u]; ix = redi[u]; }
      p_s = ix;
      piv[k] = ix;
      if (!(b > 0.0) || !isfinite(b)) ok_s = 0;
    }
    __syncthreads();
    if (!ok_s) return false;
    const int pr = p_s;
    if (pr != k)
      for (int j = tid; j < n; j += blockDim.x) {
        const double t = A[(long long)k * n + j];
        A[(long long)k * n + j] = A[(long long)pr * n + j];
        A[(long long)pr * n + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / A[(long long)k * n + k];
    for (int i = k + 1 + tid; i < n; i += blockDim.x) A[(long long)i * n + k] *= inv;
    __syncthreads();
    const int m = n - k - 1;
    for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
      const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
      A[(long long)i * n + j] -= A[(long long)i * n + k] * A[(long long)k * n + j];
    }
    __syncthreads();
  }
  return true;
}

// b (n x 3 row-major, shared memory) <- A^-1 b with the factors of lu_factor_dense; warps 0..2
// take one column each (row sums split over the lanes)
__device__ void lu_solve3_dense(const double* A, int n, const int* piv, double* b) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp < 3) {
    const int c = warp;
    if (lane == 0)
      for (int k = 0; k < n; ++k)
        if (piv[k] != k) {
          const double t = b[3 * k + c];
          b[3 * k + c] = b[3 * piv[k] + c];
          b[3 * piv[k] + c] = t;
        }
    __syncwarp();
    for (int i = 0; i < n; ++i) {
      double sacc = 0.0;
      for (int j = lane; j < i; j += 32) sacc += A[(long long)i * n + j] * b[3 * j + c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) b[3 * i + c] -= sacc;
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
      double sacc = 0.0;
      for (int j = i + 1 + lane; j < n; j += 32) sacc += A[(long long)i * n + j] * b[3 * j + c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) b[3 * i + c] = (b[3 * i + c] - sacc) / A[(long long)i * n + i];
      __syncwarp();
    }
  }
  __syncthreads();
}

// Forward LU fallback: persistent over the listed (centre, frequency) systems, one dense slot
// of lu_slot doubles per block.
__global__ void __launch_bounds__(256) k_scs_lu_forward(Work w, DevParams p, int max_n1, int max_n12, int tally) {
  extern __shared__ unsigned char smem_raw[];
  Scs2Smem sm = scs2_carve(smem_raw, max_n1, max_n12, true);
  int* piv = reinterpret_cast<int*>(sm.A);
  int* redi = reinterpret_cast<int*>(sm.y);
  double* A = w.lu + (long long)blockIdx.x * w.lu_slot;
  const int count = w.fb[0];
  if (tally && blockIdx.x == 0 && threadIdx.x == 0 && count > 0) atomicAdd(w.status + 2, count);
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    const int id = w.fb[1 + e], c = id / p.nqs, q = id % p.nqs;
    const int n1 = w.counts[c].n1, n12 = w.counts[c].n12, N1 = 3 * n1;
    const long long offp = w.off_p[c], rbase = w.off_k1[c] + c;
    scs2_load_abar(w, p, c, q, n1, n12, sm);
    __syncthreads();
    scs2_build_rhs64(w, p, c, n1, q, sm.x);
    scs2_dense_b(w, p, c, q, n1, sm, A);
    if (!lu_factor_dense(A, N1, piv, sm.red, redi)) {
      if (threadIdx.x == 0) atomicOr(w.status, LMBD_FLAG_NOT_SPD);
      __syncthreads();
      continue;
    }
    lu_solve3_dense(A, N1, piv, sm.x);
    scs2_store_solution(w, p, c, q, n1, sm.x);
    __syncthreads();
  }
}

// Adjoint LU fallback for the listed systems of centres [c0, c1): B_K is factored again (it is
// symmetric, so lambda = B_K^-T dL/dX = B_K^-1 dL/dX), then the same pair contraction as the
// Cholesky path.
__global__ void __launch_bounds__(256) k_scs_lu_adjoint(Work w, DevParams p, int c0, int c1, int max_n1,
                                                         int max_n12) {
  extern __shared__ unsigned char smem_raw[];
  Scs2Smem sm = scs2_carve(smem_raw, max_n1, max_n12, true);
  int* piv = reinterpret_cast<int*>(sm.A);
  int* redi = reinterpret_cast<int*>(sm.y);
  double* A = w.lu + (long long)blockIdx.x * w.lu_slot;
  const int count = w.fb[0];
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    const int id = w.fb[1 + e], c = id / p.nqs, q = id % p.nqs;
    if (c < c0 || c >= c1) continue;
    const int n1 = w.counts[c].n1, n12 = w.counts[c].n12, N1 = 3 * n1;
    scs2_load_abar(w, p, c, q, n1, n12, sm);
    __syncthreads();
    scs2_dense_b(w, p, c, q, n1, sm, A);
    if (!lu_factor_dense(A, N1, piv, sm.red, redi)) {
      if (threadIdx.x == 0) atomicOr(w.status, LMBD_FLAG_NOT_SPD);
      __syncthreads();
      continue;
    }
    scs2_load_adjoint_rhs(w, p, c, q, n1, sm);
    for (int u = threadIdx.x; u < 3 * N1; u += blockDim.x) sm.x[u] = sm.rhs[u];
    __syncthreads();
    lu_solve3_dense(A, N1, piv, sm.x);
    scs2_adjoint_contract(w, p, c, q, n1, n12, sm);
    __syncthreads();
  }
}

// Sum of the per-frequency site gradients of the SCS adjoint, scattered to atoms.
__global__ void __launch_bounds__(256) k_scs_site_reduce(Work w, DevParams p, int c0) {
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const int n12 = w.counts[c].n12;
  const long long sbase = (long long)c * w.site_cap;
  for (int s = threadIdx.x; s < n12; s += blockDim.x) {
    const double* g = w.sgq + (sbase + s) * p.nqs * 3;
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int q = 0; q < p.nqs; ++q) {
      gx += g[3 * q];
      gy += g[3 * q + 1];
      gz += g[3 * q + 2];
    }
    const int a = w.site_atom[sbase + s];
    if (p.paper && a != c) continue;     // the paper's forces: only atom c's own gradient
    if (gx != 0.0 || gy != 0.0 || gz != 0.0) atomic_add3(w.gacc + 3 * a, gx, gy, gz);
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
void launch_scs_count(const Work& w, const DevParams& p, int max_n12, cudaStream_t s) {
  if (w.n_atoms == 0) return;
  size_t sm = (sizeof(double) + sizeof(float)) * 3 * (size_t)max_n12;
  raise_smem_limit((const void*)k_scs_count, sm);
  k_scs_count<<<w.n_atoms, 256, sm, s>>>(w, p, max_n12);
}

void launch_scs_fill(const Work& w, const DevParams& p, int c0, int c1, int max_n12, int max_n1, cudaStream_t s) {
  if (c1 <= c0) return;
  size_t sm = sizeof(double) * 3 * (size_t)max_n12 +
              sizeof(int) * ((size_t)max_n1 * max_n1 + 6 * (size_t)max_n1 + 2 + (size_t)max_n12 + 8 * (size_t)max_n1) +
              sizeof(float) * 3 * (size_t)max_n12;
  raise_smem_limit((const void*)k_scs_fill, sm);
  k_scs_fill<<<c1 - c0, 256, sm, s>>>(w, p, c0, max_n12, max_n1);
}

void launch_pair_radial(const Work& w, const DevParams& p, cudaStream_t s) {
  if (w.n_atoms == 0) return;
  k_pair_radial<<<w.n_atoms, 128, 0, s>>>(w, p);
}

size_t scs2_forward_smem(int max_n1, int max_n12) { return scs2_smem_bytes(max_n1, max_n12, false); }
size_t scs2_adjoint_smem(int max_n1, int max_n12) { return scs2_smem_bytes(max_n1, max_n12, true); }

// Centres order[c0..c1) (or c0..c1 when order is NULL), shared memory sized for the largest
// K1 and K1 u K2 among them.
void launch_scs_factor(const Work& w, const DevParams& p, const int* order, int c0, int c1, int max_n1, int max_n12,
                       cudaStream_t s) {
  if (c1 <= c0) return;
  size_t sm = scs2_smem_bytes(max_n1, max_n12, false);
  raise_smem_limit((const void*)k_scs_factor, sm);
  k_scs_factor<<<(c1 - c0) * p.nqs, 256, sm, s>>>(w, p, order, c0, max_n1, max_n12);
}

void launch_scs_adjoint2(const Work& w, const DevParams& p, const int* order, int c0, int c1, int max_n1,
                         int max_n12, cudaStream_t s) {
  if (c1 <= c0) return;
  size_t sm = scs2_smem_bytes(max_n1, max_n12, true);
  raise_smem_limit((const void*)k_scs_adjoint2, sm);
  k_scs_adjoint2<<<(c1 - c0) * p.nqs, 256, sm, s>>>(w, p, order, c0, max_n1, max_n12);
}

// LU fallback launches: a fixed grid of lu_blocks persistent blocks (one dense slot each);
// with an empty list every block exits at once.
void launch_scs_lu_forward(const Work& w, const DevParams& p, int lu_blocks, int max_n1, int max_n12, int tally,
                           cudaStream_t s) {
  size_t sm = scs2_smem_bytes(max_n1, max_n12, true);
  raise_smem_limit((const void*)k_scs_lu_forward, sm);
  k_scs_lu_forward<<<lu_blocks, 256, sm, s>>>(w, p, max_n1, max_n12, tally);
}

void launch_scs_lu_adjoint(const Work& w, const DevParams& p, int lu_blocks, int c0, int c1, int max_n1,
                           int max_n12, cudaStream_t s) {
  size_t sm = scs2_smem_bytes(max_n1, max_n12, true);
  raise_smem_limit((const void*)k_scs_lu_adjoint, sm);
  k_scs_lu_adjoint<<<lu_blocks, 256, sm, s>>>(w, p, c0, c1, max_n1, max_n12);
}

void launch_scs_site_reduce(const Work& w, const DevParams& p, int c0, int c1, cudaStream_t s) {
  if (c1 <= c0) return;
  k_scs_site_reduce<<<c1 - c0, 256, 0, s>>>(w, p, c0);
}
