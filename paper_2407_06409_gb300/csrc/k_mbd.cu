// Stage 2: local MBD energy of every central atom (Sec. III.A) and its adjoint.
//
// For central atom k with sphere sites s = 0..ns-1 (s = 0 is k):
//   alpha~_s(omega) = (1 - f_SCS(r_s)) alpha_K,s + f_SCS(r_s) alpha_I,a(s)  if r_s < r_SCS,
//                     alpha_I,a(s) otherwise                              (Eq. full-pol)
//   R~_s = R0 (alpha~_s(0)/alpha0)^(1/3), S~_st = beta (R~_s + R~_t)        (Eq. scaled-rvdw)
//   T_LR,st = f_LR(r_st; r_MBD,p) f(r_st, S~_st) T_st, p = 1 on the central row/column
//   G(omega) = D T_LR D, D = diag(sqrt(alpha~(omega)))                    (Eq. G_frequency)
//   E_k = sum_q w_q/(2 pi) sum_{n=2}^{n_max} (-1/n) Tr[G^n]_kk                 (Eq. E_k)
// The k-block traces use Krylov blocks v_m = G^m e_k (3 ns x 3 per frequency): all
// quadrature frequencies share T_LR, so v_{m+1} = D (T (D v_m)) is one product of T with
// a 3 ns x 3 n_freq block, and Tr[G^n]_kk = <v_a, v_b> with a + b = n.
//
// Adjoint (exact gradient of L = sum_k w_k E_k):
//   dL/dG = sum_n c_n sum_{j=0}^{n-1} v_j v_{n-1-j}^T (G symmetric),
//   dL/dalpha~_s = (1/alpha~_s) Tr[(dL/dG) G]_ss = (1/alpha~_s) sum_n c_n sum_j <v_j[s], v_{n-j}[s]>,
//   dL/dT_st = sum_q D_s D_t (dL/dG)_st, contracted with dT_LR/dr and dT_LR/dS~ per pair.
#include <algorithm>

#include "ff.cuh"
#include "lmbd_internal.cuh"
#include "ozaki.cuh"
#include "pair_epilogue.cuh"

// ---------------------------------------------------------------------------------------
// prepare: blended polarisabilities, SCS radii, T_LR and the first Krylov block
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mbd_prepare(Work w, DevParams p, int c0, int max_ns) {
  extern __shared__ double smem_d[];
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const Counts cn = w.counts[c];
  const int ns = cn.ns, n1 = cn.n1, N = 3 * ns;
  double* xs = smem_d;                 // 3 x max_ns
  double* rt = xs + 3 * max_ns;        // max_ns
  const int tid = threadIdx.x;
  const long long sbase = (long long)c * w.site_cap;
  const long long offs = w.off_s[c], offk1 = w.off_k1[c];
  for (int s = tid; s < ns; s += blockDim.x) {
    int a = w.site_atom[sbase + s];
    double x0 = w.site_x[3 * (sbase + s)], x1 = w.site_x[3 * (sbase + s) + 1], x2 = w.site_x[3 * (sbase + s) + 2];
    xs[s] = x0; xs[max_ns + s] = x1; xs[2 * max_ns + s] = x2;
    rt[s] = mbd_blend_site(w, p, s, a, n1, offs, offk1, x0, x1, x2);
  }
  __syncthreads();
  double* T = w.tlr + w.off_t[c];
  // diagonal blocks are zero
  for (int e = tid; e < ns * 9; e += blockDim.x) {
    int s = e / 9, t = e % 9;
    T[(long long)(3 * s + t / 3) * N + 3 * s + t % 3] = 0.0;
  }
  const int npair = ns * (ns - 1) / 2;
  for (int e = tid; e < npair; e += blockDim.x) {
    int i = (int)((sqrtf(8.0f * e + 1.0f) + 1.0f) * 0.5f);
    while (i * (i - 1) / 2 > e) --i;
    while ((i + 1) * i / 2 <= e) ++i;
    int j = e - i * (i - 1) / 2;     // i > j
    double rr[3] = {xs[j] - xs[i], xs[max_ns + j] - xs[max_ns + i], xs[2 * max_ns + j] - xs[2 * max_ns + i]};
    double blk[3][3], kc[5];
    tlr_pair_block(p, rr, (j == 0) ? p.r_mbd1 : p.r_mbd2, rt[i], rt[j], blk, w.pcoef ? kc : nullptr);
    if (w.pcoef) {
      double* pc = w.pcoef + w.off_t[c] + 8LL * (i * (i - 1) / 2 + j);
      pc[0] = rr[0]; pc[1] = rr[1]; pc[2] = rr[2];
      pc[3] = kc[0]; pc[4] = kc[1]; pc[5] = kc[2]; pc[6] = kc[3]; pc[7] = kc[4];
    }
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
      for (int be = 0; be < 3; ++be) {
        T[(long long)(3 * i + al) * N + 3 * j + be] = blk[al][be];
        T[(long long)(3 * j + al) * N + 3 * i + be] = blk[al][be];
      }
  }
  __threadfence_block();
  __syncthreads();
  // v_1 = G e_k: column block of the central site, scaled by D_s D_0 (per frequency)
  const int ncv = 3 * p.n_freq;
  double* V1 = w.vkr + (offs * 3) * ncv;
  for (int e = tid; e < N * ncv; e += blockDim.x) {
    int row = e / ncv, col = e % ncv;
    int s = row / 3, q = col / 3 + 1, be = col % 3;
    double d = w.dsq[(offs + s) * p.nq + q] * w.dsq[offs * p.nq + q];
    V1[(long long)row * ncv + col] = d * T[(long long)row * N + be];
  }
}

// ---------------------------------------------------------------------------------------
// chain: v_{m+1} = D (T (D v_m)), one block per (central atom, 64-row tile)
// ---------------------------------------------------------------------------------------
#define CH_R 64
#define CH_K 32
#define CH_C 36

__global__ void __launch_bounds__(256) k_mbd_chain(Work w, DevParams p, int m, int c0, int tiles_per_c) {
  __shared__ double Ts[CH_R][CH_K + 1];
  __shared__ double Ws[CH_K][CH_C];
  const int c = c0 + blockIdx.x / tiles_per_c;
  const int tile = blockIdx.x % tiles_per_c;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns, N = 3 * ns;
  const int row0 = tile * CH_R;
  if (row0 >= N) return;
  const long long offs = w.off_s[c];
  const int ncv = 3 * p.n_freq;
  const double* T = w.tlr + w.off_t[c];
  const double* Vin = w.vkr + (long long)(m - 1) * w.vstride + (offs * 3) * ncv;
  double* Vout = w.vkr + (long long)m * w.vstride + (offs * 3) * ncv;
  const double* dsq = w.dsq + offs * p.nq;
  const int tid = threadIdx.x;
  const int tr = tid % CH_R, cg = tid / CH_R;     // row in tile, column group (4 x 9)
  for (int cc0 = 0; cc0 < ncv; cc0 += CH_C) {
    const int ncc = min(CH_C, ncv - cc0);
    double acc[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) acc[j] = 0.0;
    for (int k0 = 0; k0 < N; k0 += CH_K) {
      __syncthreads();
      for (int e = tid; e < CH_R * CH_K; e += blockDim.x) {
        int rr = e / CH_K, kk = e % CH_K;
        int gr = row0 + rr, gk = k0 + kk;
        Ts[rr][kk] = (gr < N && gk < N) ? T[(long long)gr * N + gk] : 0.0;
      }
      for (int e = tid; e < CH_K * CH_C; e += blockDim.x) {
        int kk = e / CH_C, cl = e % CH_C;
        int gk = k0 + kk, gc = cc0 + cl;
        double v = 0.0;
        if (gk < N && cl < ncc) v = dsq[(gk / 3) * p.nq + gc / 3 + 1] * Vin[(long long)gk * ncv + gc];
        Ws[kk][cl] = v;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < CH_K; ++kk) {
        double t = Ts[tr][kk];
#pragma unroll
        for (int j = 0; j < 9; ++j) acc[j] += t * Ws[kk][cg * 9 + j];
      }
    }
    const int gr = row0 + tr;
    if (gr < N) {
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        int gc = cc0 + cg * 9 + j;
        if (cg * 9 + j < ncc) Vout[(long long)gr * ncv + gc] = dsq[(gr / 3) * p.nq + gc / 3 + 1] * acc[j];
      }
    }
  }
}

// Series coefficient c_n of centre c at frequency column qq: -1/n (Eq. E_k), or the fitted one.
__device__ __forceinline__ double series_c(const Work& w, const DevParams& p, int c, int qq, int n) {
  return p.lanczos ? w.cfit[((long long)c * p.n_freq + qq) * LMBD_MAX_ORDER_P1 + n] : p.cn[n];
}

// ---------------------------------------------------------------------------------------
// polynomial-fit series coefficients (Sec. III.A, Eqs. diagonal_appr and polynomial-fit):
// per centre and frequency, the spectral interval [lambda_min, lambda_max] of the symmetric
// G = D T_LR D from m Lanczos steps (three-term recurrence, no reorthogonalisation, start
// vector from SplitMix64), then c_n, n = 1..n_max, of the L2 fit of ln(1 - lambda) on it.
// ---------------------------------------------------------------------------------------
#define LZ_THREADS 256
#define LZ_RPT 4          // rows per thread: 3 ns <= 1024
#define LZ_QC 12          // frequencies per pass

// SplitMix64 output for counter i (state 0 advanced i + 1 times), mapped to [-1, 1).
__device__ __forceinline__ double splitmix_unit(unsigned long long i) {
  unsigned long long z = (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-52 - 1.0;
}

// Sums the qc per-thread partials v[q] over the block; every thread gets the totals in out[].
__device__ __forceinline__ void lz_block_sum(const double* v, int qc, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < qc; ++q) {
    double t = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[q * (LZ_THREADS / 32) + warp] = t;
  }
  __syncthreads();
  for (int q = 0; q < qc; ++q) {
    double t = 0.0;
    for (int k = 0; k < LZ_THREADS / 32; ++k) t += red[q * (LZ_THREADS / 32) + k];
    out[q] = t;
  }
  __syncthreads();
}

// Number of eigenvalues below x of the symmetric tridiagonal (a, b) of order m (Sturm count).
__device__ int lz_sturm(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    const double off = i > 0 ? b[i - 1] * b[i - 1] / d : 0.0;
    d = a[i] - x - off;
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Eigenvalue number `which` (0 = smallest, m - 1 = largest) by bisection on the Sturm count.
__device__ double lz_eig(const double* a, const double* b, int m, int which) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (lz_sturm(a, b, m, mid) > which) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Eigenvalues and first eigenvector components of the symmetric tridiagonal matrix (a, b) of
// order m, in place: on return a[i] = theta_i and z[i] = first component of eigenvector i (z
// enters as e_1).  Implicit QL iteration with Wilkinson-type shifts (the tridiagonal QL
// algorithm of Bowdler, Martin, Reinsch and Wilkinson, 1968); only the first row of the
// eigenvector matrix is carried along, as in the Golub-Welsch construction of Gauss rules.
// b[m - 1] is used as scratch.  Returns false if an eigenvalue took more than 60 sweeps.
__device__ bool tridiag_ql_first_row(double* a, double* b, double* z, int m) {
  for (int i = 0; i < m; ++i) z[i] = i == 0 ? 1.0 : 0.0;
  if (m <= 1) return true;
  b[m - 1] = 0.0;
  for (int l = 0; l < m; ++l) {
    int iter = 0;
    while (true) {
      int mm = l;
      for (; mm < m - 1; ++mm) {
        const double dd = fabs(a[mm]) + fabs(a[mm + 1]);
        if (fabs(b[mm]) <= 1e-17 * dd) break;
      }
      if (mm == l) break;
      if (++iter > 60) return false;
      // shift from the 2 x 2 block at the top of the unreduced part
      double g = (a[l + 1] - a[l]) / (2.0 * b[l]);
      double r = hypot(g, 1.0);
      g = a[mm] - a[l] + b[l] / (g + (g >= 0.0 ? r : -r));
      double sn = 1.0, cs = 1.0, pp = 0.0;
      int i = mm - 1;
      bool early = false;
      for (; i >= l; --i) {
        const double f = sn * b[i], bb = cs * b[i];
        r = hypot(f, g);
        b[i + 1] = r;
        if (r == 0.0) {   // the rotation splits the matrix: deflate and restart this l
          a[i + 1] -= pp;
          b[mm] = 0.0;
          early = true;
          break;
        }
        sn = f / r;
        cs = g / r;
        g = a[i + 1] - pp;
        r = (a[i] - g) * sn + 2.0 * cs * bb;
        pp = sn * r;
        a[i + 1] = g + pp;
        g = cs * r - bb;
        const double zt = z[i + 1];
        z[i + 1] = sn * z[i] + cs * zt;
        z[i] = cs * z[i] - sn * zt;
      }
      if (early) continue;
      a[l] -= pp;
      b[l] = g;
      b[mm] = 0.0;
    }
  }
  return true;
}

// Lanczos recurrences on G(omega) = D T_LR D for every frequency of this pass (frequencies
// q0 ..), nd start vectors per frequency (vector v <-> frequency q0 + v / nd, direction v % nd):
//  * nd = 1 (polynomial-fit coefficients, Sec. III.A): SplitMix64 start vector, the extreme
//    Ritz values go to w.lam;
//  * nd = 3 (log mode): start vectors e_alpha, the centre's three rows; the Gauss rule of the
//    tridiagonal matrix J (Ritz values theta_i, squared first components z_i^2) gives
//    e_alpha^T ln(1 - G) e_alpha ~ sum_i z_i^2 ln(1 - theta_i) (exact once the Krylov space is
//    exhausted, b = 0), and the three directions sum to the k-block trace of ln(1 - G)
//    (Eq. series-expansion, the n_max -> infinity limit), stored per frequency in trbuf row 0.
__global__ void __launch_bounds__(LZ_THREADS) k_lanczos(Work w, DevParams p, int c0, int q0, int qc, int L3, int nd) {
  extern __shared__ double lzs[];
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns, N = 3 * ns;
  double* V = lzs;                                // L3 x qc, row-major
  double* Vp = V + (size_t)L3 * qc;
  double* X = Vp + (size_t)L3 * qc;
  double* al = X + (size_t)L3 * qc;               // qc x LMBD_MAX_LANCZOS
  double* be = al + qc * LMBD_MAX_LANCZOS;
  double* red = be + qc * LMBD_MAX_LANCZOS;       // qc x (threads / 32)
  __shared__ int mq[LZ_QC];                       // steps taken per frequency
  __shared__ double bprev[LZ_QC];
  const int tid = threadIdx.x;
  const double* T = w.tlr + w.off_t[c];
  const long long offs = w.off_s[c];
  const bool logm = nd == 3;
  const int m = min(logm ? p.logmode : p.lanczos, N);
  // start vectors: u / |u| for every frequency, or e_alpha
  double part[LZ_QC];
  double tot[LZ_QC];
  for (int q = 0; q < LZ_QC; ++q) part[q] = 0.0;
  double inv = 1.0;
  if (!logm) {
    for (int r = 0; r < LZ_RPT; ++r) {
      const int i = tid + r * LZ_THREADS;
      if (i < N) {
        const double u = splitmix_unit((unsigned long long)i);
        part[0] += u * u;
      }
    }
    lz_block_sum(part, 1, red, tot);
    inv = 1.0 / sqrt(tot[0]);
  }
  for (int r = 0; r < LZ_RPT; ++r) {
    const int i = tid + r * LZ_THREADS;
    if (i < N) {
      const double u = logm ? 0.0 : splitmix_unit((unsigned long long)i) * inv;
      for (int q = 0; q < qc; ++q) {
        V[i * qc + q] = logm ? (i == q % 3 ? 1.0 : 0.0) : u;
        Vp[i * qc + q] = 0.0;
      }
    }
  }
  if (tid < qc) {
    mq[tid] = 0;
    bprev[tid] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    // X = D V
    for (int e = tid; e < N * qc; e += LZ_THREADS) {
      const int i = e / qc, q = e % qc;
      X[e] = w.dsq[(offs + i / 3) * p.nq + q0 + q / nd + 1] * V[e];
    }
    __syncthreads();
    // Y = D (T X): T symmetric, so thread i reads column i of row k (coalesced)
    double y[LZ_RPT][LZ_QC];
#pragma unroll
    for (int r = 0; r < LZ_RPT; ++r)
#pragma unroll
      for (int q = 0; q < LZ_QC; ++q) y[r][q] = 0.0;
    for (int k = 0; k < N; ++k) {
      const double* Tk = T + (long long)k * N;
      const double* xk = X + k * qc;
#pragma unroll
      for (int r = 0; r < LZ_RPT; ++r) {
        const int i = tid + r * LZ_THREADS;
        if (i < N) {
          const double t = Tk[i];
#pragma unroll
          for (int q = 0; q < LZ_QC; ++q)
            if (q < qc) y[r][q] += t * xk[q];
        }
      }
    }
    // alpha_q = <v_q, y_q>
    for (int q = 0; q < LZ_QC; ++q) part[q] = 0.0;
#pragma unroll
    for (int r = 0; r < LZ_RPT; ++r) {
      const int i = tid + r * LZ_THREADS;
      if (i < N) {
#pragma unroll
        for (int q = 0; q < LZ_QC; ++q)
          if (q < qc) {
            y[r][q] *= w.dsq[(offs + i / 3) * p.nq + q0 + q / nd + 1];
            part[q] += V[i * qc + q] * y[r][q];
          }
      }
    }
    double alpha[LZ_QC];
    lz_block_sum(part, qc, red, alpha);
    // w = y - alpha v - beta v_prev, beta = |w|
    for (int q = 0; q < LZ_QC; ++q) part[q] = 0.0;
#pragma unroll
    for (int r = 0; r < LZ_RPT; ++r) {
      const int i = tid + r * LZ_THREADS;
      if (i < N) {
#pragma unroll
        for (int q = 0; q < LZ_QC; ++q)
          if (q < qc) {
            y[r][q] = y[r][q] - alpha[q] * V[i * qc + q] - bprev[q] * Vp[i * qc + q];
            part[q] += y[r][q] * y[r][q];
          }
      }
    }
    double beta[LZ_QC];
    lz_block_sum(part, qc, red, beta);
    for (int q = 0; q < LZ_QC; ++q)
      if (q < qc) beta[q] = sqrt(beta[q]);
    if (tid < qc && mq[tid] == j) {           // frequency still running: record step j
      al[tid * LMBD_MAX_LANCZOS + j] = alpha[tid];
      mq[tid] = j + 1;
      // log mode: a beta below 1e-13 of the largest recurrence coefficient so far means the
      // Krylov space is exhausted to rounding (the Gauss rule is then exact)
      double scale = 0.0;
      if (logm)
        for (int u = 0; u <= j; ++u)
          scale = fmax(scale, fabs(al[tid * LMBD_MAX_LANCZOS + u]) + (u < j ? be[tid * LMBD_MAX_LANCZOS + u] : 0.0));
      if (j < m - 1 && beta[tid] != 0.0 && !(logm && beta[tid] <= 1e-13 * scale)) {
        be[tid * LMBD_MAX_LANCZOS + j] = beta[tid];
      } else {
        mq[tid] = -(j + 1);                   // finished with j + 1 steps
      }
    }
    __syncthreads();
    // v_prev = v, v = w / beta for the frequencies still running
#pragma unroll
    for (int r = 0; r < LZ_RPT; ++r) {
      const int i = tid + r * LZ_THREADS;
      if (i < N) {
#pragma unroll
        for (int q = 0; q < LZ_QC; ++q)
          if (q < qc && mq[q] > 0) {
            Vp[i * qc + q] = V[i * qc + q];
            V[i * qc + q] = y[r][q] / beta[q];
          }
      }
    }
    if (tid < qc && mq[tid] > 0) bprev[tid] = beta[tid];
    __syncthreads();
    bool running = false;
    for (int q = 0; q < qc; ++q) running |= mq[q] > 0;
    if (!running) break;
  }
  if (!logm) {
    // extremes of the tridiagonal matrices
    if (tid < qc) {
      const int mm = mq[tid] < 0 ? -mq[tid] : mq[tid];
      const double* a = al + tid * LMBD_MAX_LANCZOS;
      const double* b = be + tid * LMBD_MAX_LANCZOS;
      double* out = w.lam + ((long long)c * p.n_freq + q0 + tid) * 2;
      out[0] = lz_eig(a, b, mm, 0);
      out[1] = lz_eig(a, b, mm, mm - 1);
    }
    return;
  }
  // log mode: Gauss rule of every tridiagonal, then the sum over the three directions
  double* lq = red;                               // qc partial traces (red is free now)
  __syncthreads();
  if (tid < qc) {
    const int mm = mq[tid] < 0 ? -mq[tid] : mq[tid];
    double* a = al + tid * LMBD_MAX_LANCZOS;
    double* b = be + tid * LMBD_MAX_LANCZOS;
    double* z = X + (size_t)tid * L3;   // X is free after the recurrence; mm <= N <= L3
    double t = 0.0;
    if (!tridiag_ql_first_row(a, b, z, mm)) {
      atomicOr(w.status, LMBD_FLAG_MODEL);
      t = nan("");
    } else {
      for (int i = 0; i < mm; ++i) t += z[i] * z[i] * log1p(-a[i]);
    }
    lq[tid] = t;
  }
  __syncthreads();
  if (tid < qc / 3) {
    const double t = lq[3 * tid] + lq[3 * tid + 1] + lq[3 * tid + 2];
    w.trbuf[((long long)c * LMBD_MAX_ORDER_P1) * 64 + q0 + tid] = t;
  }
}

// c_0..c_n_max of the L2 fit of ln(1 - lambda) by sum_{n>=1} c_n lambda^n on [lo, hi] (64-point
// Gauss-Legendre quadrature, columns in lambda / rho, Householder least squares); one thread
// per (centre, frequency).
__global__ void __launch_bounds__(128) k_series_fit(Work w, DevParams p, int c0, int c1) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = p.n_freq, order = p.order;
  if (e >= (long long)(c1 - c0) * nf) return;
  const int c = c0 + (int)(e / nf), q = (int)(e % nf);
  const double lo = w.lam[((long long)c * nf + q) * 2], hi = w.lam[((long long)c * nf + q) * 2 + 1];
  double* cf = w.cfit + ((long long)c * nf + q) * LMBD_MAX_ORDER_P1;
  cf[0] = 0.0;
  const bool degenerate = !(hi - lo > 1e-12);
  if (degenerate || !(hi < 1.0)) {            // point interval: Taylor coefficients
    if (!degenerate) atomicOr(w.status, LMBD_FLAG_MODEL);   // ln(1 - lambda) undefined
    for (int n = 1; n <= order; ++n) cf[n] = -1.0 / n;
    return;
  }
  const double rho = fmax(fabs(lo), fabs(hi));
  double A[LMBD_MAX_ORDER_P1 - 1][64];
  double y[64];
  for (int i = 0; i < 64; ++i) {
    const double lam = 0.5 * (hi - lo) * w.gl64[i] + 0.5 * (hi + lo);
    const double sw = sqrt(0.5 * (hi - lo) * w.gl64[64 + i]);
    const double t = lam / rho;
    double pw = 1.0;
    for (int n = 0; n < order; ++n) {
      pw *= t;
      A[n][i] = pw * sw;
    }
    y[i] = log1p(-lam) * sw;
  }
  double rd[LMBD_MAX_ORDER_P1 - 1];
  for (int k = 0; k < order; ++k) {
    double nrm = 0.0;
    for (int i = k; i < 64; ++i) nrm += A[k][i] * A[k][i];
    nrm = sqrt(nrm);
    const double alpha = A[k][k] > 0.0 ? -nrm : nrm;
    A[k][k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < 64; ++i) vv += A[k][i] * A[k][i];
    rd[k] = alpha;
    if (vv == 0.0) continue;
    for (int l = k + 1; l < order; ++l) {
      double d = 0.0;
      for (int i = k; i < 64; ++i) d += A[k][i] * A[l][i];
      d *= 2.0 / vv;
      for (int i = k; i < 64; ++i) A[l][i] -= d * A[k][i];
    }
    double d = 0.0;
    for (int i = k; i < 64; ++i) d += A[k][i] * y[i];
    d *= 2.0 / vv;
    for (int i = k; i < 64; ++i) y[i] -= d * A[k][i];
  }
  double dcoef[LMBD_MAX_ORDER_P1 - 1];
  for (int k = order - 1; k >= 0; --k) {
    double t = y[k];
    for (int l = k + 1; l < order; ++l) t -= A[l][k] * dcoef[l];
    dcoef[k] = t / rd[k];
  }
  double rp = 1.0;
  for (int n = 1; n <= order; ++n) {
    rp *= rho;
    cf[n] = dcoef[n - 1] / rp;
  }
}

// Lanczos passes over the frequencies: nd vectors per frequency, three L3 x (vectors) arrays in
// shared memory next to the recurrence coefficients; frequencies of one pass share T_LR reads.
static bool launch_lanczos(const Work& w, const DevParams& p, int c0, int c1, int max_ns, int nd, cudaStream_t s) {
  const int L3 = 3 * max_ns;
  if (L3 > LZ_THREADS * LZ_RPT) return false;
  const size_t per_v = sizeof(double) * (3 * (size_t)L3 + 2 * LMBD_MAX_LANCZOS + LZ_THREADS / 32);
  int qf = (int)((200 * 1024) / (per_v * nd));       // frequencies per pass
  qf = std::max(1, std::min(std::min(qf, LZ_QC / nd), p.n_freq));
  for (int q0 = 0; q0 < p.n_freq; q0 += qf) {
    const int n = std::min(qf, p.n_freq - q0);
    const size_t sm = per_v * n * nd;
    raise_smem_limit((const void*)k_lanczos, sm);
    k_lanczos<<<c1 - c0, LZ_THREADS, sm, s>>>(w, p, c0, q0, n * nd, L3, nd);
  }
  return true;
}

bool launch_series_coefficients(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s) {
  if (c1 <= c0) return true;
  if (!launch_lanczos(w, p, c0, c1, max_ns, 1, s)) return false;
  const long long items = (long long)(c1 - c0) * p.n_freq;
  k_series_fit<<<(unsigned)((items + 127) / 128), 128, 0, s>>>(w, p, c0, c1);
  return true;
}

bool launch_log_mode(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s) {
  if (c1 <= c0) return true;
  return launch_lanczos(w, p, c0, c1, max_ns, 3, s);
}

// ---------------------------------------------------------------------------------------
// fitted integrand (Sec. III.C, Eq. integrand and Eq. E_MBD_k): with I_j = I(nu_j) at
// nu_0 = 0 and the fit nodes, phi(omega) = a / (1 + sum_{n=1}^{n_max} b_n omega^(2n)) with
// a, b_n >= 0 minimises sum_j [a I_0 - sum_n b_n nu_j^(2n) I_j - I_j]^2 (Lawson-Hanson
// active set on unit-norm columns), and E_k = H I_0 sum_i wt_i phi(Omega_i).
// One thread per centre; the systems are at most 25 x 11.
// ---------------------------------------------------------------------------------------
struct FitScratch {
  double A[LMBD_MAX_ORDER_P1][LMBD_FIT_ROWS];   // columns scaled to unit norm
  double W[LMBD_MAX_ORDER_P1][LMBD_FIT_ROWS];   // Householder vectors / R of the passive columns
  double y[LMBD_FIT_ROWS];
  double qy[LMBD_FIT_ROWS];
  double sc[LMBD_MAX_ORDER_P1];                 // column norms
  double rdiag[LMBD_MAX_ORDER_P1];
};

// QR of the k passive columns idx[] (Householder); R[i][l] (i < l) is W[l][i], R[i][i] rdiag[i].
// Solves min |A_P z - y|.  Returns 0 if a column is numerically dependent on the others.
__device__ int fit_qr_solve(FitScratch& S, int J, const int* idx, int k, double* z) {
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < J; ++j) S.W[i][j] = S.A[idx[i]][j];
  for (int j = 0; j < J; ++j) S.qy[j] = S.y[j];
  for (int i = 0; i < k; ++i) {
    double nrm = 0.0;
    for (int j = i; j < J; ++j) nrm += S.W[i][j] * S.W[i][j];
    nrm = sqrt(nrm);
    if (!(nrm > 1e-14)) return 0;
    const double alpha = S.W[i][i] > 0.0 ? -nrm : nrm;
    S.W[i][i] -= alpha;
    double vv = 0.0;
    for (int j = i; j < J; ++j) vv += S.W[i][j] * S.W[i][j];
    S.rdiag[i] = alpha;
    for (int l = i + 1; l < k; ++l) {
      double d = 0.0;
      for (int j = i; j < J; ++j) d += S.W[i][j] * S.W[l][j];
      d *= 2.0 / vv;
      for (int j = i; j < J; ++j) S.W[l][j] -= d * S.W[i][j];
    }
    double d = 0.0;
    for (int j = i; j < J; ++j) d += S.W[i][j] * S.qy[j];
    d *= 2.0 / vv;
    for (int j = i; j < J; ++j) S.qy[j] -= d * S.W[i][j];
  }
  for (int i = k - 1; i >= 0; --i) {
    double t = S.qy[i];
    for (int l = i + 1; l < k; ++l) t -= S.W[l][i] * z[l];
    z[i] = t / S.rdiag[i];
  }
  return 1;
}

// Lawson-Hanson NNLS on S.A (J x C, unit-norm columns), S.y.  Writes the passive flags and x.
__device__ void fit_nnls(FitScratch& S, int J, int C, int* passive, double* x) {
  for (int c = 0; c < C; ++c) {
    passive[c] = 0;
    x[c] = 0.0;
  }
  double ny = 0.0;
  for (int j = 0; j < J; ++j) ny += S.y[j] * S.y[j];
  ny = sqrt(ny);
  if (ny == 0.0) return;
  const double tol = 1e-13 * ny;
  int idx[LMBD_MAX_ORDER_P1];
  double z[LMBD_MAX_ORDER_P1], zf[LMBD_MAX_ORDER_P1];
  for (int outer = 0; outer < 3 * C; ++outer) {
    double r[LMBD_FIT_ROWS];
    for (int j = 0; j < J; ++j) {
      double t = S.y[j];
      for (int c = 0; c < C; ++c) t -= S.A[c][j] * x[c];
      r[j] = t;
    }
    int best = -1;
    double gbest = 0.0;
    for (int c = 0; c < C; ++c) {
      if (passive[c]) continue;
      double g = 0.0;
      for (int j = 0; j < J; ++j) g += S.A[c][j] * r[j];
      if (best < 0 || g > gbest) {
        best = c;
        gbest = g;
      }
    }
    if (best < 0 || !(gbest > tol)) break;
    passive[best] = 1;
    for (int inner = 0; inner <= C; ++inner) {
      int k = 0;
      for (int c = 0; c < C; ++c)
        if (passive[c]) idx[k++] = c;
      if (!fit_qr_solve(S, J, idx, k, z))
        for (int i = 0; i < k; ++i) z[i] = 0.0;     // dependent column: step back to x
      for (int c = 0; c < C; ++c) zf[c] = 0.0;
      bool all_pos = true;
      for (int i = 0; i < k; ++i) {
        zf[idx[i]] = z[i];
        if (!(z[i] > 0.0)) all_pos = false;
      }
      if (all_pos) {
        for (int c = 0; c < C; ++c) x[c] = zf[c];
        break;
      }
      // step from x towards z until the first passive component reaches zero
      int jmin = -1;
      double smin = 0.0;
      for (int i = 0; i < k; ++i) {
        const int c = idx[i];
        if (zf[c] <= 0.0) {
          const double st = x[c] / (x[c] - zf[c]);
          if (jmin < 0 || st < smin) {
            jmin = c;
            smin = st;
          }
        }
      }
      for (int c = 0; c < C; ++c) x[c] += smin * (zf[c] - x[c]);
      x[jmin] = 0.0;
      bool any = false;
      for (int i = 0; i < k; ++i) {
        const int c = idx[i];
        if (x[c] <= 0.0) {
          x[c] = 0.0;
          passive[c] = 0;
        } else {
          any = true;
        }
      }
      if (!any) break;
    }
  }
}

// Fitted force integrand of Sec. III.D.  For every atom and Cartesian component, the force
// integrand F(nu_j) of the paper's forces at the J sample frequencies (nu_0 = 0, then the fit
// nodes) gives the ratios R_j = F(nu_j) / F(0); theta(omega) = sum_{i<=M} u_i (-omega)^i /
// (1 + sum_{l<=K} v_l omega^(2l)) with u, v >= 0 is fitted to the multiplied-out equations
// sum_i u_i (-nu_j)^i - R_j sum_l v_l nu_j^(2l) = R_j by the Lawson-Hanson NNLS above (unit-norm
// columns), and the force is F(0) times the quadrature of theta / (2 pi).  A fit whose numerator
// does not grow two orders slower than its denominator is repeated with the numerator order
// lowered by one; if none is integrable, LMBD_FLAG_MODEL.  One thread per component, its NNLS
// workspace in shared memory.
__global__ void __launch_bounds__(16) k_theta_fit(int n, const double* __restrict__ F, ThetaParams tp, double* out,
                                                  int* status) {
  extern __shared__ unsigned char theta_smem[];
  FitScratch& S = reinterpret_cast<FitScratch*>(theta_smem)[threadIdx.x];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * n) return;
  const int J = tp.J, K = tp.K;
  const double F0 = F[e];
  if (F0 == 0.0) {
    out[e] = 0.0;
    return;
  }
  // numerator order lowered until the fitted theta decays at least as omega^-2
  double x[LMBD_MAX_ORDER_P1];
  int M = tp.M;
  bool ok = false;
  for (; M >= 0 && !ok; --M) {
    const int C = M + 1 + K;
    for (int j = 0; j < J; ++j) {
      const double R = F[(long long)j * 3 * n + e] / F0;
      const double nu = tp.nu[j], nu2 = nu * nu;
      double pw = 1.0;
      for (int i = 0; i <= M; ++i) {
        S.A[i][j] = pw;
        pw *= -nu;
      }
      pw = 1.0;
      for (int l = 1; l <= K; ++l) {
        pw *= nu2;
        S.A[M + l][j] = -R * pw;
      }
      S.y[j] = R;
    }
    for (int c = 0; c < C; ++c) {
      double t = 0.0;
      for (int j = 0; j < J; ++j) t += S.A[c][j] * S.A[c][j];
      t = sqrt(t);
      S.sc[c] = t > 0.0 ? t : 1.0;
      for (int j = 0; j < J; ++j) S.A[c][j] /= S.sc[c];
    }
    int passive[LMBD_MAX_ORDER_P1];
    double xs[LMBD_MAX_ORDER_P1];
    fit_nnls(S, J, C, passive, xs);
    int ju = -1, lv = 0;
    for (int c = 0; c < C; ++c) {
      x[c] = xs[c] / S.sc[c];
      if (x[c] > 0.0) {
        if (c <= M) ju = c;
        else lv = c - M;
      }
    }
    ok = ju < 0 || 2 * lv >= ju + 2;
    if (ok) break;
  }
  if (!ok) {
    atomicOr(status, LMBD_FLAG_MODEL);
    out[e] = 0.0;
    return;
  }
  double integral = 0.0;
  for (int i = 0; i < tp.nphi; ++i) {
    const double om = tp.om[i], om2 = om * om;
    double num = 0.0, pw = 1.0;
    for (int c = 0; c <= M; ++c) {
      num += x[c] * pw;
      pw *= -om;
    }
    double den = 1.0;
    pw = 1.0;
    for (int l = 1; l <= K; ++l) {
      pw *= om2;
      den += x[M + l] * pw;
    }
    integral += tp.wt[i] * num / den;
  }
  out[e] = F0 * integral;
}

void launch_theta_fit(int n, const double* F, const ThetaParams& tp, double* out, int* status, cudaStream_t s) {
  if (n <= 0) return;
  const size_t sm = 16 * sizeof(FitScratch);
  raise_smem_limit((const void*)k_theta_fit, sm);
  k_theta_fit<<<(3 * n + 15) / 16, 16, sm, s>>>(n, F, tp, out, status);
}

// Energy of one centre from its integrand values I[0..J-1] (Hartree), and dE/dI_j into dI.
__device__ double fit_energy(FitScratch& S, const double* I, const DevParams& p, double* dI, int* status) {
  const int J = p.n_freq, C = p.order + 1;
  for (int j = 0; j < J; ++j) {
    const double nu2 = p.omega[j + 1] * p.omega[j + 1];
    S.A[0][j] = I[0];
    double pw = 1.0;
    for (int n = 1; n < C; ++n) {
      pw *= nu2;
      S.A[n][j] = -pw * I[j];
    }
    S.y[j] = I[j];
  }
  for (int c = 0; c < C; ++c) {
    double t = 0.0;
    for (int j = 0; j < J; ++j) t += S.A[c][j] * S.A[c][j];
    t = sqrt(t);
    S.sc[c] = t > 0.0 ? t : 1.0;
    for (int j = 0; j < J; ++j) S.A[c][j] /= S.sc[c];
  }
  int passive[LMBD_MAX_ORDER_P1];
  double xs[LMBD_MAX_ORDER_P1];
  fit_nnls(S, J, C, passive, xs);
  double x[LMBD_MAX_ORDER_P1];
  bool decays = false;
  for (int c = 0; c < C; ++c) {
    x[c] = xs[c] / S.sc[c];           // coefficients of the unscaled columns
    if (c > 0 && x[c] > 0.0) decays = true;
  }
  if (x[0] > 0.0 && !decays) atomicOr(status, LMBD_FLAG_MODEL);
  // E = H I_0 Phi, Phi = sum_i wt_i a / den_i
  double phi = 0.0, abar = 0.0;
  double bbar[LMBD_MAX_ORDER_P1];
  for (int n = 0; n < C; ++n) bbar[n] = 0.0;
  for (int i = 0; i < p.n_phi; ++i) {
    const double om2 = p.phi_omega[i] * p.phi_omega[i];
    double den = 1.0, pw = 1.0;
    for (int n = 1; n < C; ++n) {
      pw *= om2;
      den += x[n] * pw;
    }
    const double wt = p.phi_wt[i];
    phi += wt * x[0] / den;
    abar += wt / den;
    pw = 1.0;
    for (int n = 1; n < C; ++n) {
      pw *= om2;
      bbar[n] -= wt * x[0] * pw / (den * den);
    }
  }
  const double H = LMBD_HARTREE;
  const double E = H * I[0] * phi;
  if (dI) {
    for (int j = 0; j < J; ++j) dI[j] = 0.0;
    dI[0] = H * phi;
    int idx[LMBD_MAX_ORDER_P1];
    int k = 0;
    for (int c = 0; c < C; ++c)
      if (passive[c]) idx[k++] = c;
    double z[LMBD_MAX_ORDER_P1];
    if (k > 0 && fit_qr_solve(S, J, idx, k, z)) {
      // xbar of the passive columns (unscaled), then z = (A_P^T A_P)^-1 xbar through R
      double u[LMBD_MAX_ORDER_P1], v[LMBD_MAX_ORDER_P1], zh[LMBD_MAX_ORDER_P1];
      for (int i = 0; i < k; ++i) {
        const int c = idx[i];
        const double xb = (c == 0 ? abar : bbar[c]) * H * I[0];
        u[i] = xb / S.sc[c];
      }
      for (int i = 0; i < k; ++i) {          // R^T v = u
        double t = u[i];
        for (int l = 0; l < i; ++l) t -= S.W[i][l] * v[l];
        v[i] = t / S.rdiag[i];
      }
      for (int i = k - 1; i >= 0; --i) {     // R zh = v
        double t = v[i];
        for (int l = i + 1; l < k; ++l) t -= S.W[l][i] * zh[l];
        zh[i] = t / S.rdiag[i];
      }
      for (int j = 0; j < J; ++j) {
        double Az = 0.0, r = S.y[j];
        for (int i = 0; i < k; ++i) {
          Az += S.A[idx[i]][j] * zh[i];
          r -= S.A[idx[i]][j] * S.sc[idx[i]] * x[idx[i]];
        }
        dI[j] += Az;                                  // through y_j = I_j
        const double nu2 = p.omega[j + 1] * p.omega[j + 1];
        for (int i = 0; i < k; ++i) {
          const int c = idx[i];
          const double Abar = r * (zh[i] / S.sc[c]) - Az * x[c];
          if (c == 0) {
            dI[0] += Abar;                            // A_j0 = I_0
          } else {
            double pw = 1.0;
            for (int n = 0; n < c; ++n) pw *= nu2;
            dI[j] -= pw * Abar;                       // A_jc = -nu_j^(2c) I_j
          }
        }
      }
    }
  }
  return E;
}

// ---------------------------------------------------------------------------------------
// energy: tr_{n,q} = <v_a, v_b>_q (a + b = n) and E_k = sum_q cw_q sum_n (-1/n) tr_{n,q}
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mbd_energy(Work w, DevParams p, int c0) {
  // deterministic: G = floor(256 / 3 n_freq) row groups per column, thread (g, col) sums the rows
  // g, g + G, ... in order, then fixed-order sums over the groups and over the three columns of
  // each frequency
  __shared__ double red[LMBD_MAX_ORDER_P1][256];
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns, N = 3 * ns;
  const long long offs = w.off_s[c];
  const int ncv = 3 * p.n_freq;
  const int tid = threadIdx.x;
  const int G = ncv <= (int)blockDim.x ? (int)blockDim.x / ncv : 1;   // G ncv <= 256
  for (int it = tid; it < G * ncv && !p.logmode; it += blockDim.x) {
    const int g = it / ncv, col = it % ncv;
    double acc[LMBD_MAX_ORDER_P1];
#pragma unroll
    for (int n = 0; n < LMBD_MAX_ORDER_P1; ++n) acc[n] = 0.0;
    for (int row = g; row < N; row += G) {
      for (int n = 2; n <= p.order; ++n) {
        int a = n / 2, b = n - a;
        const double* Va = w.vkr + (long long)(a - 1) * w.vstride + (offs * 3) * ncv;
        const double* Vb = w.vkr + (long long)(b - 1) * w.vstride + (offs * 3) * ncv;
        acc[n] += Va[(long long)row * ncv + col] * Vb[(long long)row * ncv + col];
      }
    }
    for (int n = 2; n <= p.order; ++n) red[n][it] = acc[n];
  }
  __syncthreads();
  for (int col = tid; col < ncv && !p.logmode; col += blockDim.x)   // own column's slots only
    for (int n = 2; n <= p.order; ++n) {
      double sum = red[n][col];
      for (int g = 1; g < G; ++g) sum += red[n][g * ncv + col];
      red[n][col] = sum;
    }
  __syncthreads();
  __shared__ double epart[64];
  __shared__ double ival[64];
  if (tid < p.n_freq && p.logmode) {   // log mode: the k-block trace of ln(1 - G) per frequency
    const double e = w.trbuf[((long long)c * (LMBD_MAX_ORDER_P1)) * 64 + tid];
    ival[tid] = e;
    epart[tid] = e * p.cweight[tid + 1];
  } else if (tid < p.n_freq) {
    int q = tid;
    double e = 0.0;
    double tr_even[LMBD_MAX_ORDER_P1];
    for (int n = 2; n <= p.order; ++n) {
      double tr = red[n][3 * q] + red[n][3 * q + 1] + red[n][3 * q + 2];
      w.trbuf[((long long)c * (LMBD_MAX_ORDER_P1)) * 64 + n * 64 + q] = tr;
      e += series_c(w, p, c, q, n) * tr;
      tr_even[n] = tr;
    }
    // spectral proxy of the polarisation catastrophe (Sec. III.A: the series needs the
    // eigenvalues of G inside (-1, 1)): with M = floor(n_max / 2) >= 2, the traces
    // Tr[G^2M]_kk = |G^M e_k|^2 and Tr[G^(2M-2)]_kk = |G^(M-1) e_k|^2; their ratio tends to the
    // largest lambda^2 that the centre's block sees, and a ratio >= 1 is flagged
    const int M = p.order / 2;
    if (M >= 2 && tr_even[2 * M] >= tr_even[2 * M - 2]) atomicAdd(w.status + 1, 1);
    ival[q] = e;
    epart[q] = e * p.cweight[q + 1];
  }
  __syncthreads();
  if (tid == 0) {
    if (p.fit) {
      __shared__ FitScratch fs;
      w.energies[c] = fit_energy(fs, ival, p, w.fitw + (long long)c * LMBD_FITW, w.status);
    } else {
      double e = 0.0;
      for (int q = 0; q < p.n_freq; ++q) e += epart[q];
      w.energies[c] = e;
    }
  }
}

void launch_mbd_prepare_sized(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s) {
  if (c1 <= c0) return;
  size_t sm = sizeof(double) * 4 * (size_t)max_ns;
  raise_smem_limit((const void*)k_mbd_prepare, sm);
  k_mbd_prepare<<<c1 - c0, 256, sm, s>>>(w, p, c0, max_ns);
}

void launch_mbd_chain_sized(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, cudaStream_t s) {
  if (c1 <= c0) return;
  int tiles = (3 * max_ns + CH_R - 1) / CH_R;
  k_mbd_chain<<<(c1 - c0) * tiles, 256, 0, s>>>(w, p, m, c0, tiles);
}

void launch_mbd_energy(const Work& w, const DevParams& p, int c0, int c1, cudaStream_t s) {
  if (c1 <= c0) return;
  k_mbd_energy<<<c1 - c0, 256, 0, s>>>(w, p, c0);
}

// ---------------------------------------------------------------------------------------
// adjoint, part 1 (one block per central atom): dL/dalpha~ from the series, the factors
// P, Q of the pair matrix M' = P Q^T, and the central-column term X0
//   c~_{n,q} = w_k cw_q (-1/n)
//   a_j = sum_{l=1}^{n_max-1-j} c~_{j+l+1} v_l,  P_s = [D_qs v_j[s]],  Q_s = [D_qs a_j[s]]
//   X0_s = sum_q D_qs D_q0 sum_n c~_n v_{n-1}[s]
// ---------------------------------------------------------------------------------------
template <int NM, bool SPARSE>
__global__ void __launch_bounds__(256) k_mbd_adj_site(Work w, DevParams p, int c0) {
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns;
  const long long offs = w.off_s[c];
  const int ncv = 3 * p.n_freq;
  const int nm = NM;
  const double wk = w.weights ? w.weights[c] : 1.0;
  const int tid = threadIdx.x;
  const double* V0 = w.vkr + (offs * 3) * ncv;   // block of v_1, others at +vstride*(m-1)
  // per (site, frequency) work items; for each of the 9 entries of the site's 3 x 3 block at this
  // frequency the values v_1 .. v_{n_max-1} are read once into registers
  for (int e = tid; e < ns * p.n_freq; e += blockDim.x) {
    const int s = e / p.n_freq, qq = e % p.n_freq, q = qq + 1;
    const double cwq = p.fit ? w.fitw[(long long)c * LMBD_FITW + qq] : p.cweight[q];
    double ct[NM + 1];
#pragma unroll
    for (int n = 0; n <= NM; ++n) ct[n] = (n >= 2) ? wk * cwq * series_c(w, p, c, qq, n) : 0.0;
    if (SPARSE) {
      // block-sparse T_LR: the chain kept W_m = D v_m as float-float, so P_j = W_j,
      // Q_j = sum_l c~_{j+l+1} W_l and <v_j, v_l> = <W_j, W_l> / alpha~ run on the FP32 pipe
      const float2* W0 = w.wff + (offs * 3) * ncv;
      ff ctf[NM + 1], fo[NM + 1], fd[NM + 1];
#pragma unroll
      for (int n = 0; n <= NM; ++n) {
        ctf[n] = ff_from_double(ct[n]);
        fo[n] = fd[n] = ff_make(0.f, 0.f);
      }
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) {
        const int al = ab / 3, be = ab % 3;
        const long long idx = (long long)(3 * s + al) * ncv + 3 * qq + be;
        ff v[NM];
#pragma unroll
        for (int m = 1; m < NM; ++m) {
          const float2 t = W0[(long long)(m - 1) * w.vstride + idx];
          v[m] = ff_make(t.x, t.y);
        }
#pragma unroll
        for (int n = 2; n <= NM; ++n) {
#pragma unroll
          for (int j = 1; 2 * j < n; ++j) fo[n] = ff_fma(v[j], v[n - j], fo[n]);
          if (n % 2 == 0) fd[n] = ff_fma(v[n / 2], v[n / 2], fd[n]);
        }
#pragma unroll
        for (int j = 1; j <= NM - 2; ++j) {
          ff a = ff_make(0.f, 0.f);
#pragma unroll
          for (int l = 1; l <= NM - 1 - j; ++l) a = ff_fma(ctf[j + l + 1], v[l], a);
          const long long o = (offs * 3 + 3 * s + al) * (long long)w.ncol + (qq * (nm - 2) + (j - 1)) * 3 + be;
          w.pff[o] = make_float2(v[j].hi, v[j].lo);
          w.qff[o] = make_float2(a.hi, a.lo);
        }
      }
      const double ia = 1.0 / w.alphaT[(offs + s) * p.nq + q];
      double ga = 0.0;
#pragma unroll
      for (int n = 2; n <= NM; ++n) {
        double sum = ff_to_double(ff_add(ff_add(fo[n], fo[n]), fd[n])) * ia;
        if (s == 0) sum += w.trbuf[((long long)c * LMBD_MAX_ORDER_P1) * 64 + n * 64 + qq];
        ga += ct[n] * sum;
      }
      w.gbar[(offs + s) * p.nq + q] = ga * ia;
      continue;
    }
    // gs_n = sum_{j=1}^{n-1} <v_j[s], v_{n-j}[s]>: the pairs j < n - j once (doubled), j = n/2 once
    double go[NM + 1], gd[NM + 1];
#pragma unroll
    for (int n = 0; n <= NM; ++n) go[n] = gd[n] = 0.0;
    const double ds = w.dsq[(offs + s) * p.nq + q];
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) {
      const int al = ab / 3, be = ab % 3;
      const long long idx = (long long)(3 * s + al) * ncv + 3 * qq + be;
      double v[NM];   // v[m] = v_m, m = 1 .. n_max - 1
#pragma unroll
      for (int m = 1; m < NM; ++m) v[m] = V0[(long long)(m - 1) * w.vstride + idx];
#pragma unroll
      for (int n = 2; n <= NM; ++n) {
#pragma unroll
        for (int j = 1; 2 * j < n; ++j) go[n] += v[j] * v[n - j];
        if (n % 2 == 0) gd[n] += v[n / 2] * v[n / 2];
      }
      // P and Q columns of this frequency: P_j = D v_j, Q_j = D a_j, a_j = sum_l c~_{j+l+1} v_l
#pragma unroll
      for (int j = 1; j <= NM - 2; ++j) {
        double a = 0.0;
#pragma unroll
        for (int l = 1; l <= NM - 1 - j; ++l) a += ct[j + l + 1] * v[l];
        const long long o = (offs * 3 + 3 * s + al) * (long long)w.ncol + (qq * (nm - 2) + (j - 1)) * 3 + be;
        w.pmat[o] = ds * v[j];
        w.qmat[o] = ds * a;
      }
    }
    double ga = 0.0;
#pragma unroll
    for (int n = 2; n <= NM; ++n) {
      double sum = 2.0 * go[n] + gd[n];
      if (s == 0) sum += w.trbuf[((long long)c * LMBD_MAX_ORDER_P1) * 64 + n * 64 + qq];
      ga += ct[n] * sum;
    }
    w.gbar[(offs + s) * p.nq + q] = ga / w.alphaT[(offs + s) * p.nq + q];
  }
  __syncthreads();
  // X0_s (3 x 3) summed over frequencies
  for (int e = tid; e < ns * 9; e += blockDim.x) {
    int s = e / 9, al = (e % 9) / 3, be = e % 3;
    double acc = 0.0;
    for (int qq = 0; qq < p.n_freq; ++qq) {
      int q = qq + 1;
      double dd = w.dsq[(offs + s) * p.nq + q] * w.dsq[offs * p.nq + q];
      const double cwq = p.fit ? w.fitw[(long long)c * LMBD_FITW + qq] : p.cweight[q];
      double sum = 0.0;
      for (int n = 2; n <= nm; ++n)
        sum += wk * cwq * series_c(w, p, c, qq, n) * V0[(long long)(n - 2) * w.vstride + (long long)(3 * s + al) * ncv + 3 * qq + be];
      acc += dd * sum;
    }
    w.x0buf[(offs + s) * 9 + al * 3 + be] = acc;
  }
}

// ---------------------------------------------------------------------------------------
// adjoint, part 2: pair matrix M_st = (P Q^T)_st (+ X0_s if t = 0) on 16 x 16 site tiles
// of the lower triangle, contracted with dT_LR/dr (sites) and dT_LR/dS~ (SCS radii)
// ---------------------------------------------------------------------------------------
#define PT 16
#define PK 16

// Site positions and SCS radii of the row (bi) and column (bj) site blocks of a pair tile.
__device__ __forceinline__ void pair_tile_sites(const Work& w, const DevParams& p, long long offs, long long sbase,
                                                int ns, int bi, int bj, double (*xs)[PT][3], double (*rts)[PT]) {
  const int tid = threadIdx.x;
  if (tid < 2 * PT) {
    int side = tid / PT, l = tid % PT;
    int s = (side == 0 ? bi : bj) * PT + l;
    for (int d = 0; d < 3; ++d) xs[side][l][d] = s < ns ? w.site_x[3 * (sbase + s) + d] : 0.0;
    double rt = 1.0;
    if (s < ns) {
      int a = w.site_atom[sbase + s];
      rt = w.r0[a] * cbrt(w.alphaT[(offs + s) * p.nq] / w.a0[a]);
    }
    rts[side][l] = rt;
  }
}

// Deterministic reduction of the 16 x 16 pair results of a tile to its row sites (-g, seed)
// and column sites (+g, seed), then one global atomic per site.
__device__ __forceinline__ void pair_tile_reduce(const Work& w, long long offs, long long sbase, int ns, int bi,
                                                 int bj, double (*gp)[PT][4], int only_atom = -1) {
  const int tid = threadIdx.x;
  if (tid < 2 * PT) {
    const int side = tid / PT, l = tid % PT;
    const int ss = (side == 0 ? bi : bj) * PT + l;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0, sb = 0.0;
    for (int o = 0; o < PT; ++o) {
      const double* v = side == 0 ? gp[l][o] : gp[o][l];
      g0 += v[0];
      g1 += v[1];
      g2 += v[2];
      sb += v[3];
    }
    if (ss < ns) {
      const double sgn = side == 0 ? -1.0 : 1.0;
      const int a = w.site_atom[sbase + ss];
      if ((g0 != 0.0 || g1 != 0.0 || g2 != 0.0) && (only_atom < 0 || a == only_atom))
        atomic_add3(w.gacc + 3 * a, sgn * g0, sgn * g1, sgn * g2);
      if (sb != 0.0) atomicAdd(&w.rbar[offs + ss], sb);
    }
  }
}

__global__ void __launch_bounds__(256) k_mbd_adj_pair(Work w, DevParams p, int c0, int tiles_per_c) {
  __shared__ double Ps[3 * PT][PK + 1];
  __shared__ double Qs[3 * PT][PK + 1];
  __shared__ double xs[2][PT][3];
  __shared__ double rts[2][PT];
  __shared__ double gp[PT][PT][4];
  const int c = c0 + blockIdx.x / tiles_per_c;
  int tile = blockIdx.x % tiles_per_c;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns;
  const int nt = (ns + PT - 1) / PT;
  if (tile >= nt * (nt + 1) / 2) return;
  int bi = 0;
  while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
  const int bj = tile - bi * (bi + 1) / 2;
  const long long offs = w.off_s[c];
  const long long sbase = (long long)c * w.site_cap;
  const int tid = threadIdx.x;
  const int ty = tid / PT, tx = tid % PT;
  pair_tile_sites(w, p, offs, sbase, ns, bi, bj, xs, rts);
  const int s = bi * PT + ty, t = bj * PT + tx;
  double acc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  const int ncol = w.ncol;
  for (int k0 = 0; k0 < ncol; k0 += PK) {
    __syncthreads();
    for (int e = tid; e < 3 * PT * PK; e += blockDim.x) {
      int rr = e / PK, kk = e % PK;
      int gk = k0 + kk;
      int sr = bi * PT * 3 + rr, tr = bj * PT * 3 + rr;
      Ps[rr][kk] = (sr < 3 * ns && gk < ncol) ? w.pmat[(offs * 3 + sr) * (long long)ncol + gk] : 0.0;
      Qs[rr][kk] = (tr < 3 * ns && gk < ncol) ? w.qmat[(offs * 3 + tr) * (long long)ncol + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < PK; ++kk) {
      double a0 = Ps[3 * ty][kk], a1 = Ps[3 * ty + 1][kk], a2 = Ps[3 * ty + 2][kk];
      double b0 = Qs[3 * tx][kk], b1 = Qs[3 * tx + 1][kk], b2 = Qs[3 * tx + 2][kk];
      acc[0][0] += a0 * b0; acc[0][1] += a0 * b1; acc[0][2] += a0 * b2;
      acc[1][0] += a1 * b0; acc[1][1] += a1 * b1; acc[1][2] += a1 * b2;
      acc[2][0] += a2 * b0; acc[2][1] += a2 * b1; acc[2][2] += a2 * b2;
    }
  }
  __syncthreads();   // site data of the tile visible to all threads (also when ncol = 0)
  pair_epilogue(w, offs, w.off_t[c], s, t, ns, acc, gp[ty][tx]);
  __syncthreads();
  pair_tile_reduce(w, offs, sbase, ns, bi, bj, gp);
}

// ---------------------------------------------------------------------------------------
// adjoint, part 3 (one block per central atom): SCS-radius gradient into alpha~(0), then
// through the blend (Eq. full-pol) into alpha_K (local) and alpha_I (global, atomics)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mbd_adj_blend(Work w, DevParams p, int c0) {
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const Counts cn = w.counts[c];
  const int ns = cn.ns, n1 = cn.n1;
  const long long offs = w.off_s[c], offk1 = w.off_k1[c];
  const long long sbase = (long long)c * w.site_cap;
  const int tid = threadIdx.x;
  double g0[3] = {0.0, 0.0, 0.0};
  for (int s = tid; s < ns; s += blockDim.x) {
    int a = w.site_atom[sbase + s];
    double at0 = w.alphaT[(offs + s) * p.nq];
    double rt = w.r0[a] * cbrt(at0 / w.a0[a]);
    double gb0 = w.rbar[offs + s] * rt / (3.0 * at0);
    double x0 = w.site_x[3 * (sbase + s)], x1 = w.site_x[3 * (sbase + s) + 1], x2 = w.site_x[3 * (sbase + s) + 2];
    double fs = 0.0, dfs = 0.0, r = 0.0;
    if (s < n1 && s > 0) {
      r = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
      double u = r / p.r_scs;
      fs = 3.0 * u * u - 2.0 * u * u * u;
      dfs = (6.0 * u - 6.0 * u * u) / p.r_scs;
    }
    // dL/d alpha~ at the frequencies of the SCS solves
    double gs[LMBD_MAXQ];
    if (!p.lorentz) {
      for (int q = 0; q < p.nq; ++q) gs[q] = (q == 0) ? gb0 : w.gbar[(offs + s) * p.nq + q];
    } else {
      // reverse of the Lorentzian model: alpha~_q = a0 / D_q, D_q = 1 + u_q (a0/ar - 1),
      // d alpha~_q / d a0 = 1/D_q - a0 u_q / (ar D_q^2), d alpha~_q / d ar = a0^2 u_q / (ar^2 D_q^2)
      double ab[2];
      for (int qs = 0; qs < 2; ++qs) {
        const double aI = w.alphaI[(long long)a * 2 + qs];
        ab[qs] = (s < n1) ? (1.0 - fs) * w.alphaK[(offk1 + s) * 2 + qs] + fs * aI : aI;
      }
      const double a0 = ab[0], ar = ab[1];
      const double ratio = fmax(a0 / ar, 1.0);
      double g0 = gb0, g1 = 0.0;
      for (int q = 1; q < p.nq; ++q) {
        const double g = w.gbar[(offs + s) * p.nq + q];
        const double u = (p.omega[q] / p.omega_ref) * (p.omega[q] / p.omega_ref);
        const double D = 1.0 + u * (ratio - 1.0);
        g0 += g * (1.0 / D - a0 * u / (ar * D * D));
        g1 += g * (a0 * a0 * u / (ar * ar * D * D));
      }
      gs[0] = g0;
      gs[1] = g1;
    }
    double gr = 0.0;
    for (int q = 0; q < p.nqs; ++q) {
      const double g = gs[q];
      if (s < n1) {
        double aK = w.alphaK[(offk1 + s) * p.nqs + q];
        double aI = w.alphaI[(long long)a * p.nqs + q];
        w.alphaK_bar[(offk1 + s) * p.nqs + q] = (1.0 - fs) * g;
        if (fs != 0.0 && !p.paper) atomicAdd(&w.alphaI_bar[(long long)a * p.nqs + q], fs * g);
        gr += dfs * (aI - aK) * g;
      } else if (!p.paper) {             // the paper's forces hold alpha_I (Eq. full-pol-grad)
        atomicAdd(&w.alphaI_bar[(long long)a * p.nqs + q], g);
      }
    }
    if (s < n1 && s > 0 && gr != 0.0) {
      double ir = 1.0 / r;
      double gx = gr * x0 * ir, gy = gr * x1 * ir, gz = gr * x2 * ir;
      if (!p.paper || a == c) atomic_add3(w.gacc + 3 * a, gx, gy, gz);
      g0[0] -= gx; g0[1] -= gy; g0[2] -= gz;
    }
  }
  // the central site carries minus the sum of the f_SCS gradients
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int d = 0; d < 3; ++d) g0[d] += __shfl_xor_sync(0xffffffffu, g0[d], o);
  if ((tid & 31) == 0) atomic_add3(w.gacc + 3 * c, g0[0], g0[1], g0[2]);
}

// ---------------------------------------------------------------------------------------
// the paper's approximate forces (Sec. III.D, Eqs. mbd-forces and cent-appr): seeds of
//   L_k = w_k sum_q cw_q [ c_2 Tr G^2 + sum_{n>=3} c_n Tr G~^n ]   (Eq. E_k_tot, full traces)
// where G~ moves only in the row and column of the central site and alpha_I is held.  The
// reverse pass is the exact one from here on; position gradients are kept for the images of
// atom k only (F_k = -dL_k/dr_k).
//   two-body term:  dL/dalpha~_s = 2 c_2 cw sum_t alpha~_t |T_st|^2,
//                   pair block M_st = 2 c_2 cw alpha~_s alpha~_t T_st (one block of the pair);
//   central column: Z_s = sum_{n>=3} n c_n cw v_{n-1}[s], M_s0 += D_s D_0 Z_s,
//                   dL/dalpha~_s = <Z_s, v_1[s]> / alpha~_s (s > 0),
//                   dL/dalpha~_0 = sum_{n>=3} n c_n cw tr_n / alpha~_0.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_f3_site(Work w, DevParams p, int c0) {
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns, N = 3 * ns;
  const long long offs = w.off_s[c];
  const int ncv = 3 * p.n_freq, nm = p.order, nf = p.n_freq;
  const double wk = w.weights ? w.weights[c] : 1.0;
  const int tid = threadIdx.x;
  const double* T = w.tlr + w.off_t[c];
  const double* V0 = w.vkr + (offs * 3) * ncv;   // v_1, then v_m at +vstride (m - 1)
  // two-body term, eight frequencies per pass over the rows of T
  for (int s = tid; s < ns; s += blockDim.x) {
    for (int q0 = 0; q0 < nf; q0 += 8) {
      double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int t = 0; t < ns; ++t) {
        if (t == s) continue;
        double n2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const double v = T[(long long)(3 * s + a) * N + 3 * t + b];
            n2 += v * v;
          }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (q0 + j < nf) acc[j] += w.alphaT[(offs + t) * p.nq + q0 + j + 1] * n2;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (q0 + j < nf) {
          const int qq = q0 + j, q = qq + 1;
          w.gbar[(offs + s) * p.nq + q] = 2.0 * series_c(w, p, c, qq, 2) * wk * p.cweight[q] * acc[j];
        }
    }
  }
  __syncthreads();
  // central row and column, n >= 3
  for (int e = tid; e < ns * nf; e += blockDim.x) {
    const int s = e / nf, qq = e % nf, q = qq + 1;
    const double cwq = wk * p.cweight[q];
    double g = 0.0;
    if (s == 0) {
      for (int n = 3; n <= nm; ++n)
        g += n * series_c(w, p, c, qq, n) * cwq * w.trbuf[((long long)c * LMBD_MAX_ORDER_P1) * 64 + n * 64 + qq];
    } else {
      for (int n = 3; n <= nm; ++n) {
        const double* Va = V0 + (long long)(n - 2) * w.vstride;
        double d = 0.0;
        for (int al = 0; al < 3; ++al)
          for (int be = 0; be < 3; ++be) {
            const long long idx = (long long)(3 * s + al) * ncv + 3 * qq + be;
            d += Va[idx] * V0[idx];
          }
        g += n * series_c(w, p, c, qq, n) * cwq * d;
      }
    }
    w.gbar[(offs + s) * p.nq + q] += g / w.alphaT[(offs + s) * p.nq + q];
  }
  // X0_s = sum_q D_qs D_q0 Z_s, the central-column block of the pair matrix
  for (int e = tid; e < ns * 9; e += blockDim.x) {
    const int s = e / 9, al = (e % 9) / 3, be = e % 3;
    double acc = 0.0;
    for (int qq = 0; qq < nf; ++qq) {
      const int q = qq + 1;
      const double dd = w.dsq[(offs + s) * p.nq + q] * w.dsq[offs * p.nq + q];
      const double cwq = wk * p.cweight[q];
      double z = 0.0;
      for (int n = 3; n <= nm; ++n)
        z += n * series_c(w, p, c, qq, n) * cwq *
             V0[(long long)(n - 2) * w.vstride + (long long)(3 * s + al) * ncv + 3 * qq + be];
      acc += dd * z;
    }
    w.x0buf[(offs + s) * 9 + al * 3 + be] = acc;
  }
}

// Two-body pair blocks M_st = gamma_st T_LR,st, gamma_st = sum_q 2 c_2 cw_q alpha~_qs alpha~_qt,
// plus the central column, contracted with the stored pair coefficients (pair_epilogue).
__global__ void __launch_bounds__(256) k_f3_pair(Work w, DevParams p, int c0, int tiles_per_c) {
  __shared__ double alt[2][PT][LMBD_MAXQ - 1];
  __shared__ double cq[LMBD_MAXQ - 1];
  __shared__ double gp[PT][PT][4];
  const int c = c0 + blockIdx.x / tiles_per_c;
  int tile = blockIdx.x % tiles_per_c;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns;
  const int nt = (ns + PT - 1) / PT;
  if (tile >= nt * (nt + 1) / 2) return;
  int bi = 0;
  while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
  const int bj = tile - bi * (bi + 1) / 2;
  const long long offs = w.off_s[c];
  const long long sbase = (long long)c * w.site_cap;
  const int tid = threadIdx.x;
  const int ty = tid / PT, tx = tid % PT;
  const int nf = p.n_freq;
  const double wk = w.weights ? w.weights[c] : 1.0;
  for (int e = tid; e < 2 * PT * nf; e += blockDim.x) {
    const int side = e / (PT * nf), l = (e / nf) % PT, qq = e % nf;
    const int site = (side == 0 ? bi : bj) * PT + l;
    alt[side][l][qq] = site < ns ? w.alphaT[(offs + site) * p.nq + qq + 1] : 0.0;
  }
  for (int qq = tid; qq < nf; qq += blockDim.x) cq[qq] = 2.0 * series_c(w, p, c, qq, 2) * wk * p.cweight[qq + 1];
  __syncthreads();
  const int s = bi * PT + ty, t = bj * PT + tx;
  double acc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (s < ns && t < ns && s > t) {
    double gamma = 0.0;
    for (int qq = 0; qq < nf; ++qq) gamma += cq[qq] * alt[0][ty][qq] * alt[1][tx][qq];
    const double* pc = w.pcoef + w.off_t[c] + 8LL * (s * (s - 1) / 2 + t);
    const double rr[3] = {pc[0], pc[1], pc[2]};
    const double r2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
    const double cg = gamma * pc[5] / 12.0;      // pc[5] = 12 f_LR f / r^5
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) acc[a][b] = cg * (3.0 * rr[a] * rr[b] - (a == b ? r2 : 0.0));
  }
  pair_epilogue(w, offs, w.off_t[c], s, t, ns, acc, gp[ty][tx]);
  __syncthreads();
  pair_tile_reduce(w, offs, sbase, ns, bi, bj, gp, c);
}

void launch_paper_force_seeds(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s) {
  if (c1 <= c0) return;
  k_f3_site<<<c1 - c0, 256, 0, s>>>(w, p, c0);
  const int nt = (max_ns + PT - 1) / PT;
  const int tiles = nt * (nt + 1) / 2;
  k_f3_pair<<<(c1 - c0) * tiles, 256, 0, s>>>(w, p, c0, tiles);
}

void launch_mbd_adj_series(const Work& w, const DevParams& p, int c0, int c1, cudaStream_t s) {
  if (c1 <= c0) return;
  switch (p.order) {   // series order n_max: 2 .. LMBD_MAX_ORDER_P1 - 1
#define ADJ_SITE_CASE(N)                                                \
  case N:                                                               \
    if (w.wff)                                                          \
      k_mbd_adj_site<N, true><<<c1 - c0, 256, 0, s>>>(w, p, c0);        \
    else                                                                \
      k_mbd_adj_site<N, false><<<c1 - c0, 256, 0, s>>>(w, p, c0);       \
    break;
    ADJ_SITE_CASE(2) ADJ_SITE_CASE(3) ADJ_SITE_CASE(4) ADJ_SITE_CASE(5) ADJ_SITE_CASE(6)
    ADJ_SITE_CASE(7) ADJ_SITE_CASE(8) ADJ_SITE_CASE(9) ADJ_SITE_CASE(10)
#undef ADJ_SITE_CASE
    default: break;
  }
}

void launch_mbd_adj_pair(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s) {
  if (c1 <= c0) return;
  int nt = (max_ns + PT - 1) / PT;
  int tiles = nt * (nt + 1) / 2;
  k_mbd_adj_pair<<<(c1 - c0) * tiles, 256, 0, s>>>(w, p, c0, tiles);
}

void launch_mbd_adj_blend(const Work& w, const DevParams& p, int c0, int c1, cudaStream_t s) {
  if (c1 <= c0) return;
  k_mbd_adj_blend<<<c1 - c0, 256, 0, s>>>(w, p, c0);
}

void launch_mbd_adjoint_sized(const Work& w, const DevParams& p, int c0, int c1, int max_ns,
                              cudaStream_t s, int* launches) {
  launch_mbd_adj_series(w, p, c0, c1, s);
  launch_mbd_adj_pair(w, p, c0, c1, max_ns, s);
  launch_mbd_adj_blend(w, p, c0, c1, s);
  *launches += 3;
}

__global__ void k_forces_out(Work w, double* forces) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * w.n_atoms) return;
  forces[i] = -w.gacc[i] * (1.0 / LMBD_BOHR);
}

void launch_forces_out(const Work& w, double* forces, cudaStream_t s) {
  if (w.n_atoms == 0) return;
  k_forces_out<<<(3 * w.n_atoms + 255) / 256, 256, 0, s>>>(w, forces);
}

// =======================================================================================
// Sliced tensor-core products (ozaki.cuh): the Krylov chain T W and the pair matrix P Q^T
// evaluated from 7-bit digit planes on bf16 mma.sync, combined in FP64.
// Per central atom (N = 3 ns): T digit planes [Mpad][Kpad] with Mpad = 64 ceil(N/64),
// Kpad = 16 ceil(N/16); W^T digit planes [48][Kpad]; P and Q digit planes [3 ns16][Kp] with
// ns16 = 16 ceil(ns/16) and Kp = 16 ceil(ncol/16).
// =======================================================================================
__device__ __forceinline__ int oz_mpad(int n) { return (n + 63) / 64 * 64; }
__device__ __forceinline__ int oz_kpad(int n) { return (n + 15) / 16 * 16; }

// T_LR digit planes and row exponents (one block per central atom, one warp per row).  Rows of
// at most 32 SLT_REG entries are read once into registers; longer rows are read twice.
#define SLT_REG 18
template <int st>
__global__ void __launch_bounds__(256) k_slice_t(Work w, int c0) {
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const int N = 3 * w.counts[c].ns, Mpad = oz_mpad(N), Kpad = oz_kpad(N);
  const double* T = w.tlr + w.off_t[c];
  // row pitch: the centre's Kpad, or the common pitch tk of the tcgen05 path (zeros past N)
  const int ld = w.tk > 0 ? w.tk : Kpad;
  unsigned short* base = w.tk > 0 ? w.tdig + w.off_tr[c] * st * w.tk : w.tdig + w.off_tq[c] * st;
  const long long plane = (long long)Mpad * ld;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (N <= 32 * SLT_REG) {
    // one read of T: the row stays in registers between its exponent and its digits
    for (int row = warp; row < Mpad; row += nw) {
      double v[SLT_REG];
      int mx = 0;
#pragma unroll
      for (int k = 0; k < SLT_REG; ++k) {
        const int j = lane + 32 * k;
        v[k] = (row < N && j < N) ? T[(long long)row * N + j] : 0.0;
        mx = max(mx, oz_biased_exp(v[k]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int e = oz_scale_exp(mx);
      if (lane == 0) w.texp[w.off_tr[c] + row] = e;
#pragma unroll
      for (int k = 0; k < SLT_REG; ++k) {
        const int j = lane + 32 * k;
        if (j < ld) oz_store_digits<st>(base + (long long)row * ld + j, plane, v[k], e);
      }
      for (int j = lane + 32 * SLT_REG; j < ld; j += 32) oz_store_digits<st>(base + (long long)row * ld + j, plane, 0.0, e);
    }
    return;
  }
  for (int row = warp; row < Mpad; row += nw) {
    int mx = 0;
    if (row < N)
      for (int j = lane; j < N; j += 32) mx = max(mx, oz_biased_exp(T[(long long)row * N + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = oz_scale_exp(mx);
    if (lane == 0) w.texp[w.off_tr[c] + row] = e;
    for (int j = lane; j < ld; j += 32) {
      const double v = (row < N && j < N) ? T[(long long)row * N + j] : 0.0;
      oz_store_digits<st>(base + (long long)row * ld + j, plane, v, e);
    }
  }
}

// W = D v_m digit planes (stored by column) and column exponents (one block per atom).
template <int sw>
__global__ void __launch_bounds__(256) k_slice_w(Work w, DevParams p, int m, int c0) {
  __shared__ int cmax[48];
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const int N = 3 * w.counts[c].ns, Kpad = oz_kpad(N);
  const long long offs = w.off_s[c];
  const int ncv = 3 * p.n_freq;
  const double* Vin = w.vkr + (long long)(m - 1) * w.vstride + (offs * 3) * ncv;
  const double* dsq = w.dsq + offs * p.nq;
  const int ld = w.tk > 0 ? w.tk : Kpad;
  unsigned short* base = w.tk > 0 ? w.wdig + (long long)c * 48 * sw * w.tk : w.wdig + w.off_kp[c] * 48 * sw;
  const long long plane = 48LL * ld;
  const int tid = threadIdx.x;
  if (tid < 48) cmax[tid] = 0;
  __syncthreads();
  for (int e = tid; e < N * ncv; e += blockDim.x) {
    const int j = e / ncv, col = e % ncv;
    const double v = dsq[(j / 3) * p.nq + col / 3 + 1] * Vin[(long long)j * ncv + col];
    atomicMax(&cmax[col], oz_biased_exp(v));
  }
  __syncthreads();
  if (tid < 48) w.wexp[(long long)c * 48 + tid] = oz_scale_exp(cmax[tid]);
  for (int e = tid; e < 48 * ld; e += blockDim.x) {
    const int col = e / ld, j = e % ld;
    double v = 0.0;
    if (col < ncv && j < N) v = dsq[(j / 3) * p.nq + col / 3 + 1] * Vin[(long long)j * ncv + col];
    oz_store_digits<sw>(base + (long long)col * ld + j, plane, v, oz_scale_exp(cmax[col]));
  }
}

// P and Q digit planes and row exponents (blockIdx.y = 0: P, 1: Q); rows of at most 32 SLP_REG
// columns are read once into registers.
#define SLP_REG 6
template <int sp>
__global__ void __launch_bounds__(256) k_slice_pq(Work w, int c0) {
  const int c = c0 + blockIdx.x;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns, R = 3 * ((ns + 15) / 16 * 16), rows = 3 * ns;
  const int ncol = w.ncol, Kp = oz_kpad(ncol);
  const long long offs = w.off_s[c];
  const double* src = (blockIdx.y == 0 ? w.pmat : w.qmat) + offs * 3 * (long long)ncol;
  unsigned short* base = (blockIdx.y == 0 ? w.pdig : w.qdig) + w.off_sp[c] * 3 * (long long)Kp * sp;
  int* ex = (blockIdx.y == 0 ? w.pexp : w.qexp) + w.off_sp[c] * 3;
  const long long plane = (long long)R * Kp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (ncol <= 32 * SLP_REG) {
    // one read of P or Q: the row stays in registers between its exponent and its digits
    for (int row = warp; row < R; row += nw) {
      double v[SLP_REG];
      int mx = 0;
#pragma unroll
      for (int k = 0; k < SLP_REG; ++k) {
        const int j = lane + 32 * k;
        v[k] = (row < rows && j < ncol) ? src[(long long)row * ncol + j] : 0.0;
        mx = max(mx, oz_biased_exp(v[k]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int e = oz_scale_exp(mx);
      if (lane == 0) ex[row] = e;
#pragma unroll
      for (int k = 0; k < SLP_REG; ++k) {
        const int j = lane + 32 * k;
        if (j < Kp) oz_store_digits<sp>(base + (long long)row * Kp + j, plane, v[k], e);
      }
      for (int j = lane + 32 * SLP_REG; j < Kp; j += 32) oz_store_digits<sp>(base + (long long)row * Kp + j, plane, 0.0, e);
    }
    return;
  }
  for (int row = warp; row < R; row += nw) {
    int mx = 0;
    if (row < rows)
      for (int j = lane; j < ncol; j += 32) mx = max(mx, oz_biased_exp(src[(long long)row * ncol + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = oz_scale_exp(mx);
    if (lane == 0) ex[row] = e;
    for (int j = lane; j < Kp; j += 32) {
      const double v = (row < rows && j < ncol) ? src[(long long)row * ncol + j] : 0.0;
      oz_store_digits<sp>(base + (long long)row * Kp + j, plane, v, e);
    }
  }
}

// Slicing launches for the digit counts in use (4 to 7; the products use 5 and 6).
static void run_slice_t(const Work& w, int c0, int n, int st, cudaStream_t s) {
  switch (st) {
    case 4: k_slice_t<4><<<n, 256, 0, s>>>(w, c0); break;
    case 5: k_slice_t<5><<<n, 256, 0, s>>>(w, c0); break;
    case 6: k_slice_t<6><<<n, 256, 0, s>>>(w, c0); break;
    default: k_slice_t<7><<<n, 256, 0, s>>>(w, c0); break;
  }
}
static void run_slice_w(const Work& w, const DevParams& p, int m, int c0, int n, int sw, cudaStream_t s) {
  switch (sw) {
    case 4: k_slice_w<4><<<n, 256, 0, s>>>(w, p, m, c0); break;
    case 5: k_slice_w<5><<<n, 256, 0, s>>>(w, p, m, c0); break;
    case 6: k_slice_w<6><<<n, 256, 0, s>>>(w, p, m, c0); break;
    default: k_slice_w<7><<<n, 256, 0, s>>>(w, p, m, c0); break;
  }
}
static void run_slice_pq(const Work& w, int c0, int n, int sp, cudaStream_t s) {
  const dim3 g2(n, 2);
  switch (sp) {
    case 4: k_slice_pq<4><<<g2, 256, 0, s>>>(w, c0); break;
    case 5: k_slice_pq<5><<<g2, 256, 0, s>>>(w, c0); break;
    case 6: k_slice_pq<6><<<g2, 256, 0, s>>>(w, c0); break;
    default: k_slice_pq<7><<<g2, 256, 0, s>>>(w, c0); break;
  }
}

void launch_slice_t(const Work& w, int c0, int c1, int st, cudaStream_t s) {
  if (c1 <= c0) return;
  run_slice_t(w, c0, c1 - c0, st, s);
}

void launch_slice_pq(const Work& w, int c0, int c1, int digits, cudaStream_t s) {
  if (c1 <= c0) return;
  run_slice_pq(w, c0, c1 - c0, digits, s);
}

void launch_slice_w(const Work& w, const DevParams& p, int m, int c0, int c1, int digits, cudaStream_t s) {
  if (c1 <= c0) return;
  run_slice_w(w, p, m, c0, c1 - c0, digits, s);
}

// v_{m+1} = D (T W) with shared-memory staging (cp.async, two stages of 32 K), 64 x 48 outputs
// per block, 12 warps of 16 x 16, integer recombination of the digit groups.
#define OZ_KS 32
#define OZ_LD 40
template <int S>
__global__ void __launch_bounds__(384, 1) k_chain_oz2(Work w, DevParams p, int m, int c0, int tiles_per_c, int st) {
  extern __shared__ __align__(16) unsigned short oz_sm[];
  const int c = c0 + blockIdx.x / tiles_per_c;
  const int tile = blockIdx.x % tiles_per_c;
  if (c >= w.n_atoms) return;
  const int N = 3 * w.counts[c].ns, Mpad = oz_mpad(N), Kpad = oz_kpad(N);
  if (tile * 64 >= N) return;
  const long long offs = w.off_s[c];
  const int ncv = 3 * p.n_freq;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  const int wr = warp / 3, wc = warp % 3;
  const int stA = S * 64 * OZ_LD, stB = S * 48 * OZ_LD;
  unsigned short* sbuf[2] = {oz_sm, oz_sm + stA + stB};
  const unsigned short* gA = w.tdig + w.off_tq[c] * st + (long long)(tile * 64) * Kpad;
  const unsigned short* gB = w.wdig + w.off_kp[c] * 48 * S;
  const long long pA = (long long)Mpad * Kpad, pB = 48LL * Kpad;
  const int nstage = (Kpad + OZ_KS - 1) / OZ_KS;
  auto load = [&](int stage, int buf) {
    const int k0 = stage * OZ_KS;
    unsigned short* sA = sbuf[buf];
    unsigned short* sB = sA + stA;
    for (int e = tid; e < S * 64 * 4 + S * 48 * 4; e += blockDim.x) {
      const unsigned short* src;
      unsigned short* dst;
      int q;
      if (e < S * 64 * 4) {
        const int k = e / 256, r = (e >> 2) & 63;
        q = e & 3;
        src = gA + k * pA + (long long)r * Kpad + k0 + 8 * q;
        dst = sA + (k * 64 + r) * OZ_LD + 8 * q;
      } else {
        const int e2 = e - S * 256, k = e2 / 192, r = (e2 >> 2) % 48;
        q = e2 & 3;
        src = gB + k * pB + (long long)r * Kpad + k0 + 8 * q;
        dst = sB + (k * 48 + r) * OZ_LD + 8 * q;
      }
      const bool ok = k0 + 8 * q < Kpad;
      oz_cp_async16(dst, ok ? src : gA, ok ? 16 : 0);
    }
    oz_cp_commit();
  };
  float acc[S][2][4];
  long long Y[2][4];
#pragma unroll
  for (int a = 0; a < S; ++a)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[a][nt][v] = 0.f;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int v = 0; v < 4; ++v) Y[nt][v] = 0;
  load(0, 0);
  for (int sidx = 0; sidx < nstage; ++sidx) {
    if (sidx + 1 < nstage) {
      load(sidx + 1, (sidx + 1) & 1);
      oz_cp_wait<1>();
    } else {
      oz_cp_wait<0>();
    }
    __syncthreads();
    const unsigned short* sA = sbuf[sidx & 1];
    const unsigned short* sB = sA + stA;
#pragma unroll
    for (int kk = 0; kk < OZ_KS; kk += 16)
      oz_warp_k16_smem<S>(sA, 64 * OZ_LD, OZ_LD, wr * 16, sB, 48 * OZ_LD, OZ_LD, wc * 16, kk, acc);
    __syncthreads();
    if (((sidx + 1) * OZ_KS) % OZ_KCHUNK == 0 || sidx + 1 == nstage) oz_int_combine<S>(acc, Y);
  }
  double* Vout = w.vkr + (long long)m * w.vstride + (offs * 3) * ncv;
  const double* dsq = w.dsq + offs * p.nq;
  const int r0 = tile * 64 + wr * 16, cb = wc * 16;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int row = r0 + g + (v >> 1) * 8, col = cb + nt * 8 + 2 * tq + (v & 1);
      if (row < N && col < ncv) {
        const int er = w.texp[w.off_tr[c] + row], ec = w.wexp[(long long)c * 48 + col];
        const double y = (double)Y[nt][v] * oz_pow2(er + ec - 7 * (S + 1));
        Vout[(long long)row * ncv + col] = dsq[(row / 3) * p.nq + col / 3 + 1] * y;
      }
    }
}

void launch_chain_oz2(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, int digits, int st,
                      cudaStream_t s) {
  if (c1 <= c0) return;
  run_slice_w(w, p, m, c0, c1 - c0, digits, s);
  const int tiles = (3 * max_ns + 63) / 64;
  if (digits == 6) {
    const size_t sm = 2 * sizeof(unsigned short) * (6 * 64 + 6 * 48) * OZ_LD;
    raise_smem_limit((const void*)k_chain_oz2<6>, sm);
    k_chain_oz2<6><<<(c1 - c0) * tiles, 384, sm, s>>>(w, p, m, c0, tiles, st);
  } else {
    const size_t sm = 2 * sizeof(unsigned short) * (5 * 64 + 5 * 48) * OZ_LD;
    raise_smem_limit((const void*)k_chain_oz2<5>, sm);
    k_chain_oz2<5><<<(c1 - c0) * tiles, 384, sm, s>>>(w, p, m, c0, tiles, st);
  }
}

// Pair matrix M' = P Q^T on one 16 x 16 site tile with staged digit tiles (cp.async, two
// stages of 32 K) and integer recombination; 9 warps of 16 x 16 outputs, then the per-pair
// epilogue of the FP64 kernel.
template <int S>
__global__ void __launch_bounds__(288) k_mbd_adj_pair_oz2(Work w, DevParams p, int c0, int tiles_per_c) {
  extern __shared__ __align__(16) unsigned short oz_sm[];
  __shared__ double xs[2][PT][3];
  __shared__ double rts[2][PT];
  __shared__ double gp[PT][PT][4];
  const int c = c0 + blockIdx.x / tiles_per_c;
  const int tile = blockIdx.x % tiles_per_c;
  if (c >= w.n_atoms) return;
  const int ns = w.counts[c].ns;
  const int nt = (ns + PT - 1) / PT;
  if (tile >= nt * (nt + 1) / 2) return;
  int bi = 0;
  while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
  const int bj = tile - bi * (bi + 1) / 2;
  const long long offs = w.off_s[c];
  const long long sbase = (long long)c * w.site_cap;
  const int tid = threadIdx.x;
  pair_tile_sites(w, p, offs, sbase, ns, bi, bj, xs, rts);
  const int R = 3 * nt * PT, Kp = oz_kpad(w.ncol);
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  const int wr = warp / 3, wc = warp % 3;
  const long long dbase = w.off_sp[c] * 3 * (long long)Kp * S;
  const unsigned short* gA = w.pdig + dbase + (long long)(bi * 48) * Kp;
  const unsigned short* gB = w.qdig + dbase + (long long)(bj * 48) * Kp;
  const long long pl = (long long)R * Kp;
  const int st = S * 48 * OZ_LD;
  unsigned short* sbuf[2] = {oz_sm, oz_sm + 2 * st};
  const int nstage = (Kp + OZ_KS - 1) / OZ_KS;
  auto load = [&](int stage, int buf) {
    const int k0 = stage * OZ_KS;
    unsigned short* sA = sbuf[buf];
    unsigned short* sB = sA + st;
    for (int e = tid; e < 2 * S * 48 * 4; e += blockDim.x) {
      const int side = e / (S * 192), e2 = e % (S * 192), k = e2 / 192, r = (e2 >> 2) % 48, q = e2 & 3;
      const unsigned short* src = (side == 0 ? gA : gB) + k * pl + (long long)r * Kp + k0 + 8 * q;
      unsigned short* dst = (side == 0 ? sA : sB) + (k * 48 + r) * OZ_LD + 8 * q;
      const bool ok = k0 + 8 * q < Kp;
      oz_cp_async16(dst, ok ? src : gA, ok ? 16 : 0);
    }
    oz_cp_commit();
  };
  float acc[S][2][4];
  long long Y[2][4];
#pragma unroll
  for (int a = 0; a < S; ++a)
#pragma unroll
    for (int n8 = 0; n8 < 2; ++n8)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[a][n8][v] = 0.f;
#pragma unroll
  for (int n8 = 0; n8 < 2; ++n8)
#pragma unroll
    for (int v = 0; v < 4; ++v) Y[n8][v] = 0;
  load(0, 0);
  for (int sidx = 0; sidx < nstage; ++sidx) {
    if (sidx + 1 < nstage) {
      load(sidx + 1, (sidx + 1) & 1);
      oz_cp_wait<1>();
    } else {
      oz_cp_wait<0>();
    }
    __syncthreads();
    const unsigned short* sA = sbuf[sidx & 1];
    const unsigned short* sB = sA + st;
#pragma unroll
    for (int kk = 0; kk < OZ_KS; kk += 16)
      oz_warp_k16_smem<S>(sA, 48 * OZ_LD, OZ_LD, wr * 16, sB, 48 * OZ_LD, OZ_LD, wc * 16, kk, acc);
    __syncthreads();
    if (((sidx + 1) * OZ_KS) % OZ_KCHUNK == 0 || sidx + 1 == nstage) oz_int_combine<S>(acc, Y);
  }
  // FP64 pair matrix of the tile in shared memory (reuses the staging buffer)
  double* Ms = reinterpret_cast<double*>(oz_sm);
  const int* pe = w.pexp + w.off_sp[c] * 3;
  const int* qe = w.qexp + w.off_sp[c] * 3;
#pragma unroll
  for (int n8 = 0; n8 < 2; ++n8)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int rr = wr * 16 + g + (v >> 1) * 8, cc = wc * 16 + n8 * 8 + 2 * tq + (v & 1);
      Ms[rr * 49 + cc] = (double)Y[n8][v] * oz_pow2(pe[bi * 48 + rr] + qe[bj * 48 + cc] - 7 * (S + 1));
    }
  __syncthreads();
  if (tid < PT * PT) {
    const int ty = tid / PT, tx = tid % PT;
    const int s = bi * PT + ty, t = bj * PT + tx;
    double a3[3][3];
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
      for (int be = 0; be < 3; ++be) a3[al][be] = Ms[(3 * ty + al) * 49 + 3 * tx + be];
    pair_epilogue(w, offs, w.off_t[c], s, t, ns, a3, gp[ty][tx]);
  }
  __syncthreads();
  pair_tile_reduce(w, offs, sbase, ns, bi, bj, gp);
}

void launch_mbd_adj_pair_oz2(const Work& w, const DevParams& p, int c0, int c1, int max_ns, int digits,
                             cudaStream_t s) {
  if (c1 <= c0) return;
  run_slice_pq(w, c0, c1 - c0, digits, s);
  const int nt = (max_ns + PT - 1) / PT;
  const int tiles = nt * (nt + 1) / 2;
  if (digits == 6) {
    const size_t sm = 2 * 2 * sizeof(unsigned short) * 6 * 48 * OZ_LD;
    raise_smem_limit((const void*)k_mbd_adj_pair_oz2<6>, sm);
    k_mbd_adj_pair_oz2<6><<<(c1 - c0) * tiles, 288, sm, s>>>(w, p, c0, tiles);
  } else {
    const size_t sm = 2 * 2 * sizeof(unsigned short) * 5 * 48 * OZ_LD;
    raise_smem_limit((const void*)k_mbd_adj_pair_oz2<5>, sm);
    k_mbd_adj_pair_oz2<5><<<(c1 - c0) * tiles, 288, sm, s>>>(w, p, c0, tiles);
  }
}
