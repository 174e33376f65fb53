// Stage 1 in FP64 for the allocation-free entry point (lmbd_central_polarizabilities_noalloc):
// local self-consistent screening (Sec. III.B, Eq. local_pol) for every central atom k and
// frequency omega_q (q = 0 is omega = 0):
//   B_K = diag(1/alpha_bar_i) + T_SR,K,ij     (i, j in K1, Eq. local_pol)
//   d_K,i = 1 - sum_{j in K2} T_SR,K,ij alpha_bar_j
//   X = B_K^-1 d_K  (3 n1 x 3), alpha_K,i = Tr(X_i)/3, alpha_I,k = alpha_K,k
// T_SR,K,ij = f_inner f_SR (1 - f(r, S_ij)) (-T g + h) (Eqs. T_SR, g-func, h-func), factorised
// with an FP64 blocked Cholesky.  The main path (k_scs2.cu) solves the same systems in mixed
// precision.
#include "lmbd_internal.cuh"

#define NB 16
#define PS 17  // padded panel stride (doubles)

// ---------------------------------------------------------------------------------------
// dense helpers for one thread block (blockDim.x == 256)
// ---------------------------------------------------------------------------------------
// In-place right-looking blocked Cholesky of the lower triangle of A (n x n, row-major,
// leading dimension n) in global memory.  panel: (n) x PS doubles of shared memory,
// dg: NB x PS, inv: n doubles (receives 1/L_ii).  Returns via *bad a flag if a pivot
// was not positive (the pivot is then replaced by 1 so that the factor stays finite).
__device__ void block_cholesky(double* A, int n, double* panel, double* dg, double* inv, int* bad) {
  const int tid = threadIdx.x;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    // (1) diagonal block into shared memory and factor it with one warp
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      int i = e / kb, j = e % kb;
      if (j <= i) dg[i * PS + j] = A[(long long)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    if (tid < 32) {
      for (int t = 0; t < kb; ++t) {
        if (tid == 0) {
          double dv = dg[t * PS + t];
          if (!(dv > 0.0)) { *bad = 1; dv = 1.0; }
          double sq = sqrt(dv);
          dg[t * PS + t] = sq;
          inv[k0 + t] = 1.0 / sq;
        }
        __syncwarp();
        double it = inv[k0 + t];
        if (tid > t && tid < kb) dg[tid * PS + t] *= it;
        __syncwarp();
        for (int e = tid; e < kb * kb; e += 32) {
          int i = e / kb, j = e % kb;
          if (j > t && j <= i) dg[i * PS + j] -= dg[i * PS + t] * dg[j * PS + t];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = tid; e < kb * kb; e += blockDim.x) {
      int i = e / kb, j = e % kb;
      if (j <= i) A[(long long)(k0 + i) * n + k0 + j] = dg[i * PS + j];
    }
    // (2) panel below the diagonal block: L21 = A21 L11^-T, one row per thread
    const int r0 = k0 + kb;
    const int m = n - r0;
    for (int r = tid; r < m; r += blockDim.x) {
      const double* arow = A + (long long)(r0 + r) * n + k0;
      double v[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) v[t] = t < kb ? arow[t] : 0.0;
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        if (t < kb) {
          double s = v[t];
#pragma unroll
          for (int u = 0; u < t; ++u) s -= v[u] * dg[t * PS + u];
          v[t] = s * inv[k0 + t];
        }
      }
      double* wrow = A + (long long)(r0 + r) * n + k0;
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (t < kb) { panel[r * PS + t] = v[t]; wrow[t] = v[t]; }
    }
    __syncthreads();
    // (3) trailing update A22 -= L21 L21^T on the lower triangle, 16x16 tiles
    const int nt = (m + 15) / 16;
    const int ty = tid / 16, tx = tid % 16;
    for (int tile = 0; tile < nt * (nt + 1) / 2; ++tile) {
      // tile -> (bi, bj) with bj <= bi
      int bi = (int)((sqrtf(8.0f * tile + 1.0f) - 1.0f) * 0.5f);
      while (bi * (bi + 1) / 2 > tile) --bi;
      while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
      int bj = tile - bi * (bi + 1) / 2;
      int i = bi * 16 + ty, j = bj * 16 + tx;
      if (i < m && j <= i) {
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < kb) s += panel[i * PS + t] * panel[j * PS + t];
        A[(long long)(r0 + i) * n + r0 + j] -= s;
      }
    }
    __syncthreads();
  }
}

// Solve L L^T X = Y in place for 3 right-hand sides; Y is n x 3 in shared memory,
// L the lower factor in global memory, inv[i] = 1/L_ii.  red: 256 x 3 doubles scratch.
__device__ void block_solve3(const double* L, int n, const double* inv, double* Y, double* red) {
  const int tid = threadIdx.x;
  const int r = tid / 16, s = tid % 16;      // 16 rows x 16 partial sums
  // forward: L Z = Y
  for (int b0 = 0; b0 < n; b0 += 16) {
    const int bb = min(16, n - b0);
    double acc[3] = {0.0, 0.0, 0.0};
    if (r < bb) {
      const double* lrow = L + (long long)(b0 + r) * n;
      for (int t = s; t < b0; t += 16) {
        double l = lrow[t];
        acc[0] += l * Y[3 * t + 0];
        acc[1] += l * Y[3 * t + 1];
        acc[2] += l * Y[3 * t + 2];
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o, 16);
    if (s == 0 && r < bb)
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[3 * (b0 + r) + c] -= acc[c];
    __syncthreads();
    if (tid < 32) {
      for (int t = 0; t < bb; ++t) {
        if (tid < 3) Y[3 * (b0 + t) + tid] *= inv[b0 + t];
        __syncwarp();
        int i = tid / 3, c = tid % 3;      // lanes 0..29 cover rows t+1.. in groups of 10
        for (int ii = t + 1 + i; ii < bb && tid < 30; ii += 10)
          Y[3 * (b0 + ii) + c] -= L[(long long)(b0 + ii) * n + b0 + t] * Y[3 * (b0 + t) + c];
        __syncwarp();
      }
    }
    __syncthreads();
  }
  // backward: L^T X = Z
  const int nblk = (n + 15) / 16;
  for (int blk = nblk - 1; blk >= 0; --blk) {
    const int b0 = blk * 16;
    const int bb = min(16, n - b0);
    const int b1 = b0 + bb;
    double acc[3] = {0.0, 0.0, 0.0};
    if (r < bb) {
      for (int t = b1 + s; t < n; t += 16) {
        double l = L[(long long)t * n + b0 + r];
        acc[0] += l * Y[3 * t + 0];
        acc[1] += l * Y[3 * t + 1];
        acc[2] += l * Y[3 * t + 2];
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o, 16);
    if (s == 0 && r < bb)
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[3 * (b0 + r) + c] -= acc[c];
    __syncthreads();
    if (tid < 32) {
      for (int t = bb - 1; t >= 0; --t) {
        if (tid < 3) Y[3 * (b0 + t) + tid] *= inv[b0 + t];
        __syncwarp();
        int i = tid / 3, c = tid % 3;
        for (int ii = i; ii < t && tid < 30; ii += 10)
          Y[3 * (b0 + ii) + c] -= L[(long long)(b0 + t) * n + b0 + ii] * Y[3 * (b0 + t) + c];
        __syncwarp();
      }
    }
    __syncthreads();
  }
  (void)red;
}

// ---------------------------------------------------------------------------------------
// shared-memory layout of the per-centre SCS kernels
// ---------------------------------------------------------------------------------------
struct ScsSmem {
  double* x;      // 3 x n12 (site displacements, bohr)
  double* rv;     // n12 (R_vdW)
  double* ab;     // n12 (alpha_bar at the current frequency)
  double* sg;     // n12 (sigma at the current frequency)
  double* y;      // 3 n1 x 3 (right-hand side / solution)
  double* z;      // 3 n1 x 3 (X for the adjoint)
  double* inv;    // 3 n1
  double* panel;  // 3 n1 x PS
  double* dg;     // NB x PS
  double* red;    // 256 x 3
  double* gs;     // n12 x 3 site gradients (adjoint)
};

__host__ __device__ inline size_t scs_smem_bytes(int max_n12, int max_n1, bool adjoint) {
  size_t n3 = 3 * (size_t)max_n1;
  size_t d = 6 * (size_t)max_n12 + 3 * n3 + n3 + n3 * PS + NB * PS + 256 * 3;
  if (adjoint) d += 3 * n3 + 3 * (size_t)max_n12;
  return d * sizeof(double);
}

__device__ inline ScsSmem scs_carve(double* base, int max_n12, int max_n1, bool adjoint) {
  ScsSmem s;
  size_t n3 = 3 * (size_t)max_n1;
  s.x = base;
  s.rv = s.x + 3 * max_n12;
  s.ab = s.rv + max_n12;
  s.sg = s.ab + max_n12;
  s.y = s.sg + max_n12;
  s.inv = s.y + 3 * n3;
  s.panel = s.inv + n3;
  s.dg = s.panel + n3 * PS;
  s.red = s.dg + NB * PS;
  s.z = s.red + 256 * 3;
  s.gs = adjoint ? s.z + 3 * n3 : nullptr;
  return s;
}

// T_SR block prefactors for the pair (i, j): returns false if the pair is beyond r_SCS.
// Block = F (A0 I + B0 r r^T), F = f_inner f_SR (1 - f(r, S_ij)).
__device__ __forceinline__ bool tsr_pair(const DevParams& p, double r, double s_ij, double sig_ij,
                                         bool k2, double& F, double& A0, double& B0) {
  if (r >= p.r_scs) return false;
  double fsr, dfsr, fin = 1.0, dfin = 0.0, f, dfr, dfs;
  cutoff_buf(r, p.r_scs, p.r_buf, fsr, dfsr);
  if (k2) finner(r, p.r_inner, fin, dfin);
  fermi(r, s_ij, p.d, f, dfr, dfs);
  F = fin * fsr * (1.0 - f);
  tsr_value(r, sig_ij, A0, B0);
  return true;
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the SCS forward kernel.
//
// Some callers cannot call cudaMalloc: plug-ins of an MD engine that owns the device
// memory pool, and embedded runtimes that forbid allocation after start-up.  For them,
// lmbd_central_polarizabilities_noalloc (lmbd.h) computes the central polarisabilities
// with every scratch buffer carved from the fixed array below.  This array is part of the
// library image: every GPU that loads the library holds these bytes until the process
// exits.  All calls share it and it keeps the contents of the last call; calls whose
// work overlaps on the GPU (two streams, two threads) race on it and must be serialised
// by the caller.
// ---------------------------------------------------------------------------------------
#include <mutex>

#include "../../include/lmbd.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[LMBD_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array for the current device.  The first call on a
// device looks the address up with cudaGetSymbolAddress (host code cannot use the
// symbol itself: in host code it names a host-side stand-in, not device memory).
// Returns 0 on success.
int noalloc_scratch(void** ptr, size_t* bytes) {
  static void* addr[64] = {};
  static std::mutex mtx;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return -1;
  }
  std::lock_guard<std::mutex> lock(mtx);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return -1;
    }
    addr[dev] = p;
  }
  *ptr = addr[dev];
  *bytes = sizeof(g_noalloc_scratch);
  return 0;
}

// Same arithmetic as k_scs_forward (assembly, Cholesky, solves), but persistent over
// central atoms with the matrix of the current (atom, frequency) in this block's slot of
// the scratch array, and only alpha_I written out.
__global__ void __launch_bounds__(256) k_scs_central_noalloc(Work w, DevParams p, double* bslots,
                                                           long long slot_doubles, int max_n12, int max_n1) {
  extern __shared__ double smem_d[];
  ScsSmem sm = scs_carve(smem_d, max_n12, max_n1, false);
  const int tid = threadIdx.x;
  double* B = bslots + (long long)blockIdx.x * slot_doubles;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int c = blockIdx.x; c < w.n_atoms; c += gridDim.x) {
    __syncthreads();
    const Counts cn = w.counts[c];
    const int n1 = cn.n1, n12 = cn.n12, N1 = 3 * n1;
    const long long sbase = (long long)c * w.site_cap;
    for (int s = tid; s < n12; s += blockDim.x) {
      int a = w.site_atom[sbase + s];
      sm.x[s] = w.site_x[3 * (sbase + s) + 0];
      sm.x[max_n12 + s] = w.site_x[3 * (sbase + s) + 1];
      sm.x[2 * max_n12 + s] = w.site_x[3 * (sbase + s) + 2];
      sm.rv[s] = w.rvdw[a];
    }
    const int npair = n1 * (n1 - 1) / 2;
    for (int q = 0; q < p.nq; ++q) {
      __syncthreads();
      for (int s = tid; s < n12; s += blockDim.x) {
        int a = w.site_atom[sbase + s];
        sm.ab[s] = w.abar[a * p.nq + q];
        sm.sg[s] = w.sig[a * p.nq + q];
      }
      __syncthreads();
      for (int e = tid; e < n1 * 6; e += blockDim.x) {
        int i = e / 6, t = e % 6;
        int al = t < 3 ? t : (t == 3 ? 1 : 2), be = t < 3 ? t : (t == 3 ? 0 : (t == 4 ? 0 : 1));
        B[(long long)(3 * i + al) * N1 + 3 * i + be] = (al == be) ? 1.0 / sm.ab[i] : 0.0;
      }
      for (int e = tid; e < npair; e += blockDim.x) {
        int i = (int)((sqrtf(8.0f * e + 1.0f) + 1.0f) * 0.5f);
        while (i * (i - 1) / 2 > e) --i;
        while ((i + 1) * i / 2 <= e) ++i;
        int j = e - i * (i - 1) / 2;
        double rx = sm.x[j] - sm.x[i];
        double ry = sm.x[max_n12 + j] - sm.x[max_n12 + i];
        double rz = sm.x[2 * max_n12 + j] - sm.x[2 * max_n12 + i];
        double r = sqrt(rx * rx + ry * ry + rz * rz);
        double F = 0.0, A0 = 0.0, B0 = 0.0;
        double sig = sqrt(sm.sg[i] * sm.sg[i] + sm.sg[j] * sm.sg[j]);
        if (!tsr_pair(p, r, p.beta * (sm.rv[i] + sm.rv[j]), sig, false, F, A0, B0)) F = 0.0;
        double a = F * A0, b = F * B0;
        double rr[3] = {rx, ry, rz};
        double* blk = B + (long long)(3 * i) * N1 + 3 * j;
#pragma unroll
        for (int al = 0; al < 3; ++al)
#pragma unroll
          for (int be = 0; be < 3; ++be)
            blk[(long long)al * N1 + be] = b * rr[al] * rr[be] + (al == be ? a : 0.0);
      }
      const int warp = tid / 32, lane = tid % 32;
      for (int i = warp; i < n1; i += blockDim.x / 32) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        double xi = sm.x[i], yi = sm.x[max_n12 + i], zi = sm.x[2 * max_n12 + i];
        for (int j = n1 + lane; j < n12; j += 32) {
          double rx = sm.x[j] - xi, ry = sm.x[max_n12 + j] - yi, rz = sm.x[2 * max_n12 + j] - zi;
          double r2 = rx * rx + ry * ry + rz * rz;
          if (r2 >= p.r_scs * p.r_scs) continue;
          double r = sqrt(r2);
          double F, A0, B0;
          double sig = sqrt(sm.sg[i] * sm.sg[i] + sm.sg[j] * sm.sg[j]);
          if (!tsr_pair(p, r, p.beta * (sm.rv[i] + sm.rv[j]), sig, true, F, A0, B0)) continue;
          double a = F * A0 * sm.ab[j], b = F * B0 * sm.ab[j];
          acc[0] += a + b * rx * rx;
          acc[1] += a + b * ry * ry;
          acc[2] += a + b * rz * rz;
          acc[3] += b * rx * ry;
          acc[4] += b * rx * rz;
          acc[5] += b * ry * rz;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int t = 0; t < 6; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
        if (lane == 0) {
          double* y = sm.y + 9 * i;
          y[0] = 1.0 - acc[0]; y[1] = -acc[3];      y[2] = -acc[4];
          y[3] = -acc[3];      y[4] = 1.0 - acc[1]; y[5] = -acc[5];
          y[6] = -acc[4];      y[7] = -acc[5];      y[8] = 1.0 - acc[2];
        }
      }
      __threadfence_block();
      __syncthreads();
      block_cholesky(B, N1, sm.panel, sm.dg, sm.inv, &bad);
      block_solve3(B, N1, sm.inv, sm.y, sm.red);
      if (tid == 0) w.alphaI[(long long)c * p.nq + q] = (sm.y[0] + sm.y[4] + sm.y[8]) / 3.0;
    }
  }
  __syncthreads();
  if (tid == 0 && bad) atomicOr(w.status, LMBD_FLAG_NOT_SPD);
}

void launch_scs_central_noalloc(const Work& w, const DevParams& p, double* bslots, long long slot_doubles,
                                int nslots, int max_n12, int max_n1, cudaStream_t s) {
  size_t sm = scs_smem_bytes(max_n12, max_n1, false);
  raise_smem_limit((const void*)k_scs_central_noalloc, sm);
  k_scs_central_noalloc<<<nslots, 256, sm, s>>>(w, p, bslots, slot_doubles, max_n12, max_n1);
}
