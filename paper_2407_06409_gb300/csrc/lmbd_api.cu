// Host engine and C ABI of the lMBD library (declared in include/lmbd.h).
//
// One call of lmbd_energy_forces runs, on one stream:
//   free-atom quantities -> cell list and site lists -> per-centre offsets
//   -> (one small device-to-host read of the sizes to size the workspaces)
//   -> SCS solves for all centres and frequencies (stage 1)
//   -> blend / T_LR / Krylov chain / energies (stage 2)
//   -> [forces] series adjoint, pair contractions, blend adjoint, SCS adjoint
// Every arithmetic step runs in the kernels of k_*.cu; the host only validates
// arguments, sizes buffers and orders launches.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/lmbd.h"
#include "lmbd_internal.cuh"
#include <nvtx3/nvToolsExt.h>

void raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mtx;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mtx);
  size_t& cur = limit[{dev, func}];
  if (bytes > cur && cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    cur = bytes;
}

namespace {

constexpr int LMBD_ESTALE = -1;   // internal: the kept forward state does not match the inputs

// One NVTX range open at a time (the current phase of a call); closed when the call returns.
struct NvtxPhase {
  bool open = false;
  void enter(const char* name) {
    if (open) nvtxRangePop();
    open = name != nullptr;
    if (open) nvtxRangePushA(name);
  }
  ~NvtxPhase() {
    if (open) nvtxRangePop();
  }
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Ctx {
  lmbd_params prm;
  std::vector<double> table;     // S x 3
  int n_species = 0;
  int n_freq = 0, order = 0;
  std::vector<double> omega, weight;   // quadrature (n_freq)
  int launch_mode = LMBD_LAUNCH_BATCHED;
  int profiling = 0;
  int precision = LMBD_PREC_SLICED;
  int mma_path = LMBD_MMA_TC05;
  long long tc_wait = 0;           // main-loop wait bound of the tcgen05 kernels (0: 2^32 cycles)
  int lorentz = 0;                 // frequency model (lmbd_set_frequency_model)
  double omega_ref = 0.0;
  int fit_nodes = 0;               // integrand model (lmbd_set_integrand_fit): 0 = quadrature
  std::vector<double> fit_omega;   // omega = 0, then the fit nodes
  int lanczos = 0;                 // polynomial-fit coefficients (lmbd_set_series_fit): steps
  int logmode = 0;                 // log mode (lmbd_set_log_mode): Lanczos steps, 0 = series
  int paper_forces = 0;            // force model (lmbd_set_force_model)
  int bucket_width = 6;            // |K1| range of one SCS launch (lmbd_autotune)
  int spectral_fail = 0;           // lmbd_set_spectral_check: return LMBD_CATASTROPHE when flagged
  int sparse = 0;                  // lmbd_set_sparse_tlr: block-sparse T_LR
  // forward state kept for a reverse sweep (lmbd_energy_keep / lmbd_forces_kept)
  int split = 0;
  bool kept_valid = false;
  int kept_n = 0;
  DevBuf kept_pos, kept_spec;
  int theta_sample = -1;           // paper forces with the fitted integrand: the sample of this pass
  // resident site lists (lmbd_set_verlet_skin): candidates within the list radius + skin of the
  // reference frame, refreshed while no atom has moved by half the skin
  double skin = 0.0;
  bool ref_valid = false;
  int ref_n = 0, ref_periodic = 0;
  double ref_cell[9] = {};
  DevBuf ref_pos, ref_spec;
  DevBuf theta_f, theta_out;       // force integrands at the samples (J x N x 3); fitted forces
  int last_nqs = 0;                // columns of the central polarisabilities of the last call
  cudaEvent_t ev[LMBD_NPHASE + 1] = {};
  // around the bucket launches of the SCS factor (pass A) and SCS adjoint (pass C): their own
  // wall time, fork to join, without the pair-list and radial-table kernels of the phase
  cudaEvent_t kev[4] = {};
  // side streams for independent bucket launches (same priority as the caller's stream)
  static constexpr int kSide = 3;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
  int side_prio = 0;
  int site_cap = 0;
  int last_n = 0;
  lmbd_stats stats{};
  size_t mem_budget = 0;          // bytes the context may hold on the device (0 = free memory)
  // device buffers: whole-structure arrays, then one arena for the per-wave workspaces
  DevBuf table_d, pos_d, species_d, nu_d, weights_d, out_e_d, out_f_d;
  DevBuf abar, sig, rvdw, a0, r0, wpos, cell_of, cell_count, cell_start, cell_atoms, grid;
  DevBuf site_atom, site_x, site_img, wrap, counts, offs, totals, status, pcount;
  DevBuf alphaK, alphaI, energies, trbuf, wexp, alphaK_bar, alphaI_bar, gacc, rad_ab, rad_ff;
  DevBuf order1_d, order3_d, fitw, cfit, lam, gl64, fb, fb_flag, lu, sp_cnt, sp_np;
  DevBuf arena;
  std::vector<Counts> counts_h;
  std::vector<long long> offs_h;
  std::vector<int> order1_h, order3_h;
  static constexpr int kMaxWhole = 64;
  DevBuf* whole_bufs[kMaxWhole] = {};
  int n_whole = 0;
  Ctx() {
    DevBuf* l[] = {&table_d, &pos_d, &species_d, &nu_d, &weights_d, &out_e_d, &out_f_d, &abar, &sig, &rvdw,
                   &a0, &r0, &wpos, &cell_of, &cell_count, &cell_start, &cell_atoms, &grid, &site_atom,
                   &site_x, &counts, &offs, &totals, &status, &pcount, &alphaK, &alphaI, &energies, &trbuf,
                   &wexp, &alphaK_bar, &alphaI_bar, &gacc, &order1_d, &order3_d, &rad_ab, &rad_ff, &fitw, &cfit, &lam, &gl64,
                   &fb, &fb_flag, &lu, &theta_f, &theta_out, &site_img, &wrap, &ref_pos, &ref_spec, &kept_pos, &kept_spec,
                   &sp_cnt, &sp_np};
    static_assert(sizeof(l) / sizeof(l[0]) <= kMaxWhole, "whole-structure buffer list exceeds its array");
    for (DevBuf* b : l) whole_bufs[n_whole++] = b;
  }
  size_t whole_bytes() const {
    size_t t = 0;
    for (int i = 0; i < n_whole; ++i) t += whole_bufs[i]->bytes;
    return t;
  }
  long long* totals_h = nullptr;   // pinned
  int* status_h = nullptr;         // pinned
};

int ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return LMBD_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  size_t want = bytes + bytes / 8;     // a little headroom for the next call
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return LMBD_ENOMEM;
    }
    want = bytes;
  }
  b.bytes = want;
  return LMBD_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre_unit(int n, std::vector<double>& x, std::vector<double>& wx) {
  x.assign(n, 0.0);
  wx.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[n - 1 - i] = z;
    wx[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Gauss-Legendre nodes and weights mapped to [0, inf) with omega = L (1 + x) / (1 - x).
void gauss_legendre(int n, double L, std::vector<double>& om, std::vector<double>& w) {
  std::vector<double> x, wx;
  gauss_legendre_unit(n, x, wx);
  om.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    om[i] = L * (1.0 + x[i]) / (1.0 - x[i]);
    w[i] = 2.0 * L * wx[i] / ((1.0 - x[i]) * (1.0 - x[i]));
  }
}

double sphere_radius(const lmbd_params& p) { return p.r_sphere > 0 ? p.r_sphere : p.r_mbd1 + p.r_mbd2; }

int next_pow2(long long v) {
  int p = 1;
  while (p < v && p < (1 << 20)) p <<= 1;
  return p;
}

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) {                   \
      cudaGetLastError();                       \
      return LMBD_ECUDA;                        \
    }                                           \
  } while (0)
#define TRY(x)                    \
  do {                            \
    int _st = (x);                \
    if (_st != LMBD_OK) return _st; \
  } while (0)

int stage_input(DevBuf& buf, const void* src, size_t bytes, cudaStream_t s, const void** out) {
  if (is_device_ptr(src)) {
    *out = src;
    return LMBD_OK;
  }
  TRY(ensure(buf, bytes));
  CK(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s));
  *out = buf.p;
  return LMBD_OK;
}

// ---- per-wave workspaces ------------------------------------------------------------------
// Central atoms are processed in contiguous waves [c0, c1) whose per-centre arrays fit the
// memory budget.  The arrays of a wave live in one arena; every pointer is rebased by the
// wave's first offset, so kernels index them with the whole-structure offsets unchanged.
enum { O_K1, O_S, O_B, O_T, O_P, O_A, O_TQ, O_TR, O_KP, O_SP, O_NP, O_COUNT };

struct Offs {
  const long long* h;
  int N;
  long long at(int k, int i) const { return h[(size_t)k * (N + 1) + i]; }
  long long span(int k, int c0, int c1) const { return at(k, c1) - at(k, c0); }
};

struct Carver {
  char* base;   // NULL: sizing only
  size_t used;
  // n elements of T; the returned pointer is shifted down by `shift` elements
  template <class T>
  T* take(long long n, long long shift) {
    used = (used + 255) & ~(size_t)255;
    T* p = nullptr;
    if (base) p = reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(base + used) - (uintptr_t)shift * sizeof(T));
    used += (size_t)(n > 0 ? n : 1) * sizeof(T);
    return p;
  }
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
  int nq, ncv, nvec, ncol, kp_pair, st, dig_p, site_cap;
  bool forces, sliced_chain, sliced_pair;
  int nqs;   // frequencies of the SCS solves (stage-1 arrays)
  int tk;    // tcgen05 path: row pitch of the T and W digit planes (0: per-centre Kpad)
  bool sparse;   // block-sparse T_LR: coupled pairs and float-float chain/pair operands
  int binv_slot; // floats of the diagonal-block inverses of one SCS system (largest |K1|)

  // stage 1 (SCS): pair lists, FP32 factors and solutions of centres [c0, c1)
  size_t stage1(const Offs& o, int c0, int c1, char* base, Work* w) const {
    Carver cv{base, 0};
    const long long p0 = o.at(O_P, c0), np = o.span(O_P, c0, c1);
    const long long a0 = o.at(O_A, c0), na = o.span(O_A, c0, c1);
    const long long k0 = o.at(O_K1, c0), nk = o.span(O_K1, c0, c1);
    const long long n = c1 - c0;
    float* lfac = cv.take<float>(o.span(O_B, c0, c1), o.at(O_B, c0));
    float* binvg = cv.take<float>((long long)binv_slot * nqs * n, (long long)binv_slot * nqs * c0);
    int* pr_ij = cv.take<int>(2 * (np + 1), 2 * p0);
    double* pr_geo = cv.take<double>(8 * (np + 1), 8 * p0);
    float2* pr_rad_ff = cv.take<float2>(2LL * nqs * (np + 1), 2LL * nqs * p0);
    int* pr_g = cv.take<int>(np + 1, p0);
    float2* pr_gff = cv.take<float2>(6 * (np + 1), 6 * p0);
    int* k2rev = cv.take<int>(np + 1, p0);
    int* prow = cv.take<int>(nk + n, k0 + c0);
    int* prow_k2 = cv.take<int>(nk + n, k0 + c0);
    int* arow = cv.take<int>(nk + n, k0 + c0);
    int* adj = cv.take<int>(2 * (na + 1), 2 * a0);
    int* k2ptr = cv.take<int>(n * site_cap + 1, (long long)c0 * site_cap);
    double* xsol = cv.take<double>(9LL * nqs * nk, 9LL * nqs * k0);
    if (w) {
      w->lfac = lfac;
      w->binvg = binvg;
      w->binv_slot = binv_slot;
      w->pr_ij = pr_ij;
      w->pr_geo = pr_geo;
      w->pr_rad_ff = pr_rad_ff;
      w->pr_g = pr_g;
      w->pr_gff = pr_gff;
      w->k2rev = k2rev;
      w->prow = prow;
      w->prow_k2 = prow_k2;
      w->arow = arow;
      w->adj = adj;
      w->k2ptr = k2ptr;
      w->xsol = xsol;
    }
    return align256(cv.used);
  }

  // scratch of the SCS adjoint: pair and site gradients of centres [c0, c1)
  size_t scs_adjoint(const Offs& o, int c0, int c1, char* base, Work* w) const {
    Carver cv{base, 0};
    const long long p0 = o.at(O_P, c0), np = o.span(O_P, c0, c1);
    double* gstage = cv.take<double>(3LL * nqs * (np + 1), 3LL * nqs * p0);
    double* sgq = cv.take<double>(3LL * nqs * (c1 - c0) * site_cap, 3LL * nqs * c0 * site_cap);
    if (w) {
      w->gstage = gstage;
      w->sgq = sgq;
    }
    return align256(cv.used);
  }

  // stage 2 (MBD): blended polarisabilities, T_LR, Krylov blocks, slices and adjoint arrays
  size_t stage2(const Offs& o, int c0, int c1, char* base, Work* w, unsigned short** wdig_raw) const {
    Carver cv{base, 0};
    const long long s0 = o.at(O_S, c0), ns = o.span(O_S, c0, c1);
    const long long t0 = o.at(O_T, c0), nt = o.span(O_T, c0, c1);
    const long long np0 = o.at(O_NP, c0), npn = o.span(O_NP, c0, c1);
    double* alphaT = cv.take<double>((long long)nq * ns, (long long)nq * s0);
    double* dsq = cv.take<double>((long long)nq * ns, (long long)nq * s0);
    double* tlr = sparse ? nullptr : cv.take<double>(nt, t0);
    double* vkr = cv.take<double>((long long)nvec * ns * 3 * ncv, s0 * 3 * ncv);
    if (w) {
      w->alphaT = alphaT;
      w->dsq = dsq;
      w->tlr = tlr;
      w->vkr = vkr;
      w->vstride = ns * 3 * ncv;
    }
    if (sparse) {
      int4* sp_row = cv.take<int4>(ns, s0);
      int2* sp_ent = cv.take<int2>(2 * npn, 2 * np0);
      int2* sp_pair = cv.take<int2>(npn, np0);
      float4* sp_blk = cv.take<float4>(3 * npn, 3 * np0);
      float2* wff = cv.take<float2>((long long)nvec * ns * 3 * ncv, s0 * 3 * ncv);
      float2* dsq_ff = cv.take<float2>((long long)nq * ns, (long long)nq * s0);
      if (w) {
        w->dsq_ff = dsq_ff;
        w->sp_row = sp_row;
        w->sp_ent = sp_ent;
        w->sp_pair = sp_pair;
        w->sp_blk = sp_blk;
        w->wff = wff;
      }
    }
    if (sliced_chain) {
      // T planes: per centre st planes of Mpad rows, row pitch Kpad (warp-level path) or the
      // common pitch tk (tcgen05 path: one tensor map covers the wave)
      unsigned short* tdig =
          tk > 0 ? cv.take<unsigned short>((long long)st * o.span(O_TR, c0, c1) * tk, (long long)st * o.at(O_TR, c0) * tk)
                 : cv.take<unsigned short>((long long)st * o.span(O_TQ, c0, c1), (long long)st * o.at(O_TQ, c0));
      int* texp = cv.take<int>(o.span(O_TR, c0, c1), o.at(O_TR, c0));
      // W planes: the digit count varies per chain step, so the pointer is rebased per launch
      unsigned short* wdig = tk > 0 ? cv.take<unsigned short>(48LL * st * (c1 - c0) * tk, 0)
                                    : cv.take<unsigned short>(48LL * st * o.span(O_KP, c0, c1), 0);
      if (w) {
        w->tdig = tdig;
        w->texp = texp;
        *wdig_raw = wdig;
        w->tk = tk;
        w->trow0 = (long long)st * o.at(O_TR, c0);
        w->trows = (long long)st * o.span(O_TR, c0, c1);
        w->wc0 = c0;
        w->wcn = c1 - c0;
      }
    }
    if (forces) {
      const long long nc = ncol > 0 ? ncol : 1;
      double* gbar = cv.take<double>((long long)nq * ns, (long long)nq * s0);
      // P and Q: FP64 for the dense products, float-float for the sparse pair products
      double* pmat = sparse ? nullptr : cv.take<double>(3 * ns * nc, 3 * s0 * nc);
      double* qmat = sparse ? nullptr : cv.take<double>(3 * ns * nc, 3 * s0 * nc);
      float2* pff = sparse ? cv.take<float2>(3 * ns * nc, 3 * s0 * nc) : nullptr;
      float2* qff = sparse ? cv.take<float2>(3 * ns * nc, 3 * s0 * nc) : nullptr;
      double* x0buf = cv.take<double>(9 * ns, 9 * s0);
      double* pcoef = sparse ? cv.take<double>(8 * npn, 8 * np0) : cv.take<double>(nt, t0);
      double* rbar = cv.take<double>(ns, s0);
      if (w) {
        w->gbar = gbar;
        w->pmat = pmat;
        w->qmat = qmat;
        w->pff = pff;
        w->qff = qff;
        w->x0buf = x0buf;
        w->pcoef = pcoef;
        w->rbar = rbar;
      }
      if (sliced_pair) {
        const long long sp0 = o.at(O_SP, c0), nsp = o.span(O_SP, c0, c1);
        const long long per = 3LL * kp_pair * dig_p;
        unsigned short* pdig = cv.take<unsigned short>(per * nsp, per * sp0);
        unsigned short* qdig = cv.take<unsigned short>(per * nsp, per * sp0);
        int* pexp = cv.take<int>(3 * nsp, 3 * sp0);
        int* qexp = cv.take<int>(3 * nsp, 3 * sp0);
        if (w) {
          w->pdig = pdig;
          w->qdig = qdig;
          w->pexp = pexp;
          w->qexp = qexp;
          w->prow0 = 3LL * dig_p * sp0;
          w->prows = 3LL * dig_p * nsp;
        }
      }
    }
    return align256(cv.used);
  }
};

// Contiguous waves [cuts[i], cuts[i+1]) with size(c0, c1) <= cap; false when one centre alone
// does not fit.
template <class F>
bool partition(int N, size_t cap, F size, std::vector<int>& cuts) {
  cuts.assign(1, 0);
  int c0 = 0;
  while (c0 < N) {
    if (size(c0, c0 + 1) > cap) return false;
    int c1 = c0 + 1;
    while (c1 < N && size(c0, c1 + 1) <= cap) ++c1;
    cuts.push_back(c1);
    c0 = c1;
  }
  return true;
}

// Size buckets for the SCS kernels: within each wave, centres sorted by |K1|, one launch per
// bucket of width 6 in |K1| with shared memory sized to the bucket.
struct Bucket {
  int b0, b1, n1, n12;
};
void make_buckets(const std::vector<Counts>& cnt, const std::vector<int>& cuts, std::vector<int>& order,
                  std::vector<std::vector<Bucket>>& buckets, int width) {
  const int N = (int)cnt.size();
  order.resize(N);
  for (int i = 0; i < N; ++i) order[i] = i;
  buckets.assign(cuts.size() - 1, {});
  for (size_t wv = 0; wv + 1 < cuts.size(); ++wv) {
    const int c0 = cuts[wv], c1 = cuts[wv + 1];
    std::stable_sort(order.begin() + c0, order.begin() + c1, [&](int x, int y) { return cnt[x].n1 < cnt[y].n1; });
    int b0 = c0;
    while (b0 < c1) {
      const int lo = cnt[order[b0]].n1;
      int b1 = b0, n1m = 0, n12m = 0;
      while (b1 < c1 && cnt[order[b1]].n1 < lo + width) {
        n1m = std::max(n1m, cnt[order[b1]].n1);
        n12m = std::max(n12m, cnt[order[b1]].n12);
        ++b1;
      }
      buckets[wv].push_back({b0, b1, n1m, n12m});
      b0 = b1;
    }
  }
}

// Side streams with the priority of s, created on first use (or again when the priority changes).
int side_streams(Ctx* c, cudaStream_t s) {
  int prio = 0;
  if (cudaStreamGetPriority(s, &prio) != cudaSuccess) prio = 0;
  if (c->side[0] && prio == c->side_prio) return LMBD_OK;
  for (int i = 0; i < Ctx::kSide; ++i) {
    if (c->side[i]) cudaStreamDestroy(c->side[i]);
    c->side[i] = nullptr;
    if (cudaStreamCreateWithPriority(&c->side[i], cudaStreamNonBlocking, prio) != cudaSuccess) return LMBD_ECUDA;
    if (!c->join_ev[i] && cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming) != cudaSuccess)
      return LMBD_ECUDA;
  }
  if (!c->fork_ev && cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess) return LMBD_ECUDA;
  c->side_prio = prio;
  return LMBD_OK;
}

// Launches of independent buckets spread over s and the side streams: fork after the work
// already queued on s, join back into s at the end.
struct Fork {
  Ctx* c;
  cudaStream_t s;
  int n;
  Fork(Ctx* c_, cudaStream_t s_, int buckets) : c(c_), s(s_), n(std::min(buckets, Ctx::kSide + 1)) {
    cudaEventRecord(c->fork_ev, s);
    for (int i = 0; i + 1 < n; ++i) cudaStreamWaitEvent(c->side[i], c->fork_ev, 0);
  }
  cudaStream_t stream(int b) const { return b % n == 0 ? s : c->side[b % n - 1]; }
  void join() {
    for (int i = 0; i + 1 < n; ++i) {
      cudaEventRecord(c->join_ev[i], c->side[i]);
      cudaStreamWaitEvent(s, c->join_ev[i], 0);
    }
  }
};

int run(Ctx* c, int N, const double* pos_in, const double* cell, const int* spec_in, const double* nu_in,
        const double* w_in, double* e_out, double* f_out, cudaStream_t s) {
  lmbd_stats st{};
  c->stats = st;
  c->last_n = N;
  if (N == 0) return LMBD_OK;
  TRY(side_streams(c, s));
  const lmbd_params& P = c->prm;
  // frequencies at which the integrand is evaluated: the quadrature nodes, or omega = 0 and
  // the fit nodes of the fitted integrand
  const int nf = c->fit_nodes ? c->fit_nodes + 1 : c->n_freq;
  const int nq = nf + 1;
  // split: 0 a whole call; 1 (lmbd_energy_keep) the forward passes with the layout of a forces
  // call, the state kept for a later reverse sweep; 2 (lmbd_forces_kept) the reverse sweep alone
  // on that state, for the same inputs
  const int split = c->split;
  const bool reverse_only = split == 2;
  const bool forces = f_out != nullptr || split == 1;
  if (!reverse_only) c->kept_valid = false;   // the forward state is about to be overwritten
  int launches = 0;

  // ---- inputs ---------------------------------------------------------------------------
  const void *pos, *spec, *nu, *wts = nullptr;
  TRY(stage_input(c->pos_d, pos_in, sizeof(double) * 3 * N, s, &pos));
  TRY(stage_input(c->species_d, spec_in, sizeof(int) * N, s, &spec));
  TRY(stage_input(c->nu_d, nu_in, sizeof(double) * N, s, &nu));
  if (w_in) TRY(stage_input(c->weights_d, w_in, sizeof(double) * N, s, &wts));

  // ---- parameters -------------------------------------------------------------------------
  DevParams dp{};
  const double ib = 1.0 / LMBD_BOHR;
  const double rsph = sphere_radius(P);
  // with resident site lists the lists hold every site within the list radius + skin
  const double rlist = fmax(2.0 * P.r_scs, rsph) + c->skin;
  dp.r_scs = P.r_scs * ib;
  dp.r_mbd1 = P.r_mbd1 * ib;
  dp.r_mbd2 = P.r_mbd2 * ib;
  dp.r_buf = P.r_buf * ib;
  dp.r_inner = P.r_inner * ib;
  dp.beta = P.beta;
  dp.d = P.d;
  dp.r2_scs_ang = P.r_scs * P.r_scs;
  dp.r2_sphere_ang = rsph * rsph;
  dp.r2_scs2_ang = 4.0 * P.r_scs * P.r_scs;
  dp.r2_list_ang = rlist * rlist;
  dp.n_freq = nf;
  dp.nq = nq;
  dp.order = c->order;
  dp.n_species = c->n_species;
  dp.omega[0] = 0.0;
  dp.cweight[0] = 0.0;
  const double pi = 3.14159265358979323846;
  if (c->fit_nodes) {
    dp.fit = 1;
    for (int q = 0; q < nf; ++q) {
      dp.omega[q + 1] = c->fit_omega[q];
      dp.cweight[q + 1] = 0.0;
    }
    dp.n_phi = c->n_freq;
    for (int i = 0; i < c->n_freq; ++i) {
      dp.phi_omega[i] = c->omega[i];
      dp.phi_wt[i] = c->weight[i] / (2.0 * pi);
    }
  } else {
    for (int q = 0; q < c->n_freq; ++q) {
      dp.omega[q + 1] = c->omega[q];
      dp.cweight[q + 1] = LMBD_HARTREE * c->weight[q] / (2.0 * pi);
    }
  }
  dp.lorentz = c->lorentz;
  dp.lanczos = c->lanczos;
  dp.logmode = c->logmode;
  if (c->logmode && forces) return LMBD_EUNSUPPORTED;   // the log mode gives energies only
  if (c->logmode && c->lanczos) return LMBD_EINVAL;
  for (int n = 1; n < LMBD_MAX_ORDER_P1; ++n) dp.cn[n] = -1.0 / n;
  dp.paper = c->paper_forces && forces;
  // the block-sparse T_LR serves the series energy and its exact adjoint; the Lanczos-based
  // modes and the paper's forces read the dense matrix
  if (c->sparse && (c->logmode || c->lanczos || dp.paper)) return LMBD_EUNSUPPORTED;
  dp.tc_wait = c->tc_wait > 0 ? c->tc_wait : (1LL << 32);
  // the paper's forces with the fitted integrand run once per sample frequency (run_theta): the
  // frequency weights of that pass select the bare integrand at that sample
  if (dp.paper && c->fit_nodes && c->theta_sample < 0) return LMBD_EINVAL;
  if (dp.paper && c->fit_nodes)
    for (int q = 0; q < nf; ++q) dp.cweight[q + 1] = q == c->theta_sample ? LMBD_HARTREE : 0.0;
  dp.omega_ref = c->omega_ref;
  dp.nqs = c->lorentz ? 2 : nq;
  for (int q = 0; q < dp.nqs; ++q) dp.omega_s[q] = c->lorentz ? (q == 0 ? 0.0 : c->omega_ref) : dp.omega[q];
  c->last_nqs = dp.nqs;

  // ---- search grid ------------------------------------------------------------------------
  Grid g{};
  double vol_est = 0.0;
  if (cell) {
    double hc[9];
    if (is_device_ptr(cell)) {
      CK(cudaMemcpyAsync(hc, cell, sizeof(hc), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    } else {
      memcpy(hc, cell, sizeof(hc));
    }
    for (int i = 0; i < 9; ++i)
      if (!std::isfinite(hc[i])) return LMBD_EINVAL;
    double det = hc[0] * (hc[4] * hc[8] - hc[5] * hc[7]) - hc[1] * (hc[3] * hc[8] - hc[5] * hc[6]) +
                 hc[2] * (hc[3] * hc[7] - hc[4] * hc[6]);
    if (!(fabs(det) > 1e-9)) return LMBD_EINVAL;
    g.periodic = 1;
    memcpy(g.cell, hc, sizeof(hc));
    // inverse (cofactor / det), frac = pos * inv
    double inv[9] = {(hc[4] * hc[8] - hc[5] * hc[7]) / det, -(hc[1] * hc[8] - hc[2] * hc[7]) / det,
                     (hc[1] * hc[5] - hc[2] * hc[4]) / det, -(hc[3] * hc[8] - hc[5] * hc[6]) / det,
                     (hc[0] * hc[8] - hc[2] * hc[6]) / det, -(hc[0] * hc[5] - hc[2] * hc[3]) / det,
                     (hc[3] * hc[7] - hc[4] * hc[6]) / det, -(hc[0] * hc[7] - hc[1] * hc[6]) / det,
                     (hc[0] * hc[4] - hc[1] * hc[3]) / det};
    memcpy(g.inv, inv, sizeof(inv));
    vol_est = fabs(det);
    for (int d = 0; d < 3; ++d) {
      const double* a = hc + 3 * ((d + 1) % 3);
      const double* b = hc + 3 * ((d + 2) % 3);
      double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
      double width = fabs(det) / sqrt(cx * cx + cy * cy + cz * cz);
      int nc = (int)(width / rlist);
      if (nc < 1) nc = 1;
      if (nc > 64) nc = 64;
      g.nc[d] = nc;
      g.reach[d] = (int)ceil(rlist / (width / nc) - 1e-12);
      if (g.reach[d] < 1) g.reach[d] = 1;
    }
  }
  const int ncells = cell ? g.nc[0] * g.nc[1] * g.nc[2] : 64 * 64 * 64;

  // ---- per-atom buffers ----------------------------------------------------------------------
  TRY(ensure(c->abar, sizeof(double) * N * nq));
  TRY(ensure(c->sig, sizeof(double) * N * nq));
  TRY(ensure(c->rvdw, sizeof(double) * N));
  TRY(ensure(c->a0, sizeof(double) * N));
  TRY(ensure(c->r0, sizeof(double) * N));
  TRY(ensure(c->wpos, sizeof(double) * 3 * N));
  TRY(ensure(c->cell_of, sizeof(int) * N));
  TRY(ensure(c->cell_count, sizeof(int) * ncells));
  TRY(ensure(c->cell_start, sizeof(int) * (ncells + 1)));
  TRY(ensure(c->cell_atoms, sizeof(int) * N));
  TRY(ensure(c->wrap, sizeof(int) * 3 * (size_t)N));
  TRY(ensure(c->grid, sizeof(Grid)));
  TRY(ensure(c->counts, sizeof(Counts) * N));
  TRY(ensure(c->offs, sizeof(long long) * O_COUNT * (size_t)(N + 1)));
  TRY(ensure(c->totals, sizeof(long long) * 16));
  TRY(ensure(c->pcount, sizeof(int) * 2 * N));
  TRY(ensure(c->status, sizeof(int) * 4));
  TRY(ensure(c->alphaI, sizeof(double) * N * nq));
  TRY(ensure(c->energies, sizeof(double) * N));
  TRY(ensure(c->trbuf, sizeof(double) * (size_t)N * LMBD_MAX_ORDER_P1 * 64));
  TRY(ensure(c->fb, sizeof(int) * (1 + (size_t)N * nq)));
  TRY(ensure(c->fb_flag, sizeof(int) * (size_t)N * nq));

  // site capacity from the density (sites within r_list), grown on overflow
  {
    const double four_pi_3 = 4.18879020478639098;
    double dens = cell ? N / vol_est : 0.1;
    long long expect = (long long)(dens * four_pi_3 * rlist * rlist * rlist) + 1;
    if (!cell && expect > N) expect = N;
    int cap = next_pow2((long long)(1.5 * expect) + 64);
    if (cap < 64) cap = 64;
    if (cap > 4096) cap = 4096;
    if (cap < c->site_cap) cap = c->site_cap;
    c->site_cap = cap;
  }

  Work w{};
  w.n_atoms = N;
  w.pos = (const double*)pos;
  w.species = (const int*)spec;
  w.nu = (const double*)nu;
  w.table = (const double*)c->table_d.p;
  w.weights = (const double*)wts;
  w.abar = (double*)c->abar.p;
  w.sig = (double*)c->sig.p;
  w.rvdw = (double*)c->rvdw.p;
  w.a0 = (double*)c->a0.p;
  w.r0 = (double*)c->r0.p;
  w.wpos = (double*)c->wpos.p;
  w.cell_of = (int*)c->cell_of.p;
  w.cell_count = (int*)c->cell_count.p;
  w.cell_start = (int*)c->cell_start.p;
  w.cell_atoms = (int*)c->cell_atoms.p;
  w.wrap = (int*)c->wrap.p;
  w.ncells = ncells;
  w.grid = (Grid*)c->grid.p;
  w.counts = (Counts*)c->counts.p;
  long long* const ob = (long long*)c->offs.p;
  w.off_k1 = ob + (size_t)O_K1 * (N + 1);
  w.off_s = ob + (size_t)O_S * (N + 1);
  w.off_b = ob + (size_t)O_B * (N + 1);
  w.off_t = ob + (size_t)O_T * (N + 1);
  w.off_p = ob + (size_t)O_P * (N + 1);
  w.off_a = ob + (size_t)O_A * (N + 1);
  w.off_tq = ob + (size_t)O_TQ * (N + 1);
  w.off_tr = ob + (size_t)O_TR * (N + 1);
  w.off_kp = ob + (size_t)O_KP * (N + 1);
  w.off_sp = ob + (size_t)O_SP * (N + 1);
  w.off_np = ob + (size_t)O_NP * (N + 1);
  w.totals = (long long*)c->totals.p;
  w.status = (int*)c->status.p;
  w.pcount = (int*)c->pcount.p;
  w.alphaI = (double*)c->alphaI.p;
  w.energies = (double*)c->energies.p;
  w.trbuf = (double*)c->trbuf.p;
  w.fb = (int*)c->fb.p;
  w.fb_flag = (int*)c->fb_flag.p;

  // species indices must be in range and inputs finite: checked here when the caller passed
  // host arrays, and by the free-atom kernel for device arrays (LMBD_FLAG_BAD_INPUT).
  if (!is_device_ptr(spec_in))
    for (int i = 0; i < N; ++i)
      if (spec_in[i] < 0 || spec_in[i] >= c->n_species) return LMBD_EINVAL;
  if (!is_device_ptr(nu_in))
    for (int i = 0; i < N; ++i)
      if (!(nu_in[i] > 0.0) || !std::isfinite(nu_in[i])) return LMBD_EINVAL;
  if (!is_device_ptr(pos_in))
    for (int i = 0; i < 3 * N; ++i)
      if (!std::isfinite(pos_in[i])) return LMBD_EINVAL;

  const bool prof_req = c->profiling && c->launch_mode == LMBD_LAUNCH_BATCHED;
  bool prof = prof_req;   // per-phase events only when every stage runs as one wave
  int phase_launch[LMBD_NPHASE] = {};
  bool marked[LMBD_NPHASE + 1] = {};
  // phase boundaries: CUDA events when profiling, and an NVTX range per phase (host-side
  // annotations that a profiler attaches to the launches; nearly free without one)
  static const char* const kPhaseName[LMBD_NPHASE] = {"lmbd neighbours", "lmbd SCS", "lmbd prepare",
                                                      "lmbd chain", "lmbd energy", "lmbd adjoint series",
                                                      "lmbd adjoint pair", "lmbd adjoint blend",
                                                      "lmbd SCS adjoint", "lmbd output"};
  NvtxPhase nvtx;
  auto mark = [&](int ph) {
    nvtx.enter(ph < LMBD_NPHASE ? kPhaseName[ph] : nullptr);
    if (prof) {
      cudaEventRecord(c->ev[ph], s);
      marked[ph] = true;
    }
  };
  mark(LMBD_PHASE_NEIGHBORS);
  if (reverse_only) {   // the kept forward state must belong to these positions and species
    w.site_cap = c->site_cap;
    w.site_atom = (int*)c->site_atom.p;
    w.site_x = (double*)c->site_x.p;
    w.site_img = (int*)c->site_img.p;
    CK(cudaMemsetAsync(w.status, 0, sizeof(int) * 4, s));
    launch_skin_check(w, (const double*)c->kept_pos.p, (const int*)c->kept_spec.p, 1e-300, w.status + 3, s);
    CK(cudaMemcpyAsync(c->status_h, w.status + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*c->status_h != 0) return LMBD_ESTALE;
  }
  // resident site lists: a frame of the same structure (atom count, cell, species) whose atoms
  // all moved by less than half the skin since the lists were built refreshes them in place
  bool refresh = false;
  if (!reverse_only && c->skin > 0.0 && c->ref_valid && c->ref_n == N && c->ref_periodic == (cell ? 1 : 0) &&
      (!cell || memcmp(c->ref_cell, g.cell, sizeof(c->ref_cell)) == 0) && c->site_atom.p) {
    w.site_cap = c->site_cap;
    CK(cudaMemsetAsync(w.status, 0, sizeof(int) * 4, s));
    launch_skin_check(w, (const double*)c->ref_pos.p, (const int*)c->ref_spec.p, 0.25 * c->skin * c->skin,
                      w.status + 3, s);
    CK(cudaMemcpyAsync(c->status_h, w.status + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    refresh = *c->status_h == 0;
    ++launches;
  }
  if (!refresh && !reverse_only) c->ref_valid = false;   // rebuilt below; valid again on success
  for (int attempt = 0; attempt < 4 && !reverse_only; ++attempt) {
    TRY(ensure(c->site_atom, sizeof(int) * (size_t)N * c->site_cap));
    TRY(ensure(c->site_x, sizeof(double) * 3 * (size_t)N * c->site_cap));
    TRY(ensure(c->site_img, sizeof(int) * 3 * (size_t)N * c->site_cap));
    w.site_cap = c->site_cap;
    w.site_atom = (int*)c->site_atom.p;
    w.site_x = (double*)c->site_x.p;
    w.site_img = (int*)c->site_img.p;
    CK(cudaMemsetAsync(w.status, 0, sizeof(int) * 4, s));
    if (attempt == 0) {   // after the status reset: it validates device-resident inputs
      launch_free_atom(w, dp, s);
      ++launches;
    }
    if (refresh)
      launch_sites_refresh(w, dp, g, s, &launches);
    else
      launch_neighbors(w, dp, g, s, &launches);
    if (c->sparse) {   // coupled T_LR partners of every site: the offsets size the pair arrays
      TRY(ensure(c->sp_cnt, sizeof(int2) * (size_t)N * c->site_cap));
      TRY(ensure(c->sp_np, sizeof(int) * (size_t)N));
      w.sp_cnt = (int2*)c->sp_cnt.p;
      w.sp_np = (int*)c->sp_np.p;
      launch_sp_count(w, dp, s);
      ++launches;
    }
    launch_scs_count(w, dp, w.site_cap, s);
    launch_offsets(w, dp, s);
    launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->totals_h, w.totals, sizeof(long long) * 16, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->status_h, w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*c->status_h & LMBD_FLAG_BAD_INPUT) return LMBD_EINVAL;
    if (!(*c->status_h & LMBD_FLAG_CAPACITY)) {
      if (*c->status_h & LMBD_FLAG_COINCIDENT) return LMBD_EINVAL;
      break;
    }
    refresh = false;   // a grown capacity needs a full build
    if (c->site_cap >= 4096 || attempt == 3) return LMBD_ECAPACITY;
    c->site_cap *= 2;
  }
  phase_launch[LMBD_PHASE_NEIGHBORS] = launches;
  c->stats.sites_refreshed = refresh ? 1 : 0;
  if (c->skin > 0.0 && !refresh && !reverse_only) {   // the lists were built for this frame: it is the reference
    TRY(ensure(c->ref_pos, sizeof(double) * 3 * (size_t)N));
    TRY(ensure(c->ref_spec, sizeof(int) * (size_t)N));
    CK(cudaMemcpyAsync(c->ref_pos.p, w.pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->ref_spec.p, w.species, sizeof(int) * N, cudaMemcpyDeviceToDevice, s));
    c->ref_valid = true;
    c->ref_n = N;
    c->ref_periodic = cell ? 1 : 0;
    memcpy(c->ref_cell, g.cell, sizeof(c->ref_cell));
  }
  const long long sum_n1 = c->totals_h[0];
  const int max_n1 = (int)c->totals_h[4], max_ns = (int)c->totals_h[5], max_n12 = (int)c->totals_h[6];
  // kernel shared-memory capacities (per-centre systems live in shared memory)
  // (the block-sparse T_LR path keeps no dense 3 ns x 3 ns matrix: spheres up to the site capacity)
  if (max_n1 > 96 || max_ns > (c->sparse ? 4096 : 1024) || max_n12 > 4096) return LMBD_ECAPACITY;
  const int max_pairs = (int)c->totals_h[11];
  if (scs2_adjoint_smem(max_n1, max_n12) > 227 * 1024) return LMBD_ECAPACITY;
  // dense FP64 slots of the LU fallback, one per persistent block
  const int lu_blocks = 32;
  w.lu_slot = 9LL * max_n1 * max_n1;
  TRY(ensure(c->lu, sizeof(double) * (size_t)lu_blocks * (size_t)w.lu_slot));
  w.lu = (double*)c->lu.p;
  if (!reverse_only) {   // the reverse sweep reuses the host copies of the kept forward call
    c->counts_h.resize(N);
    c->offs_h.resize((size_t)O_COUNT * (N + 1));
    CK(cudaMemcpyAsync(c->counts_h.data(), w.counts, sizeof(Counts) * N, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->offs_h.data(), ob, sizeof(long long) * O_COUNT * (N + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  const Offs o{c->offs_h.data(), N};

  // ---- whole-structure arrays -------------------------------------------------------------
  const int ncv = 3 * nf;
  const int nvec = forces ? (c->order - 1) : (c->order + 1) / 2;
  const int ncol = 3 * nf * (c->order - 2);
  // sliced tensor-core products: digits per product (see ozaki.cuh and the design notes)
  const bool sliced = c->precision == LMBD_PREC_SLICED;
  const bool sparse = c->sparse != 0;
  const bool sliced_chain = sliced && ncv <= 48 && !c->logmode && !sparse;
  const bool sliced_pair = sliced && ncol > 0 && !sparse;
  const bool tc05 = c->mma_path == LMBD_MMA_TC05;
  const int ST = 6, DIG_E = 6, DIG_A = 5, DIG_P = 5;
  TRY(ensure(c->alphaK, sizeof(double) * (size_t)sum_n1 * nq));
  TRY(ensure(c->rad_ab, sizeof(double) * 2 * (size_t)sum_n1 * nq));
  TRY(ensure(c->rad_ff, sizeof(float2) * 4 * (size_t)sum_n1 * nq));
  w.alphaK = (double*)c->alphaK.p;
  w.rad_ab = (double*)c->rad_ab.p;
  w.rad_ff = (float2*)c->rad_ff.p;
  w.nvec = nvec;
  w.ncol = ncol;
  if (sliced_chain) {
    TRY(ensure(c->wexp, sizeof(int) * (size_t)48 * N));
    w.wexp = (int*)c->wexp.p;
  }
  if (forces) {
    TRY(ensure(c->alphaK_bar, sizeof(double) * (size_t)sum_n1 * nq));
    TRY(ensure(c->alphaI_bar, sizeof(double) * (size_t)N * nq));
    TRY(ensure(c->gacc, sizeof(double) * 3 * (size_t)N));
    w.alphaK_bar = (double*)c->alphaK_bar.p;
    w.alphaI_bar = (double*)c->alphaI_bar.p;
    w.gacc = (double*)c->gacc.p;
    if (!is_device_ptr(f_out)) TRY(ensure(c->out_f_d, sizeof(double) * 3 * N));
  }
  TRY(ensure(c->order1_d, sizeof(int) * N));
  TRY(ensure(c->order3_d, sizeof(int) * N));
  if (c->fit_nodes) {
    TRY(ensure(c->fitw, sizeof(double) * LMBD_FITW * (size_t)N));
    w.fitw = (double*)c->fitw.p;
  }
  if (c->lanczos) {
    TRY(ensure(c->cfit, sizeof(double) * LMBD_MAX_ORDER_P1 * (size_t)nf * N));
    TRY(ensure(c->lam, sizeof(double) * 2 * (size_t)nf * N));
    TRY(ensure(c->gl64, sizeof(double) * 128));
    static double gl_h[128];
    static std::once_flag gl_once;
    std::call_once(gl_once, [] {
      std::vector<double> x, wx;
      gauss_legendre_unit(64, x, wx);
      for (int i = 0; i < 64; ++i) {
        gl_h[i] = x[i];
        gl_h[64 + i] = wx[i];
      }
    });
    CK(cudaMemcpyAsync(c->gl64.p, gl_h, sizeof(gl_h), cudaMemcpyHostToDevice, s));
    w.cfit = (double*)c->cfit.p;
    w.lam = (double*)c->lam.p;
    w.gl64 = (const double*)c->gl64.p;
  }

  // ---- waves under the memory budget --------------------------------------------------------
  const Layout L{nq, ncv, nvec, ncol, (ncol + 15) / 16 * 16, ST, DIG_P, c->site_cap, forces, sliced_chain,
                 sliced_pair, dp.nqs, tc05 ? (3 * max_ns + 15) / 16 * 16 : 0, sparse,
                 (3 * max_n1 + 15) / 16 * 136};
  auto s1 = [&](int a, int b) { return L.stage1(o, a, b, nullptr, nullptr); };
  auto s1x = [&](int a, int b) { return forces ? L.scs_adjoint(o, a, b, nullptr, nullptr) : (size_t)0; };
  auto s2 = [&](int a, int b) { return L.stage2(o, a, b, nullptr, nullptr, nullptr); };
  auto s1_and_x = [&](int a, int b) { return s1(a, b) + s1x(a, b); };
  size_t avail;
  {
    const size_t whole = c->whole_bytes();
    if (c->mem_budget) {
      avail = c->mem_budget > whole ? c->mem_budget - whole : 0;
    } else {
      size_t fr = 0, tot = 0;
      CK(cudaMemGetInfo(&fr, &tot));
      const size_t reserve = (size_t)1 << 30;
      avail = fr + c->arena.bytes;
      avail = avail > reserve ? avail - reserve : 0;
    }
  }
  // cutA: waves of the forward SCS; cutC: waves of the SCS adjoint; cut2: waves of stage 2.
  // persist: the stage-1 arrays of all centres stay resident from the forward SCS to its
  // adjoint; otherwise stage 1 of each adjoint wave is computed again before its adjoint.
  std::vector<int> cutA, cutC, cut2;
  bool persist = true;
  size_t R1 = 0, arena_need = 0;
  {
    const size_t S1all = s1(0, N), S2all = s2(0, N), X1all = s1x(0, N);
    auto maxw = [](const std::vector<int>& cuts, auto f) {
      size_t m = 0;
      for (size_t i = 0; i + 1 < cuts.size(); ++i) m = std::max(m, (size_t)f(cuts[i], cuts[i + 1]));
      return m;
    };
    if (reverse_only) {   // the kept forward call ran as one wave with resident stage-1 arrays
      cutA = cutC = cut2 = {0, N};
      R1 = S1all;
      arena_need = 0;
    } else if (S1all + std::max(S2all, X1all) <= avail) {
      cutA = cutC = cut2 = {0, N};
      R1 = S1all;
      arena_need = S1all + std::max(S2all, X1all);
    } else if (!forces) {
      persist = false;
      if (!partition(N, avail, s1, cutA) || !partition(N, avail, s2, cut2)) return LMBD_ENOMEM;
      cutC = cutA;
      arena_need = std::max(maxw(cutA, s1), maxw(cut2, s2));
    } else if (S1all <= avail / 2) {
      cutA = {0, N};
      R1 = S1all;
      if (!partition(N, avail - R1, s2, cut2) || !partition(N, avail - R1, s1x, cutC)) return LMBD_ENOMEM;
      arena_need = R1 + std::max(maxw(cut2, s2), maxw(cutC, s1x));
    } else {
      persist = false;
      if (!partition(N, avail, s1_and_x, cutA) || !partition(N, avail, s2, cut2)) return LMBD_ENOMEM;
      cutC = cutA;
      arena_need = std::max(maxw(cutA, s1_and_x), maxw(cut2, s2));
    }
    if (!reverse_only && (c->arena.bytes < arena_need || (c->mem_budget && c->arena.bytes > avail))) {
      release(c->arena);
      size_t want = std::min(arena_need + arena_need / 8, std::max(avail, arena_need));
      if (cudaMalloc(&c->arena.p, want) != cudaSuccess) {
        cudaGetLastError();
        c->arena.p = nullptr;
        return LMBD_ENOMEM;
      }
      c->arena.bytes = want;
    }
  }
  char* const arena = (char*)c->arena.p;
  std::vector<std::vector<Bucket>> bucketsA, bucketsC;
  make_buckets(c->counts_h, cutA, c->order1_h, bucketsA, c->bucket_width);
  CK(cudaMemcpyAsync(c->order1_d.p, c->order1_h.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s));
  const int* orderA = (const int*)c->order1_d.p;
  const int* orderC = orderA;
  if (forces && cutC != cutA) {
    make_buckets(c->counts_h, cutC, c->order3_h, bucketsC, c->bucket_width);
    CK(cudaMemcpyAsync(c->order3_d.p, c->order3_h.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s));
    orderC = (const int*)c->order3_d.p;
  } else {
    bucketsC = bucketsA;
  }
  const int nwA = (int)cutA.size() - 1, nw2 = (int)cut2.size() - 1, nwC = (int)cutC.size() - 1;
  const bool one_wave = nwA == 1 && nw2 == 1 && nwC == 1;
  const bool per_atom = c->launch_mode == LMBD_LAUNCH_PER_ATOM;

  // stage-1 forward of one wave: pair lists, FP32 factorisation, refined solutions, alpha_K
  bool kmark_fwd = false;   // record kev[0], kev[1] around the factor buckets (pass A, profiling)
  bool tally_lu = true;     // count LU-fallback systems in pass A only (pass C may recompute)
  auto stage1_forward = [&](int wv, const std::vector<int>& cuts, const std::vector<std::vector<Bucket>>& bk,
                            const int* order) -> int {
    const int c0 = cuts[wv], c1 = cuts[wv + 1];
    L.stage1(o, c0, c1, arena, &w);
    CK(cudaMemsetAsync(w.fb, 0, sizeof(int), s));   // LU-fallback list of this wave
    launch_scs_fill(w, dp, c0, c1, max_n12, max_n1, s);
    ++phase_launch[LMBD_PHASE_SCS];
    if (per_atom) {
      for (int cc = c0; cc < c1; ++cc)
        launch_scs_factor(w, dp, nullptr, cc, cc + 1, c->counts_h[cc].n1, c->counts_h[cc].n12, s);
      phase_launch[LMBD_PHASE_SCS] += c1 - c0;
    } else {
      if (kmark_fwd) cudaEventRecord(c->kev[0], s);
      nvtxRangePushA("lmbd SCS factor buckets");
      Fork fk(c, s, (int)bk[wv].size());
      for (size_t i = 0; i < bk[wv].size(); ++i) {
        const Bucket& b = bk[wv][i];
        launch_scs_factor(w, dp, order, b.b0, b.b1, b.n1, b.n12, fk.stream((int)i));
      }
      fk.join();
      nvtxRangePop();
      if (kmark_fwd) cudaEventRecord(c->kev[1], s);
      phase_launch[LMBD_PHASE_SCS] += (int)bk[wv].size();
    }
    launch_scs_lu_forward(w, dp, lu_blocks, max_n1, max_n12, tally_lu ? 1 : 0, s);
    ++phase_launch[LMBD_PHASE_SCS];
    CK(cudaGetLastError());
    return LMBD_OK;
  };

  // ---- pass A: stage 1 (SCS) of all centres --------------------------------------------------
  prof = prof_req && one_wave;
  mark(LMBD_PHASE_SCS);
  launch_pair_radial(w, dp, s);
  ++phase_launch[LMBD_PHASE_SCS];
  kmark_fwd = prof && !per_atom;
  if (reverse_only)   // the kept stage-1 arrays: their pointers, no work
    L.stage1(o, cutA[0], cutA[1], arena, &w);
  for (int wv = 0; wv < nwA && !reverse_only; ++wv) TRY(stage1_forward(wv, cutA, bucketsA, orderA));
  kmark_fwd = false;

  // ---- pass B: stage 2 (MBD energy) and its adjoint, per wave --------------------------------
  if (forces) {
    CK(cudaMemsetAsync(w.gacc, 0, sizeof(double) * 3 * N, s));
    CK(cudaMemsetAsync(w.alphaI_bar, 0, sizeof(double) * N * nq, s));
  }
  char* const base2 = arena + (persist ? R1 : 0);
  for (int wv = 0; wv < nw2; ++wv) {
    const int c0 = cut2[wv], c1 = cut2[wv + 1];
    unsigned short* wdig_raw = nullptr;
    L.stage2(o, c0, c1, base2, &w, &wdig_raw);
    // W digit planes at the wave's start for the digit count of each chain step
    auto chain_work = [&](int digits) {
      Work wm = w;
      const long long shift = L.tk > 0 ? (long long)c0 * 48 * digits * L.tk : o.at(O_KP, c0) * 48 * digits;
      if (wdig_raw)
        wm.wdig = reinterpret_cast<unsigned short*>(reinterpret_cast<uintptr_t>(wdig_raw) -
                                                    (uintptr_t)shift * sizeof(unsigned short));
      return wm;
    };
    if (!reverse_only) {   // the forward of stage 2 (kept state in a reverse sweep)
    if (per_atom) {
      for (int cc = c0; cc < c1; ++cc) {
        if (sparse)
          launch_sp_prepare(w, dp, cc, cc + 1, max_ns, s);
        else
          launch_mbd_prepare_sized(w, dp, cc, cc + 1, max_ns, s);
        if (sliced_chain) launch_slice_t(w, cc, cc + 1, ST, s);
        if (dp.lanczos) {
          if (!launch_series_coefficients(w, dp, cc, cc + 1, max_ns, s)) return LMBD_ECAPACITY;
          phase_launch[LMBD_PHASE_PREPARE] += 2;
        }
        if (dp.logmode && !launch_log_mode(w, dp, cc, cc + 1, max_ns, s)) return LMBD_ECAPACITY;
        for (int m = 1; m < (dp.logmode ? 1 : nvec); ++m) {
          const int dg = m + 1 <= (c->order + 1) / 2 ? DIG_E : DIG_A;
          if (sliced_chain && tc05) {
            if (!launch_chain_tc(chain_work(dg), dp, m, cc, cc + 1, max_ns, dg, ST, s)) return LMBD_ECUDA;
          }
          else if (sliced_chain)
            launch_chain_oz2(chain_work(dg), dp, m, cc, cc + 1, max_ns, dg, ST, s);
          else if (sparse)
            launch_sp_chain(w, dp, m, cc, cc + 1, max_ns, s);
          else
            launch_mbd_chain_sized(w, dp, m, cc, cc + 1, max_ns, s);
        }
        launch_mbd_energy(w, dp, cc, cc + 1, s);
      }
      phase_launch[LMBD_PHASE_PREPARE] += c1 - c0;
      phase_launch[LMBD_PHASE_CHAIN] += (c1 - c0) * (dp.logmode ? 1 : nvec - 1);
      phase_launch[LMBD_PHASE_ENERGY] += c1 - c0;
    } else {
      mark(LMBD_PHASE_PREPARE);
      if (sparse)
        launch_sp_prepare(w, dp, c0, c1, max_ns, s);
      else
        launch_mbd_prepare_sized(w, dp, c0, c1, max_ns, s);
      if (sliced_chain) launch_slice_t(w, c0, c1, ST, s);
      if (dp.lanczos) {
        if (!launch_series_coefficients(w, dp, c0, c1, max_ns, s)) return LMBD_ECAPACITY;
        phase_launch[LMBD_PHASE_PREPARE] += 2;
      }
      mark(LMBD_PHASE_CHAIN);
      // log mode: Lanczos Gauss rules of ln(1 - G) in place of the Krylov chain
      if (dp.logmode && !launch_log_mode(w, dp, c0, c1, max_ns, s)) return LMBD_ECAPACITY;
      for (int m = 1; m < (dp.logmode ? 1 : nvec); ++m) {
        const int dg = m + 1 <= (c->order + 1) / 2 ? DIG_E : DIG_A;
        if (sliced_chain && tc05) {
          if (!launch_chain_tc(chain_work(dg), dp, m, c0, c1, max_ns, dg, ST, s)) return LMBD_ECUDA;
        }
        else if (sliced_chain)
          launch_chain_oz2(chain_work(dg), dp, m, c0, c1, max_ns, dg, ST, s);
        else if (sparse)
          launch_sp_chain(w, dp, m, c0, c1, max_ns, s);
        else
          launch_mbd_chain_sized(w, dp, m, c0, c1, max_ns, s);
      }
      mark(LMBD_PHASE_ENERGY);
      launch_mbd_energy(w, dp, c0, c1, s);
      phase_launch[LMBD_PHASE_PREPARE] += 1;
      phase_launch[LMBD_PHASE_CHAIN] += dp.logmode ? 1 : nvec - 1;
      phase_launch[LMBD_PHASE_ENERGY] += 1;
    }
    }   // !reverse_only
    CK(cudaGetLastError());
    if (!forces || split == 1) continue;   // energies only, or the forward state kept
    CK(cudaMemsetAsync(w.rbar + o.at(O_S, c0), 0, sizeof(double) * o.span(O_S, c0, c1), s));
    if (per_atom) {
      for (int cc = c0; cc < c1; ++cc) {
        if (dp.paper) {
          launch_paper_force_seeds(w, dp, cc, cc + 1, max_ns, s);
        } else {
          launch_mbd_adj_series(w, dp, cc, cc + 1, s);
          if (sliced_pair && tc05) {
            if (!launch_pair_tc(w, dp, cc, cc + 1, max_ns, DIG_P, s)) return LMBD_ECUDA;
          }
          else if (sliced_pair)
            launch_mbd_adj_pair_oz2(w, dp, cc, cc + 1, max_ns, DIG_P, s);
          else if (sparse)
            launch_sp_adj_pair(w, dp, cc, cc + 1, max_pairs, s);
          else
            launch_mbd_adj_pair(w, dp, cc, cc + 1, max_ns, s);
        }
        launch_mbd_adj_blend(w, dp, cc, cc + 1, s);
      }
      phase_launch[LMBD_PHASE_ADJ_SERIES] += c1 - c0;
      phase_launch[LMBD_PHASE_ADJ_PAIR] += c1 - c0;
      phase_launch[LMBD_PHASE_ADJ_BLEND] += c1 - c0;
    } else {
      mark(LMBD_PHASE_ADJ_SERIES);
      if (dp.paper) {
        launch_paper_force_seeds(w, dp, c0, c1, max_ns, s);
        mark(LMBD_PHASE_ADJ_PAIR);
      } else {
        launch_mbd_adj_series(w, dp, c0, c1, s);
        mark(LMBD_PHASE_ADJ_PAIR);
        if (sliced_pair && tc05) {
          if (!launch_pair_tc(w, dp, c0, c1, max_ns, DIG_P, s)) return LMBD_ECUDA;
        }
        else if (sliced_pair)
          launch_mbd_adj_pair_oz2(w, dp, c0, c1, max_ns, DIG_P, s);
        else if (sparse)
          launch_sp_adj_pair(w, dp, c0, c1, max_pairs, s);
        else
          launch_mbd_adj_pair(w, dp, c0, c1, max_ns, s);
      }
      mark(LMBD_PHASE_ADJ_BLEND);
      launch_mbd_adj_blend(w, dp, c0, c1, s);
      phase_launch[LMBD_PHASE_ADJ_SERIES] += 1;
      phase_launch[LMBD_PHASE_ADJ_PAIR] += 1;
      phase_launch[LMBD_PHASE_ADJ_BLEND] += 1;
    }
    CK(cudaGetLastError());
  }

  // ---- pass C: SCS adjoint (needs dL/d alpha_I of every centre, complete after pass B) --------
  tally_lu = false;
  if (forces && split != 1) {
    mark(LMBD_PHASE_ADJ_SCS);
    for (int wv = 0; wv < nwC; ++wv) {
      const int c0 = cutC[wv], c1 = cutC[wv + 1];
      size_t x_at = R1;
      if (!persist) {
        TRY(stage1_forward(wv, cutC, bucketsC, orderC));
        x_at = s1(c0, c1);
      }
      L.scs_adjoint(o, c0, c1, arena + x_at, &w);
      if (per_atom) {
        for (int cc = c0; cc < c1; ++cc)
          launch_scs_adjoint2(w, dp, nullptr, cc, cc + 1, c->counts_h[cc].n1, c->counts_h[cc].n12, s);
        launch_scs_lu_adjoint(w, dp, lu_blocks, c0, c1, max_n1, max_n12, s);
        for (int cc = c0; cc < c1; ++cc) launch_scs_site_reduce(w, dp, cc, cc + 1, s);
        phase_launch[LMBD_PHASE_ADJ_SCS] += 2 * (c1 - c0) + 1;
      } else {
        if (prof) cudaEventRecord(c->kev[2], s);
        nvtxRangePushA("lmbd SCS adjoint buckets");
        Fork fk(c, s, (int)bucketsC[wv].size());
        for (size_t i = 0; i < bucketsC[wv].size(); ++i) {
          const Bucket& b = bucketsC[wv][i];
          launch_scs_adjoint2(w, dp, orderC, b.b0, b.b1, b.n1, b.n12, fk.stream((int)i));
        }
        fk.join();
        nvtxRangePop();
        if (prof) cudaEventRecord(c->kev[3], s);
        launch_scs_lu_adjoint(w, dp, lu_blocks, c0, c1, max_n1, max_n12, s);
        launch_scs_site_reduce(w, dp, c0, c1, s);
        phase_launch[LMBD_PHASE_ADJ_SCS] += (int)bucketsC[wv].size() + 2;
      }
      CK(cudaGetLastError());
    }
  }
  c->stats.waves_scs = nwA;
  c->stats.waves_mbd = nw2;
  c->stats.scs_recomputed = (forces && !persist) ? 1 : 0;
  c->stats.bytes_arena = (double)c->arena.bytes;

  // ---- outputs ----------------------------------------------------------------------------------
  CK(cudaGetLastError());   // before is_device_ptr, which clears the error state of a failed query
  mark(LMBD_PHASE_OUTPUT);
  if (e_out) {
    bool dev = is_device_ptr(e_out);
    CK(cudaMemcpyAsync(e_out, w.energies, sizeof(double) * N, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  }
  if (forces && f_out) {
    bool dev = is_device_ptr(f_out);
    double* dst = f_out;
    if (!dev) {
      TRY(ensure(c->out_f_d, sizeof(double) * 3 * N));
      dst = (double*)c->out_f_d.p;
    }
    launch_forces_out(w, dst, s);
    ++phase_launch[LMBD_PHASE_OUTPUT];
    if (!dev) CK(cudaMemcpyAsync(f_out, dst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s));
  }
  mark(LMBD_NPHASE);
  if (split == 1 && one_wave && persist && !per_atom) {   // inputs of the kept forward state
    TRY(ensure(c->kept_pos, sizeof(double) * 3 * (size_t)N));
    TRY(ensure(c->kept_spec, sizeof(int) * (size_t)N));
    CK(cudaMemcpyAsync(c->kept_pos.p, w.pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->kept_spec.p, w.species, sizeof(int) * N, cudaMemcpyDeviceToDevice, s));
  }
  CK(cudaMemcpyAsync(c->status_h, w.status, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());

  // ---- statistics (algorithmic work from the actual sizes) ----------------------------------
  {
    const std::vector<Counts>& hc = c->counts_h;
    lmbd_stats& S = c->stats;
    S.tlr_pairs = 0;
    for (int i = 0; i < N; ++i) {
      double n1 = 3.0 * hc[i].n1, n = 3.0 * hc[i].ns;
      // coupled site pairs of the sparse path, every pair of the sphere on the dense one
      const double npair = sparse ? (double)(o.at(O_NP, i + 1) - o.at(O_NP, i)) : 0.5 * hc[i].ns * (hc[i].ns - 1.0);
      S.tlr_pairs += (long long)npair;
      S.flops[LMBD_PHASE_SCS] += dp.nqs * (n1 * n1 * n1 / 3.0 + 6.0 * n1 * n1);
      if (sparse)   // 9 multiply-adds per column of every entry (both blocks of a pair)
        S.flops[LMBD_PHASE_CHAIN] += (nvec - 1) * 2.0 * 9.0 * 2.0 * npair * ncv;
      else
        S.flops[LMBD_PHASE_CHAIN] += dp.logmode ? 3.0 * dp.logmode * 2.0 * n * n * nf : (nvec - 1) * 2.0 * n * n * ncv;
      if (forces) {
        if (sparse)
          S.flops[LMBD_PHASE_ADJ_PAIR] += 2.0 * 9.0 * npair * ncol;
        else
          S.flops[LMBD_PHASE_ADJ_PAIR] += 2.0 * (n * (n + 48.0) / 2.0) * ncol;   // lower tiles of P Q^T
        S.flops[LMBD_PHASE_ADJ_SCS] += dp.nqs * 6.0 * n1 * n1;
      }
    }
    for (int ph = 0; ph < LMBD_NPHASE; ++ph) {
      S.launches[ph] = phase_launch[ph];
      launches += ph == LMBD_PHASE_NEIGHBORS ? 0 : phase_launch[ph];
    }
    if (prof)
      for (int ph = 0; ph < LMBD_NPHASE; ++ph) {
        if (!marked[ph]) continue;
        int nx = ph + 1;
        while (nx <= LMBD_NPHASE && !marked[nx]) ++nx;
        float ms = 0.f;
        if (nx <= LMBD_NPHASE && cudaEventElapsedTime(&ms, c->ev[ph], c->ev[nx]) == cudaSuccess) S.ms[ph] = ms;
        cudaGetLastError();
      }
    if (prof && !per_atom) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->kev[0], c->kev[1]) == cudaSuccess) S.ms_kernel[0] = ms;
      cudaGetLastError();
      ms = 0.f;
      if (forces && cudaEventElapsedTime(&ms, c->kev[2], c->kev[3]) == cudaSuccess) S.ms_kernel[1] = ms;
      cudaGetLastError();
    }
    S.scs_lu_systems = c->status_h[2];
    S.reused_forward = reverse_only ? 1 : 0;
    S.spectral_flags = c->status_h[1];
    S.n_sites = c->totals_h[7];
    S.scs_pairs = c->totals_h[8];
    S.scs_adjacency = c->totals_h[9];
    S.max_k1 = max_n1;
    S.max_sphere = max_ns;
    S.max_sites = c->site_cap;
    S.kernel_launches = launches;
    S.bytes_workspace = (double)(c->whole_bytes() + c->arena.bytes);
  }
  // a tensor-core kernel that gave up leaves its outputs undefined, which later stages may
  // report as failures of their own: the timeout is the cause
  if (*c->status_h & LMBD_FLAG_TIMEOUT) return LMBD_ETIMEOUT;
  // the block-sparse fill found other partners than its count: cannot happen for one site list
  if (*c->status_h & LMBD_FLAG_PATTERN) return LMBD_ECUDA;
  if (*c->status_h & (LMBD_FLAG_NOT_SPD | LMBD_FLAG_NOT_CONVERGED)) return LMBD_NOT_SPD;
  if (*c->status_h & LMBD_FLAG_MODEL) return LMBD_EMODEL;
  if (split == 1 && one_wave && persist && !per_atom) {
    c->kept_valid = true;
    c->kept_n = N;
  }
  if (c->spectral_fail && c->status_h[1] > 0) return LMBD_CATASTROPHE;
  return LMBD_OK;
}

}  // namespace

struct lmbd_ctx {
  Ctx c;
};

extern "C" {

int lmbd_default_params(lmbd_params* out) {
  if (!out) return LMBD_EINVAL;
  out->r_scs = 5.0;
  out->r_mbd1 = 7.0;
  out->r_mbd2 = 7.0;
  out->r_sphere = 7.0;
  out->r_buf = 0.5;
  out->r_inner = 2.0;
  out->beta = 0.83;
  out->d = 6.0;
  out->omega_scale = 0.6;
  return LMBD_OK;
}

int lmbd_create(const lmbd_species* species, int n_species, const lmbd_params* params, int n_freq,
                int series_order, lmbd_ctx** out) {
  if (!out || !species || !params || n_species <= 0) return LMBD_EINVAL;
  *out = nullptr;
  if (n_freq < 1 || n_freq > LMBD_MAX_FREQ) return LMBD_EINVAL;
  if (series_order < 2 || series_order > LMBD_MAX_ORDER) return LMBD_EUNSUPPORTED;
  const lmbd_params& p = *params;
  double rs = p.r_sphere > 0 ? p.r_sphere : p.r_mbd1 + p.r_mbd2;
  if (!(p.r_scs > 0) || !(p.r_buf > 0) || !(p.r_inner > 0) || !(p.r_mbd1 > 0) || !(p.r_mbd2 > 0) ||
      !(p.beta > 0) || !(p.d > 0) || !(p.omega_scale > 0) || p.r_scs > rs || p.r_buf > p.r_scs ||
      p.r_buf > p.r_mbd1 || p.r_buf > p.r_mbd2)
    return LMBD_EINVAL;
  for (int i = 0; i < n_species; ++i)
    if (!(species[i].alpha0 > 0) || !(species[i].c6 > 0) || !(species[i].r0 > 0)) return LMBD_EINVAL;
  lmbd_ctx* h = new (std::nothrow) lmbd_ctx();
  if (!h) return LMBD_ENOMEM;
  Ctx& c = h->c;
  c.prm = p;
  c.n_species = n_species;
  c.n_freq = n_freq;
  c.order = series_order;
  c.table.resize(3 * n_species);
  for (int i = 0; i < n_species; ++i) {
    c.table[3 * i] = species[i].alpha0;
    c.table[3 * i + 1] = species[i].c6;
    c.table[3 * i + 2] = species[i].r0;
  }
  gauss_legendre(n_freq, p.omega_scale, c.omega, c.weight);
  int st = ensure(c.table_d, sizeof(double) * c.table.size());
  if (st == LMBD_OK &&
      cudaMemcpy(c.table_d.p, c.table.data(), sizeof(double) * c.table.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    st = LMBD_ECUDA;
  if (st == LMBD_OK && cudaMallocHost((void**)&c.totals_h, sizeof(long long) * 16) != cudaSuccess) st = LMBD_ENOMEM;
  if (st == LMBD_OK && cudaMallocHost((void**)&c.status_h, sizeof(int) * 4) != cudaSuccess) st = LMBD_ENOMEM;
  if (st != LMBD_OK) {
    cudaGetLastError();
    lmbd_destroy(h);
    return st;
  }
  *out = h;
  return LMBD_OK;
}

// The paper's forces with the fitted integrand (Sec. III.D): one pass per sample frequency
// (omega = 0 and the fit nodes), each returning the force integrand at that sample, then the
// theta fit per atom and component.  The energies (fitted integrand phi) come from the first pass.
int run_theta(Ctx* c, int N, const double* pos, const double* cell, const int* spec, const double* nu,
              const double* w_in, double* e_out, double* f_out, cudaStream_t s) {
  const int J = c->fit_nodes + 1;
  if (N == 0) return run(c, N, pos, cell, spec, nu, w_in, e_out, f_out, s);
  TRY(ensure(c->theta_f, sizeof(double) * 3 * (size_t)N * J));
  TRY(ensure(c->theta_out, sizeof(double) * 3 * (size_t)N));
  double* Fj = (double*)c->theta_f.p;
  int st = LMBD_OK;
  for (int j = 0; j < J && st == LMBD_OK; ++j) {
    c->theta_sample = j;
    st = run(c, N, pos, cell, spec, nu, w_in, j == 0 ? e_out : nullptr, Fj + (size_t)j * 3 * N, s);
  }
  c->theta_sample = -1;
  if (st != LMBD_OK) return st;
  ThetaParams tp{};
  tp.J = J;
  tp.M = tp.K = std::min(c->fit_nodes / 2, 5);
  tp.nphi = c->n_freq;
  tp.nu[0] = 0.0;
  for (int j = 1; j < J; ++j) tp.nu[j] = c->fit_omega[j];
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < c->n_freq; ++i) {
    tp.om[i] = c->omega[i];
    tp.wt[i] = c->weight[i] / (2.0 * pi);
  }
  int* status = (int*)c->status.p;
  CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  const bool dev = is_device_ptr(f_out);
  double* dst = dev ? f_out : (double*)c->theta_out.p;
  launch_theta_fit(N, Fj, tp, dst, status, s);
  CK(cudaGetLastError());
  if (!dev) CK(cudaMemcpyAsync(f_out, dst, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->status_h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*c->status_h & LMBD_FLAG_MODEL) return LMBD_EMODEL;
  return LMBD_OK;
}

int lmbd_energy_forces_weighted(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell,
                                const int* species, const double* hirshfeld, const double* energy_weights,
                                double* energies, double* forces, void* stream) {
  if (!ctx || n_atoms < 0) return LMBD_EINVAL;
  if (n_atoms > 0 && (!positions || !species || !hirshfeld)) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  int st = forces && c.paper_forces && c.fit_nodes
               ? run_theta(&c, n_atoms, positions, cell, species, hirshfeld, energy_weights, energies, forces,
                           (cudaStream_t)stream)
               : run(&c, n_atoms, positions, cell, species, hirshfeld, energy_weights, energies, forces,
                     (cudaStream_t)stream);
  if (st != LMBD_OK) cudaGetLastError();
  return st;
}

int lmbd_energy_keep(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell, const int* species,
                     const double* hirshfeld, double* energies, void* stream) {
  if (!ctx || n_atoms < 0) return LMBD_EINVAL;
  if (n_atoms > 0 && (!positions || !species || !hirshfeld)) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  if (c.paper_forces && c.fit_nodes) {   // the fitted force integrand needs its own passes
    c.kept_valid = false;
    return lmbd_energy_forces(ctx, n_atoms, positions, cell, species, hirshfeld, energies, nullptr, stream);
  }
  c.split = c.logmode || c.launch_mode == LMBD_LAUNCH_PER_ATOM ? 0 : 1;
  int st = run(&c, n_atoms, positions, cell, species, hirshfeld, nullptr, energies, nullptr, (cudaStream_t)stream);
  c.split = 0;
  if (st != LMBD_OK) {
    c.kept_valid = false;
    cudaGetLastError();
  }
  return st;
}

int lmbd_forces_kept(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell, const int* species,
                     const double* hirshfeld, const double* energy_weights, double* forces, void* stream) {
  if (!ctx || n_atoms < 0 || (n_atoms > 0 && !forces)) return LMBD_EINVAL;
  if (n_atoms > 0 && (!positions || !species || !hirshfeld)) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  if (c.kept_valid && c.kept_n == n_atoms && n_atoms > 0) {
    c.split = 2;
    int st = run(&c, n_atoms, positions, cell, species, hirshfeld, energy_weights, nullptr, forces,
                 (cudaStream_t)stream);
    c.split = 0;
    c.kept_valid = false;   // the reverse sweep overwrites the stage-2 arrays
    if (st != LMBD_ESTALE) {
      if (st != LMBD_OK) cudaGetLastError();
      return st;
    }
  }
  return lmbd_energy_forces_weighted(ctx, n_atoms, positions, cell, species, hirshfeld, energy_weights, nullptr,
                                     forces, stream);
}

int lmbd_energy_forces(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell,
                       const int* species, const double* hirshfeld, double* energies, double* forces,
                       void* stream) {
  return lmbd_energy_forces_weighted(ctx, n_atoms, positions, cell, species, hirshfeld, nullptr, energies,
                                     forces, stream);
}

int lmbd_autotune(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell, const int* species,
                  const double* hirshfeld, double* energies, double* forces, void* stream, int* bucket_width) {
  if (!ctx || n_atoms <= 0 || !positions || !species || !hirshfeld || !energies) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  if (c.launch_mode != LMBD_LAUNCH_BATCHED) return LMBD_EINVAL;
  static const int cand[] = {2, 3, 4, 6, 8, 12, 16};
  const int save_prof = c.profiling, save_w = c.bucket_width;
  int st = lmbd_set_profiling(ctx, 1);
  if (st != LMBD_OK) return st;
  double best = 1e300;
  int best_w = save_w;
  for (int wdt : cand) {
    c.bucket_width = wdt;
    double t = 0.0;
    for (int rep = 0; rep < 2; ++rep) {       // the first call settles allocations, the second is timed
      st = run(&c, n_atoms, positions, cell, species, hirshfeld, nullptr, energies, forces, (cudaStream_t)stream);
      if (st != LMBD_OK) {
        cudaGetLastError();
        c.bucket_width = save_w;
        c.profiling = save_prof;
        return st;
      }
      t = c.stats.ms[LMBD_PHASE_SCS] + c.stats.ms[LMBD_PHASE_ADJ_SCS];
    }
    if (t < best) {
      best = t;
      best_w = wdt;
    }
  }
  c.bucket_width = best_w;
  c.profiling = save_prof;
  if (bucket_width) *bucket_width = best_w;
  return LMBD_OK;
}

int lmbd_set_profiling(lmbd_ctx* ctx, int on) {
  if (!ctx) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  if (on && !c.ev[0]) {
    for (int i = 0; i <= LMBD_NPHASE; ++i)
      if (cudaEventCreate(&c.ev[i]) != cudaSuccess) {
        cudaGetLastError();
        return LMBD_ECUDA;
      }
    for (int i = 0; i < 4; ++i)
      if (cudaEventCreate(&c.kev[i]) != cudaSuccess) {
        cudaGetLastError();
        return LMBD_ECUDA;
      }
  }
  c.profiling = on ? 1 : 0;
  return LMBD_OK;
}

int lmbd_set_spectral_check(lmbd_ctx* ctx, int fail) {
  if (!ctx || (fail != 0 && fail != 1)) return LMBD_EINVAL;
  ctx->c.spectral_fail = fail;
  return LMBD_OK;
}

int lmbd_set_sparse_tlr(lmbd_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return LMBD_EINVAL;
  ctx->c.sparse = on;
  ctx->c.kept_valid = false;   // a kept forward state has the other layout
  return LMBD_OK;
}

int lmbd_set_precision(lmbd_ctx* ctx, int mode) {
  if (!ctx || (mode != LMBD_PREC_FP64 && mode != LMBD_PREC_SLICED)) return LMBD_EINVAL;
  ctx->c.precision = mode;
  return LMBD_OK;
}

int lmbd_set_mma_path(lmbd_ctx* ctx, int path) {
  if (!ctx || (path != LMBD_MMA_WARP && path != LMBD_MMA_TC05)) return LMBD_EINVAL;
  ctx->c.mma_path = path;
  return LMBD_OK;
}

int lmbd_set_wait_budget(lmbd_ctx* ctx, long long cycles) {
  if (!ctx || cycles < 0) return LMBD_EINVAL;
  ctx->c.tc_wait = cycles;
  return LMBD_OK;
}

int lmbd_set_frequency_model(lmbd_ctx* ctx, int model, double omega_ref) {
  if (!ctx) return LMBD_EINVAL;
  if (model == LMBD_FREQ_QUADRATURE) {
    ctx->c.lorentz = 0;
    ctx->c.omega_ref = 0.0;
    return LMBD_OK;
  }
  if (model != LMBD_FREQ_LORENTZIAN || !(omega_ref > 0.0) || !std::isfinite(omega_ref)) return LMBD_EINVAL;
  ctx->c.lorentz = 1;
  ctx->c.omega_ref = omega_ref;
  return LMBD_OK;
}

static_assert(LMBD_FIT_ROWS == LMBD_MAX_FIT_NODES + 1 && LMBD_FITW >= LMBD_FIT_ROWS,
              "fit scratch sizes follow the public node limit");

int lmbd_set_integrand_fit(lmbd_ctx* ctx, int n_fit_nodes) {
  if (!ctx) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  if (n_fit_nodes == 0) {
    c.fit_nodes = 0;
    c.fit_omega.clear();
    return LMBD_OK;
  }
  if (n_fit_nodes < c.order || n_fit_nodes > LMBD_MAX_FIT_NODES) return LMBD_EINVAL;
  std::vector<double> om, wt;
  gauss_legendre(n_fit_nodes, c.prm.omega_scale, om, wt);
  c.fit_omega.assign(1, 0.0);
  c.fit_omega.insert(c.fit_omega.end(), om.begin(), om.end());
  c.fit_nodes = n_fit_nodes;
  return LMBD_OK;
}

int lmbd_set_force_model(lmbd_ctx* ctx, int model) {
  if (!ctx || (model != LMBD_FORCES_EXACT && model != LMBD_FORCES_PAPER)) return LMBD_EINVAL;
  ctx->c.paper_forces = model == LMBD_FORCES_PAPER;
  return LMBD_OK;
}

int lmbd_set_verlet_skin(lmbd_ctx* ctx, double skin) {
  if (!ctx || !(skin >= 0.0) || !std::isfinite(skin)) return LMBD_EINVAL;
  ctx->c.skin = skin;
  ctx->c.ref_valid = false;
  return LMBD_OK;
}

int lmbd_set_log_mode(lmbd_ctx* ctx, int lanczos_steps) {
  if (!ctx || lanczos_steps < 0 || lanczos_steps > LMBD_MAX_LANCZOS) return LMBD_EINVAL;
  ctx->c.logmode = lanczos_steps;
  return LMBD_OK;
}

int lmbd_set_series_fit(lmbd_ctx* ctx, int lanczos_steps) {
  if (!ctx || lanczos_steps < 0 || lanczos_steps > LMBD_MAX_LANCZOS) return LMBD_EINVAL;
  ctx->c.lanczos = lanczos_steps;
  return LMBD_OK;
}

int lmbd_set_memory_budget(lmbd_ctx* ctx, size_t bytes) {
  if (!ctx) return LMBD_EINVAL;
  ctx->c.mem_budget = bytes;
  return LMBD_OK;
}

int lmbd_release_workspace(lmbd_ctx* ctx) {
  if (!ctx) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  for (int i = 0; i < c.n_whole; ++i)
    if (c.whole_bufs[i] != &c.table_d) release(*c.whole_bufs[i]);
  release(c.arena);
  c.last_n = 0;
  c.ref_valid = false;
  c.kept_valid = false;
  return LMBD_OK;
}

int lmbd_held_bytes(const lmbd_ctx* ctx, size_t* out) {
  if (!ctx || !out) return LMBD_EINVAL;
  *out = ctx->c.whole_bytes() + ctx->c.arena.bytes;
  return LMBD_OK;
}

int lmbd_set_launch_mode(lmbd_ctx* ctx, int mode) {
  if (!ctx || (mode != LMBD_LAUNCH_BATCHED && mode != LMBD_LAUNCH_PER_ATOM)) return LMBD_EINVAL;
  ctx->c.launch_mode = mode;
  return LMBD_OK;
}

int lmbd_get_central_polarizabilities(lmbd_ctx* ctx, double* out, void* stream) {
  if (!ctx || !out) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  if (c.last_n == 0) return LMBD_OK;
  cudaStream_t s = (cudaStream_t)stream;
  bool dev = is_device_ptr(out);
  if (cudaMemcpyAsync(out, c.alphaI.p, sizeof(double) * c.last_n * c.last_nqs,
                      dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LMBD_ECUDA;
  }
  return LMBD_OK;
}

int lmbd_get_site_counts(lmbd_ctx* ctx, int* out, void* stream) {
  if (!ctx || !out) return LMBD_EINVAL;
  Ctx& c = ctx->c;
  if (c.last_n == 0) return LMBD_OK;
  cudaStream_t s = (cudaStream_t)stream;
  bool dev = is_device_ptr(out);
  if (cudaMemcpyAsync(out, c.counts.p, sizeof(Counts) * c.last_n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LMBD_ECUDA;
  }
  return LMBD_OK;
}

int lmbd_get_quadrature(const lmbd_ctx* ctx, double* omega, double* weight) {
  if (!ctx || !omega || !weight) return LMBD_EINVAL;
  for (int i = 0; i < ctx->c.n_freq; ++i) {
    omega[i] = ctx->c.omega[i];
    weight[i] = ctx->c.weight[i];
  }
  return LMBD_OK;
}

int lmbd_get_stats(const lmbd_ctx* ctx, lmbd_stats* out) {
  if (!ctx || !out) return LMBD_EINVAL;
  *out = ctx->c.stats;
  return LMBD_OK;
}

int lmbd_destroy(lmbd_ctx* ctx) {
  if (!ctx) return LMBD_OK;
  Ctx& c = ctx->c;
  for (int i = 0; i < c.n_whole; ++i) release(*c.whole_bufs[i]);
  release(c.arena);
  for (int i = 0; i <= LMBD_NPHASE; ++i)
    if (c.ev[i]) cudaEventDestroy(c.ev[i]);
  for (int i = 0; i < 4; ++i)
    if (c.kev[i]) cudaEventDestroy(c.kev[i]);
  for (int i = 0; i < Ctx::kSide; ++i) {
    if (c.side[i]) cudaStreamDestroy(c.side[i]);
    if (c.join_ev[i]) cudaEventDestroy(c.join_ev[i]);
  }
  if (c.fork_ev) cudaEventDestroy(c.fork_ev);
  if (c.totals_h) cudaFreeHost(c.totals_h);
  if (c.status_h) cudaFreeHost(c.status_h);
  delete ctx;
  return LMBD_OK;
}

const char* lmbd_status_string(int status) {
  switch (status) {
    case LMBD_OK: return "ok";
    case LMBD_EINVAL: return "invalid argument";
    case LMBD_ENOMEM: return "device allocation failed";
    case LMBD_NOT_SPD: return "screening matrix singular (zero pivot in the LU fallback)";
    case LMBD_ECUDA: return "CUDA runtime error";
    case LMBD_ECAPACITY: return "too many sites around one atom for the kernels";
    case LMBD_EUNSUPPORTED: return "unsupported option";
    case LMBD_ESCRATCH: return "problem exceeds the fixed scratch of the allocation-free entry point";
    case LMBD_EMODEL: return "Lorentzian frequency model not applicable: a polarisability rises between 0 and omega_ref";
    case LMBD_ETIMEOUT: return "a bounded device wait in a tensor-core kernel ran out";
    case LMBD_CATASTROPHE: return "spectral proxy of G reached 1 for some centre and frequency (polarisation catastrophe); outputs were written";
    default: return "unknown status";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Allocation-free central polarisabilities (lmbd_central_polarizabilities_noalloc).
// Every buffer is carved from the library's static device scratch array; the host side
// uses fixed-size stack arrays only.  Nothing here allocates memory.
// ---------------------------------------------------------------------------------------
namespace {

// Regions of the fixed scratch array, 256-byte aligned.  A region that does not fit sets
// the sticky `failed` bit (and yields nullptr); the caller tests the bit once, before any
// device work, so no kernel ever receives a pointer past the array.
struct Carve {
  unsigned char* base;
  size_t used, cap;
  bool failed;
  template <class T>
  T* take(size_t n) {
    size_t off = (used + 255) & ~size_t(255);
    size_t bytes = n * sizeof(T);
    if (failed || off + bytes > cap) {
      failed = true;
      return nullptr;
    }
    used = off + bytes;
    return reinterpret_cast<T*>(base + off);
  }
};

// Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n, mapped to [0, inf);
// fixed-size output arrays (n <= LMBD_MAX_FREQ).
void gauss_legendre_fixed(int n, double L, double* om, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double x = z, wx = 2.0 / ((1.0 - z * z) * dp * dp);
    om[n - 1 - i] = L * (1.0 + x) / (1.0 - x);
    w[n - 1 - i] = 2.0 * L * wx / ((1.0 - x) * (1.0 - x));
  }
}

int noalloc_central(const lmbd_species* species_params, int n_species, const lmbd_params* params, int n_freq,
                    int N, const double* positions, const double* cell, const int* species,
                    const double* hirshfeld, double* alpha_central, cudaStream_t s) {
  const lmbd_params& P = *params;
  double rsph = sphere_radius(P);
  if (!(P.r_scs > 0) || !(P.r_buf > 0) || !(P.r_inner > 0) || !(P.r_mbd1 > 0) || !(P.r_mbd2 > 0) ||
      !(P.beta > 0) || !(P.d > 0) || !(P.omega_scale > 0) || P.r_scs > rsph || P.r_buf > P.r_scs)
    return LMBD_EINVAL;
  for (int i = 0; i < n_species; ++i)
    if (!(species_params[i].alpha0 > 0) || !(species_params[i].c6 > 0) || !(species_params[i].r0 > 0))
      return LMBD_EINVAL;
  if (!is_device_ptr(species))
    for (int i = 0; i < N; ++i)
      if (species[i] < 0 || species[i] >= n_species) return LMBD_EINVAL;
  if (!is_device_ptr(hirshfeld))
    for (int i = 0; i < N; ++i)
      if (!(hirshfeld[i] > 0.0) || !std::isfinite(hirshfeld[i])) return LMBD_EINVAL;
  if (!is_device_ptr(positions))
    for (int i = 0; i < 3 * N; ++i)
      if (!std::isfinite(positions[i])) return LMBD_EINVAL;

  void* base = nullptr;
  size_t cap = 0;
  if (noalloc_scratch(&base, &cap) != 0) return LMBD_ECUDA;
  const int nq = n_freq + 1;

  // parameters (same definitions as lmbd_energy_forces)
  DevParams dp{};
  const double ib = 1.0 / LMBD_BOHR;
  const double rlist = fmax(2.0 * P.r_scs, rsph);
  dp.r_scs = P.r_scs * ib;
  dp.r_mbd1 = P.r_mbd1 * ib;
  dp.r_mbd2 = P.r_mbd2 * ib;
  dp.r_buf = P.r_buf * ib;
  dp.r_inner = P.r_inner * ib;
  dp.beta = P.beta;
  dp.d = P.d;
  dp.r2_scs_ang = P.r_scs * P.r_scs;
  dp.r2_sphere_ang = rsph * rsph;
  dp.r2_scs2_ang = 4.0 * P.r_scs * P.r_scs;
  dp.r2_list_ang = rlist * rlist;
  dp.n_freq = n_freq;
  dp.nq = nq;
  dp.nqs = nq;
  dp.lorentz = 0;
  dp.order = 2;
  dp.n_species = n_species;
  double om[LMBD_MAX_FREQ], wt[LMBD_MAX_FREQ];
  gauss_legendre_fixed(n_freq, P.omega_scale, om, wt);
  for (int q = 0; q < n_freq; ++q) dp.omega[q + 1] = om[q];
  for (int q = 0; q < nq; ++q) dp.omega_s[q] = dp.omega[q];

  // search grid
  Grid g{};
  if (cell) {
    double hc[9];
    CK(cudaMemcpy(hc, cell, sizeof(hc), cudaMemcpyDefault));
    for (int i = 0; i < 9; ++i)
      if (!std::isfinite(hc[i])) return LMBD_EINVAL;
    double det = hc[0] * (hc[4] * hc[8] - hc[5] * hc[7]) - hc[1] * (hc[3] * hc[8] - hc[5] * hc[6]) +
                 hc[2] * (hc[3] * hc[7] - hc[4] * hc[6]);
    if (!(fabs(det) > 1e-9)) return LMBD_EINVAL;
    g.periodic = 1;
    memcpy(g.cell, hc, sizeof(hc));
    double inv[9] = {(hc[4] * hc[8] - hc[5] * hc[7]) / det, -(hc[1] * hc[8] - hc[2] * hc[7]) / det,
                     (hc[1] * hc[5] - hc[2] * hc[4]) / det, -(hc[3] * hc[8] - hc[5] * hc[6]) / det,
                     (hc[0] * hc[8] - hc[2] * hc[6]) / det, -(hc[0] * hc[5] - hc[2] * hc[3]) / det,
                     (hc[3] * hc[7] - hc[4] * hc[6]) / det, -(hc[0] * hc[7] - hc[1] * hc[6]) / det,
                     (hc[0] * hc[4] - hc[1] * hc[3]) / det};
    memcpy(g.inv, inv, sizeof(inv));
    for (int d = 0; d < 3; ++d) {
      const double* a = hc + 3 * ((d + 1) % 3);
      const double* b = hc + 3 * ((d + 2) % 3);
      double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
      double width = fabs(det) / sqrt(cx * cx + cy * cy + cz * cz);
      int nc = (int)(width / rlist);
      if (nc < 1) nc = 1;
      if (nc > 64) nc = 64;
      g.nc[d] = nc;
      g.reach[d] = (int)ceil(rlist / (width / nc) - 1e-12);
      if (g.reach[d] < 1) g.reach[d] = 1;
    }
  }
  const int ncells = cell ? g.nc[0] * g.nc[1] * g.nc[2] : 64 * 64 * 64;
  const int site_cap = LMBD_NOALLOC_SITE_CAP;

  // carve the scratch array
  Carve cv{static_cast<unsigned char*>(base), 0, cap, false};
  double* table = cv.take<double>(3 * (size_t)n_species);
  double* pos = cv.take<double>(3 * (size_t)N);
  int* spec = cv.take<int>(N);
  double* nu = cv.take<double>(N);
  Work w{};
  w.n_atoms = N;
  w.site_cap = site_cap;
  w.abar = cv.take<double>((size_t)N * nq);
  w.sig = cv.take<double>((size_t)N * nq);
  w.rvdw = cv.take<double>(N);
  w.a0 = cv.take<double>(N);
  w.r0 = cv.take<double>(N);
  w.wpos = cv.take<double>(3 * (size_t)N);
  w.cell_of = cv.take<int>(N);
  w.cell_count = cv.take<int>(ncells);
  w.cell_start = cv.take<int>(ncells + 1);
  w.cell_atoms = cv.take<int>(N);
  w.ncells = ncells;
  w.grid = cv.take<Grid>(1);
  w.wrap = cv.take<int>(3 * (size_t)N);
  w.site_img = cv.take<int>(3 * (size_t)N * site_cap);
  w.site_atom = cv.take<int>((size_t)N * site_cap);
  w.site_x = cv.take<double>(3 * (size_t)N * site_cap);
  w.counts = cv.take<Counts>(N);
  w.off_k1 = cv.take<long long>(N + 1);
  w.off_s = cv.take<long long>(N + 1);
  w.off_b = cv.take<long long>(N + 1);
  w.off_t = cv.take<long long>(N + 1);
  w.totals = cv.take<long long>(16);   // the offsets kernel writes 16 totals
  w.status = cv.take<int>(4);
  w.alphaI = cv.take<double>((size_t)N * nq);
  const long long slot_doubles = 9LL * LMBD_NOALLOC_MAX_K1 * LMBD_NOALLOC_MAX_K1;
  if (cv.failed) return LMBD_ESCRATCH;
  size_t used = (cv.used + 255) & ~size_t(255);
  long long nslots = (long long)((cap - used) / (sizeof(double) * slot_doubles));
  if (nslots > 128) nslots = 128;
  if (nslots < 1) return LMBD_ESCRATCH;
  double* slots = cv.take<double>((size_t)nslots * slot_doubles);
  if (cv.failed) return LMBD_ESCRATCH;
  w.pos = pos;
  w.species = spec;
  w.nu = nu;
  w.table = table;

  // inputs into the scratch (host or device sources)
  double htab[3 * 64];
  for (int i = 0; i < n_species; ++i) {
    htab[3 * i] = species_params[i].alpha0;
    htab[3 * i + 1] = species_params[i].c6;
    htab[3 * i + 2] = species_params[i].r0;
  }
  CK(cudaMemcpyAsync(table, htab, sizeof(double) * 3 * n_species, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(pos, positions, sizeof(double) * 3 * N, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(spec, species, sizeof(int) * N, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(nu, hirshfeld, sizeof(double) * N, cudaMemcpyDefault, s));
  CK(cudaMemsetAsync(w.status, 0, sizeof(int) * 4, s));   // flags must start at zero

  int launches = 0;
  launch_free_atom(w, dp, s);
  launch_neighbors(w, dp, g, s, &launches);
  launch_offsets(w, dp, s);
  CK(cudaGetLastError());
  long long tot[16];
  int flags = 0;
  CK(cudaMemcpyAsync(tot, w.totals, sizeof(tot), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&flags, w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flags & LMBD_FLAG_BAD_INPUT) return LMBD_EINVAL;
  if (flags & LMBD_FLAG_CAPACITY) return LMBD_ESCRATCH;
  if (flags & LMBD_FLAG_COINCIDENT) return LMBD_EINVAL;
  const int max_n1 = (int)tot[4], max_n12 = (int)tot[6];
  if (max_n1 > LMBD_NOALLOC_MAX_K1 || max_n12 > site_cap) return LMBD_ESCRATCH;
  launch_scs_central_noalloc(w, dp, slots, slot_doubles, (int)nslots, max_n12, max_n1, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(alpha_central, w.alphaI, sizeof(double) * N * nq, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(&flags, w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flags & LMBD_FLAG_NOT_SPD) return LMBD_NOT_SPD;
  return LMBD_OK;
}

}  // namespace

extern "C" int lmbd_central_polarizabilities_noalloc(const lmbd_species* species_params, int n_species,
                                                     const lmbd_params* params, int n_freq, int n_atoms,
                                                     const double* positions, const double* cell,
                                                     const int* species, const double* hirshfeld,
                                                     double* alpha_central, void* stream) {
  if (!species_params || !params || n_species <= 0 || n_species > 64 || n_freq < 1 || n_freq > LMBD_MAX_FREQ ||
      n_atoms < 0)
    return LMBD_EINVAL;
  // A capturing stream allows none of the synchronous copies and stream synchronisations of
  // this call (the sizes are read back to the host before the solve); refuse it before any
  // other CUDA call, so that the caller's capture stays valid.
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap_status) != cudaSuccess) {
    cudaGetLastError();
    return LMBD_EUNSUPPORTED;
  }
  if (cap_status != cudaStreamCaptureStatusNone) return LMBD_EUNSUPPORTED;
  if (n_atoms > LMBD_NOALLOC_MAX_ATOMS) return LMBD_ESCRATCH;
  if (n_atoms == 0) return LMBD_OK;
  if (!positions || !species || !hirshfeld || !alpha_central) return LMBD_EINVAL;
  int st = noalloc_central(species_params, n_species, params, n_freq, n_atoms, positions, cell, species,
                           hirshfeld, alpha_central, (cudaStream_t)stream);
  if (st != LMBD_OK) cudaGetLastError();
  return st;
}
