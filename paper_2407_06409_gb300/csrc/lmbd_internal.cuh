// Internal declarations of the lMBD CUDA library: device parameter block,
// workspace layout, pair functions of the model and kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define LMBD_BOHR 0.529177210903       // Angstrom per bohr, CODATA 2018
#define LMBD_HARTREE 27.211386245988   // eV per hartree, CODATA 2018
#define LMBD_MAXQ 65                   // omega = 0 plus up to 64 quadrature nodes
#define LMBD_MAX_ORDER_P1 11           // series order n_max <= 10

// Error bits written by kernels into the device status word.
#define LMBD_FLAG_NOT_SPD 1
#define LMBD_FLAG_CAPACITY 2
#define LMBD_FLAG_COINCIDENT 4
#define LMBD_FLAG_NOT_CONVERGED 8
#define LMBD_FLAG_MODEL 16          // Lorentzian model not applicable: alpha~(0) < alpha~(omega_ref),
                                    // or a fitted phi without decaying term
#define LMBD_FLAG_TIMEOUT 32        // a bounded device wait (tensor-core pipeline) ran out
// status[0]: the flags above; status[1]: (centre, frequency) terms whose spectral proxy reached
// 1 (energy kernel); status[2]: SCS systems solved by the LU fallback (forward pass)
#define LMBD_FLAG_BAD_INPUT 64      // a species index out of range, or a non-finite position or
                                    // non-positive Hirshfeld ratio, in device-resident inputs
#define LMBD_FLAG_PATTERN 128     // the block-sparse T_LR fill found other partners than its count
#define LMBD_FITW 32                // stride of the per-centre integrand weights dE/dI(omega_j)
#define LMBD_FIT_ROWS 25            // omega = 0 plus at most 24 fit nodes
#define LMBD_MAX_LANCZOS 64         // Lanczos steps of the polynomial-fit coefficients

struct DevParams {
  // lengths in bohr
  double r_scs, r_mbd1, r_mbd2, r_buf, r_inner, beta, d;
  // squared membership radii in Angstrom^2 (sets are decided on Angstrom distances)
  double r2_scs_ang, r2_sphere_ang, r2_scs2_ang, r2_list_ang;
  int n_freq;        // quadrature nodes
  int nq;            // n_freq + 1 (column 0 is omega = 0)
  int order;         // series order n_max
  int n_species;
  double omega[LMBD_MAXQ];
  double cweight[LMBD_MAXQ];  // hartree->eV * w_q / (2 pi) for q >= 1, 0 for q = 0
  // frequencies of the SCS solves: every omega[q] (nqs = nq), or with the Lorentzian model of
  // Sec. III.C (lorentz = 1) only 0 and omega_ref (nqs = 2)
  int nqs;
  int lorentz;
  double omega_ref;
  double omega_s[LMBD_MAXQ];
  // fitted integrand of Sec. III.C (fit = 1): omega[1..n_freq] are omega = 0 and the fit
  // nodes; the integral of phi uses the n_phi-point quadrature (phi_omega, phi_wt = w / 2 pi)
  int fit;
  int n_phi;
  // polynomial-fit series coefficients (Sec. III.A): Lanczos steps, 0 = c_n = -1/n
  int lanczos;
  // log mode (Sec. III.A, the n_max -> infinity limit): Lanczos steps of the Gauss rules of
  // [ln(1 - G)]_kk, 0 = the truncated series
  int logmode;
  double cn[LMBD_MAX_ORDER_P1];   // -1/n (Eq. E_k), so that kernels need no FP64 division
  // force model: 0 = exact gradient of sum_k w_k E_k, 1 = the paper's approximate forces
  // (Sec. III.D: F_k = -dE^{k,tot}/dr_k, alpha_I held, central row and column only for n >= 3)
  int paper;
  // bound of each mbarrier wait in the main loop of the tcgen05 kernels (SM clock cycles)
  long long tc_wait;
  double phi_omega[LMBD_MAXQ - 1];
  double phi_wt[LMBD_MAXQ - 1];
};

// Geometry of the neighbour search (host-computed from the cell).
struct Grid {
  int periodic;
  int nc[3];          // cells per direction
  int reach[3];       // cell offsets to scan per direction
  double cell[9];     // rows = lattice vectors (Angstrom)
  double inv[9];      // inverse of the cell matrix (frac = pos * inv)
  double origin[3];   // non-periodic: lower corner of the bounding box
  double h[3];        // non-periodic: cell edge length
};

// Per-centre counts: n1 = |K1|, ns = |sphere|, n12 = |K1 u K2|, nt = all sites.
struct Counts {
  int n1, ns, n12, nt;
};

// Workspace pointers handed to kernels (all device memory).
struct Work {
  int n_atoms;
  int site_cap;                // capacity of one centre's site list
  // inputs (device copies)
  const double* pos;           // N x 3 Angstrom
  const int* species;          // N
  const double* nu;            // N
  const double* table;         // S x 3
  const double* weights;       // N energy weights (NULL = ones)
  // free-atom quantities
  double* abar;                // N x nq
  double* sig;                 // N x nq
  double* rvdw;                // N
  double* a0;                  // N
  double* r0;                  // N
  // neighbour search
  double* wpos;                // N x 3 wrapped positions (Angstrom)
  int* cell_of;                // N
  int* cell_count;             // ncells
  int* cell_start;             // ncells + 1
  int* cell_atoms;             // N
  int ncells;
  Grid* grid;                  // device copy of the search grid
  int* wrap;                   // N x 3 lattice translation of each atom: pos = wpos + wrap C
  int* site_img;               // N x site_cap x 3 lattice image of each site relative to the
                               // unwrapped positions (site = pos_j + img C - pos_k)
  int* site_atom;              // N x site_cap
  double* site_x;              // N x site_cap x 3, displacement from the centre (bohr)
  Counts* counts;              // N
  // per-centre offsets (exclusive prefix sums, N + 1 entries)
  long long* off_k1;           // sum n1
  long long* off_s;            // sum ns
  long long* off_b;            // sum nq (3 n1)^2
  long long* off_t;            // sum (3 ns)^2
  long long* off_p;            // sum of SCS pairs per centre
  long long* off_a;            // sum of SCS adjacency entries per centre
  long long* totals;           // 16 entries written by the offsets kernel
  // SCS pair lists (one list per central atom; rows = coupled sites of K1)
  int* pcount;                 // N x 2: pairs, adjacency entries
  int* pr_ij;                  // pairs x 2: owner row i (K1), partner j (K1 with j < i, or K2)
  double* pr_geo;              // pairs x 8: r = x_j - x_i (3), |r|, F, dF/dr, 1/|r|, unused
  float2* pr_rad_ff;           // pairs x nq x 2: F A0, F B0 as float-float (residual updates)
  int* pr_g;                   // pairs: index of the pair in the atom-pair radial table, -1 = none
  // radial terms of T_SR per atom pair and frequency, independent of the central atom: entry
  // off_k1[a] + s is atom a with site s (1 <= s < n1) of its own K1 list
  double* rad_ab;              // sum n1 x nq x 2: A0, B0
  float2* rad_ff;              // sum n1 x nq x 4: A0, B0, dA0/dr, dB0/dr as float-float (hi, lo)
  float2* pr_gff;              // pairs x 6: r (3), F, dF/dr, 1/|r| as float-float (SCS adjoint)
  int* prow;                   // (sum n1 + N): first pair of each row, per centre n1 + 1 entries
  int* prow_k2;                // (sum n1 + N): first K2 pair of each row
  int* arow;                   // (sum n1 + N): first adjacency entry of each row
  int* adj;                    // entries x 2: K1 partner j, pair index
  int* k2ptr;                  // N x site_cap: first reverse-list entry of each K2 site
  int* k2rev;                  // per centre (off_p): pair indices grouped by K2 partner
  double* sgq;                 // N x site_cap x nq x 3: SCS-adjoint site gradients per frequency
  double* gstage;              // sum pairs x nq x 3: SCS-adjoint pair gradients (scratch; 8-byte
                               // entries, written and read as float-float pairs)
  float* lfac;                 // packed FP32 Cholesky factors, off_b
  float* binvg;                // inverses of their 16 x 16 diagonal blocks, binv_slot floats per
                               // (centre, SCS frequency), indexed by the global centre
  int binv_slot;
  // LU fallback of the SCS solves (systems whose FP32 Cholesky pivot is not positive or whose
  // refinement does not converge): fb[0] = count, fb[1 + e] = c * nqs + q; fb_flag[c * nqs + q]
  // = 1 for such a system (its FP32 factor is not used); lu: per-block dense slots of lu_slot
  // doubles ((3 max n1)^2)
  int* fb;
  int* fb_flag;
  double* lu;
  long long lu_slot;
  // sliced tensor-core products (ozaki.cuh)
  long long* off_tq;           // sum Mpad Kpad (T digit plane sizes)
  long long* off_tr;           // sum Mpad (T rows)
  long long* off_kp;           // sum Kpad (W digit planes are 48 x Kpad)
  long long* off_sp;           // sum ns16 (P, Q rows are 3 ns16)
  // tcgen05 path: T and W digit planes with one row pitch tk for all centres (0 on the warp-level
  // path, which uses each centre's Kpad), addressed through tensor maps over the current wave:
  // T rows [trow0, trow0 + trows) of the rebased pointer, W planes of centres [wc0, wc0 + wcn),
  // P and Q rows [prow0, prow0 + prows) (pitch Kp)
  int tk;
  long long trow0, trows;
  int wc0, wcn;
  long long prow0, prows;
  unsigned short* tdig;        // T digit planes (bf16 bits)
  int* texp;                   // T row scale exponents
  unsigned short* wdig;        // W digit planes
  int* wexp;                   // W column exponents, N x 48
  unsigned short* pdig;        // P digit planes
  unsigned short* qdig;        // Q digit planes
  int* pexp;                   // P row exponents
  int* qexp;                   // Q row exponents
  // stage 1 (SCS)
  double* bmat;                // FP64 matrices of the allocation-free variant
  double* xsol;                // X = B^-1 d, off_k1 * nq * 9
  double* alphaK;              // off_k1 * nq
  double* alphaI;              // N x nq
  // stage 2 (MBD)
  double* alphaT;              // blended alpha, off_s * nq
  double* tlr;                 // T_LR, off_t
  double* dsq;                 // sqrt(alpha~), off_s * nq
  double* vkr;                 // Krylov vectors: nvec blocks of (off_s total * 3) x (3 n_freq)
  int nvec;
  long long vstride;           // doubles per Krylov block
  double* energies;            // N, eV
  double* trbuf;               // N x 11 x 64 k-block traces tr_{n,q}
  // adjoint
  double* gbar;                // dL/d alpha~, off_s * nq
  double* fitw;                // N x LMBD_FITW: dE_k/dI_k(omega_j) of the fitted integrand
  double* cfit;                // N x n_freq x LMBD_MAX_ORDER_P1: fitted c_n per centre and frequency
  double* lam;                 // N x n_freq x 2: Lanczos estimate of G's spectral interval
  const double* gl64;          // 64 Gauss-Legendre nodes on [-1, 1], then their weights
  double* pmat;                // off_s*3 x ncol
  double* qmat;                // off_s*3 x ncol
  int ncol;                    // 3 n_freq (n_max - 2)
  double* x0buf;               // off_s x 9, central-column term of the pair matrix
  double* pcoef;               // off_t: per site pair (s > t) r (3) and 5 derivative coefficients
  double* rbar;                // dL/d R~ per sphere site, off_s
  // block-sparse T_LR (Sec. III.A: only the central row and column reach r_MBD,1, every other
  // pair couples within r_MBD,2): per centre the coupled site pairs (s, t), s > t, in row order,
  // and for every site s a row of entries (partner t, pair index), partners ascending
  int2* sp_cnt;                // N x site_cap: coupled partners below / above each site
  int* sp_np;                  // N: coupled pairs per centre
  long long* off_np;           // sum of coupled pairs per centre
  int4* sp_row;                // off_s: first entry, entries, first pair, pairs (partners below)
  int2* sp_ent;                // 2 off_np: partner site, pair index within the centre
  int2* sp_pair;               // off_np: (s, t), s > t
  float4* sp_blk;              // 3 off_np: T_LR,st as float-float (00, 11), (22, 01), (02, 12)
  float2* wff;                 // nvec blocks of (off_s total * 3) x (3 n_freq): W_m = D v_m as
                               // float-float, block m - 1 (P_j = W_j and Q of the adjoint)
  float2* dsq_ff;              // off_s x nq: sqrt(alpha~) as float-float
  float2* pff;                 // off_s*3 x ncol: P as float-float (replaces pmat)
  float2* qff;                 // off_s*3 x ncol: Q as float-float (replaces qmat)
  double* alphaK_bar;          // off_k1 * nq
  double* alphaI_bar;          // N x nq
  double* gacc;                // N x 3, dL/dR in eV/bohr (accumulated)
  int* status;                 // device status word
};

// ---------------------------------------------------------------------------------------
// model functions (device)
// ---------------------------------------------------------------------------------------
// f_SR / f_LR: 1 below rc - rb, 1 - 3t^2 + 2t^3 in the buffer, 0 beyond (Sec. III.A/B).
__device__ __forceinline__ void cutoff_buf(double r, double rc, double rb, double& f, double& df) {
  if (r < rc - rb) { f = 1.0; df = 0.0; return; }
  if (r >= rc) { f = 0.0; df = 0.0; return; }
  const double irb = 1.0 / rb;
  double t = (r - rc + rb) * irb;
  f = 1.0 - 3.0 * t * t + 2.0 * t * t * t;
  df = (-6.0 * t + 6.0 * t * t) * irb;
}

// f_inner (Sec. III.B): 3u^2 - 2u^3 with u = r/r_inner for r < r_inner, else 1.
__device__ __forceinline__ void finner(double r, double rin, double& f, double& df) {
  if (r >= rin) { f = 1.0; df = 0.0; return; }
  double u = r / rin;
  f = 3.0 * u * u - 2.0 * u * u * u;
  df = (6.0 * u - 6.0 * u * u) / rin;
}

// Fermi damping f(r, S) = 1/(1 + exp(-d (r/S - 1))) (Eq. damping-function) and
// its partial derivatives with respect to r and S.
__device__ __forceinline__ void fermi(double r, double s, double d, double& f, double& dfr, double& dfs) {
  const double is = 1.0 / s;
  const double x = r * is;
  double e = exp(-d * (x - 1.0));
  f = 1.0 / (1.0 + e);
  double g = f * (1.0 - f) * d * is;  // df/dr
  dfr = g;
  dfs = -g * x;                       // df/dS
}

// T_SR written as F(r) [A0(r) I + B0(r) r r^T] (Eq. T_SR with Eqs. g-func, h-func):
// A0 = g / r^3, B0 = (h~ - 3 g) / r^5 with x = r/sigma, h~ = (4/sqrt(pi)) x^3 exp(-x^2).
// Also returns the radial derivatives A0', B0'.
__device__ __forceinline__ void tsr_radial(double r, double sigma, double& A0, double& B0,
                                           double& dA0, double& dB0) {
  const double two_over_sqrtpi = 1.1283791670955126;
  double x = r / sigma;
  double ex = exp(-x * x);
  double g = erf(x) - two_over_sqrtpi * x * ex;
  double ht = 2.0 * two_over_sqrtpi * x * x * x * ex;
  double ir = 1.0 / r;
  double ir2 = ir * ir;
  double ir3 = ir2 * ir;
  double ir4 = ir2 * ir2;
  A0 = g * ir3;
  B0 = (ht - 3.0 * g) * ir4 * ir;
  dA0 = (ht - 3.0 * g) * ir4;
  dB0 = (15.0 * g - 5.0 * ht - 2.0 * x * x * ht) * ir4 * ir2;
}

__device__ __forceinline__ void tsr_value(double r, double sigma, double& A0, double& B0) {
  const double two_over_sqrtpi = 1.1283791670955126;
  double x = r / sigma;
  double ex = exp(-x * x);
  double g = erf(x) - two_over_sqrtpi * x * ex;
  double ht = 2.0 * two_over_sqrtpi * x * x * x * ex;
  double ir = 1.0 / r;
  double ir2 = ir * ir;
  A0 = g * ir2 * ir;
  B0 = (ht - 3.0 * g) * ir2 * ir2 * ir;
}

// Blended polarisabilities of sphere site s of centre c at every frequency (Eq. full-pol, or
// the Lorentzian model of Sec. III.C), written to alphaT and dsq; returns the SCS-scaled vdW
// radius R~_s (Eq. scaled-rvdw).  x: the site's displacement from the centre (bohr).
__device__ __forceinline__ double mbd_blend_site(const Work& w, const DevParams& p, int s, int a, int n1,
                                                 long long offs, long long offk1, double x0, double x1, double x2) {
  double fs = 0.0;
  if (s < n1 && s > 0) {
    double u = sqrt(x0 * x0 + x1 * x1 + x2 * x2) / p.r_scs;
    fs = 3.0 * u * u - 2.0 * u * u * u;
  }
  if (!p.lorentz) {
    for (int q = 0; q < p.nq; ++q) {
      double aI = w.alphaI[(long long)a * p.nqs + q];
      double at = aI;
      if (s < n1) at = (1.0 - fs) * w.alphaK[(offk1 + s) * p.nqs + q] + fs * aI;
      w.alphaT[(offs + s) * p.nq + q] = at;
      w.dsq[(offs + s) * p.nq + q] = sqrt(at);
    }
  } else {
    // alpha~(omega) = alpha~(0) / (1 + (omega/omega~)^2) with
    // (omega/omega~)^2 = (omega/omega_ref)^2 (alpha~(0)/alpha~(omega_ref) - 1) (Eq. char-freq)
    double ab[2];
    for (int qs = 0; qs < 2; ++qs) {
      const double aI = w.alphaI[(long long)a * 2 + qs];
      ab[qs] = (s < n1) ? (1.0 - fs) * w.alphaK[(offk1 + s) * 2 + qs] + fs * aI : aI;
    }
    double ratio = ab[0] / ab[1];
    if (!(ratio >= 1.0)) {   // alpha~ rises with frequency: Eq. char-freq has no real solution
      atomicOr(w.status, LMBD_FLAG_MODEL);
      ratio = 1.0;
    }
    for (int q = 0; q < p.nq; ++q) {
      const double u = p.omega[q] / p.omega_ref;
      const double at = ab[0] / (1.0 + u * u * (ratio - 1.0));
      w.alphaT[(offs + s) * p.nq + q] = at;
      w.dsq[(offs + s) * p.nq + q] = sqrt(at);
    }
  }
  return w.r0[a] * cbrt(w.alphaT[(offs + s) * p.nq] / w.a0[a]);
}

// T_LR block of the site pair at displacement rr = x_t - x_s (bohr) with SCS radii R~_s, R~_t
// and cutoff rc: blk = f_LR f(r, S~) T(rr) (symmetric, 0 beyond rc), and with kc non-null the
// derivative coefficients of d<M, T_LR>/dr = (k1 r.M.r + k2 Tr M) r + k3 M r and
// d<M, T_LR>/dS~ beta = k4 r.M.r + k5 Tr M (both pair blocks counted).  FP64 throughout; the
// operation count is kept low because every site pair of every sphere goes through it on the
// FP64 pipe: 1/r from one reciprocal square root, the Fermi damping (Eq. damping-function) with
// x = r / S~ as the only division besides 1/(1 + e), its derivatives through 1/r, and the six
// distinct entries of the symmetric block from two shared factors.
__device__ __forceinline__ void tlr_pair_block(const DevParams& p, const double (&rr)[3], double rc, double rts,
                                               double rtt, double (&blk)[3][3], double* kc) {
#pragma unroll
  for (int al = 0; al < 3; ++al)
#pragma unroll
    for (int be = 0; be < 3; ++be) blk[al][be] = 0.0;
  if (kc)
    for (int i = 0; i < 5; ++i) kc[i] = 0.0;
  const double r2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
  if (!(r2 < rc * rc)) return;
  const double ir = rsqrt(r2);
  const double r = r2 * ir;
  double flr, dflr;
  cutoff_buf(r, rc, p.r_buf, flr, dflr);
  // f = 1 / (1 + exp(-d (x - 1))), x = r / S~; df/dr = f (1 - f) d / S~ = f (1 - f) d x / r,
  // df/dS~ = -x df/dr
  const double x = r / (p.beta * (rts + rtt));
  const double e = exp(-p.d * (x - 1.0));
  const double f = 1.0 / (1.0 + e);
  const double dfr = f * (1.0 - f) * p.d * x * ir;
  const double C = flr * f;
  const double ir2 = ir * ir;
  const double ir3 = ir2 * ir;
  const double ir5 = ir3 * ir2;
  const double a = 3.0 * C * ir5, b = C * ir3;
  blk[0][0] = a * rr[0] * rr[0] - b;
  blk[1][1] = a * rr[1] * rr[1] - b;
  blk[2][2] = a * rr[2] * rr[2] - b;
  blk[0][1] = blk[1][0] = a * rr[0] * rr[1];
  blk[0][2] = blk[2][0] = a * rr[0] * rr[2];
  blk[1][2] = blk[2][1] = a * rr[1] * rr[2];
  if (kc) {
    const double dfs = -dfr * x;
    const double dC = dflr * f + flr * dfr, CS = flr * dfs;
    const double ir4 = ir2 * ir2, ir6 = ir4 * ir2, ir7 = ir6 * ir;
    kc[0] = 2.0 * (3.0 * dC * ir6 - 15.0 * C * ir7);
    kc[1] = 2.0 * (3.0 * C * ir5 - dC * ir4);
    kc[2] = 12.0 * C * ir5;
    kc[3] = 6.0 * p.beta * CS * ir5;
    kc[4] = -2.0 * p.beta * CS * ir3;
  }
}

// atomicAdd for doubles is native on sm_60+.
__device__ __forceinline__ void atomic_add3(double* p, double a, double b, double c) {
  atomicAdd(p, a);
  atomicAdd(p + 1, b);
  atomicAdd(p + 2, c);
}

// ---------------------------------------------------------------------------------------
// launchers (host)
// ---------------------------------------------------------------------------------------
// Each launcher enqueues its kernels on stream s for central atoms [c0, c1).
void launch_free_atom(const Work& w, const DevParams& p, cudaStream_t s);
void launch_sites_refresh(const Work& w, const DevParams& p, const Grid& g, cudaStream_t s, int* launches);
void launch_skin_check(const Work& w, const double* ref_pos, const int* ref_spec, double half_skin2, int* flag,
                       cudaStream_t s);
void launch_neighbors(const Work& w, const DevParams& p, const Grid& g, cudaStream_t s, int* launches);
void launch_offsets(const Work& w, const DevParams& p, cudaStream_t s);
void launch_scs_count(const Work& w, const DevParams& p, int max_n12, cudaStream_t s);
void launch_scs_fill(const Work& w, const DevParams& p, int c0, int c1, int max_n12, int max_n1, cudaStream_t s);
void launch_pair_radial(const Work& w, const DevParams& p, cudaStream_t s);
void launch_scs_factor(const Work& w, const DevParams& p, const int* order, int c0, int c1, int max_n1, int max_n12,
                       cudaStream_t s);
void launch_scs_adjoint2(const Work& w, const DevParams& p, const int* order, int c0, int c1, int max_n1,
                         int max_n12, cudaStream_t s);
void launch_scs_site_reduce(const Work& w, const DevParams& p, int c0, int c1, cudaStream_t s);
void launch_scs_lu_forward(const Work& w, const DevParams& p, int lu_blocks, int max_n1, int max_n12, int tally,
                           cudaStream_t s);
void launch_scs_lu_adjoint(const Work& w, const DevParams& p, int lu_blocks, int c0, int c1, int max_n1,
                           int max_n12, cudaStream_t s);
size_t scs2_forward_smem(int max_n1, int max_n12);
size_t scs2_adjoint_smem(int max_n1, int max_n12);
void launch_mbd_prepare_sized(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s);
void launch_mbd_chain_sized(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, cudaStream_t s);
void launch_mbd_energy(const Work& w, const DevParams& p, int c0, int c1, cudaStream_t s);
// polynomial-fit coefficients: Lanczos interval of every (centre, frequency), then the fit;
// returns false when the sphere is too large for the kernel (3 max_ns > 1024)
bool launch_log_mode(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s);
// fitted force integrand (Sec. III.D): sample frequencies nu[0..J) (nu_0 = 0), orders M, K of
// theta, and the n_phi-point quadrature of its integral (om, wt = w / 2 pi)
struct ThetaParams {
  int J, M, K, nphi;
  double nu[LMBD_FIT_ROWS];
  double om[LMBD_MAXQ - 1];
  double wt[LMBD_MAXQ - 1];
};
void launch_theta_fit(int n, const double* F, const ThetaParams& tp, double* out, int* status, cudaStream_t s);
bool launch_series_coefficients(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s);
// seeds of the paper's approximate forces (replace the series and pair-matrix adjoint)
void launch_paper_force_seeds(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s);
void launch_mbd_adjoint_sized(const Work& w, const DevParams& p, int c0, int c1, int max_ns,
                              cudaStream_t s, int* launches);
void launch_mbd_adj_series(const Work& w, const DevParams& p, int c0, int c1, cudaStream_t s);
void launch_mbd_adj_pair(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s);
void launch_mbd_adj_blend(const Work& w, const DevParams& p, int c0, int c1, cudaStream_t s);
// block-sparse T_LR (k_sparse.cu): coupled partners of every site (before the offsets), then
// per wave the pattern, blocks and first Krylov block, the float-float chain step and the pair
// adjoint over the coupled pairs only
void launch_sp_count(const Work& w, const DevParams& p, cudaStream_t s);
void launch_sp_prepare(const Work& w, const DevParams& p, int c0, int c1, int max_ns, cudaStream_t s);
void launch_sp_chain(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, cudaStream_t s);
void launch_sp_adj_pair(const Work& w, const DevParams& p, int c0, int c1, int max_pairs, cudaStream_t s);
void launch_forces_out(const Work& w, double* forces, cudaStream_t s);
void launch_slice_t(const Work& w, int c0, int c1, int st, cudaStream_t s);
void launch_chain_oz2(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, int digits, int st,
                      cudaStream_t s);
// W = D v_m digit planes for chain step m (one block per central atom)
void launch_slice_w(const Work& w, const DevParams& p, int m, int c0, int c1, int digits, cudaStream_t s);
// chain step on the fifth-generation tensor cores (tcgen05, TMEM accumulators), digits 5 or 6
// (digits 5 or 6; returns false for another digit count or when a tensor map cannot be encoded)
bool launch_chain_tc(const Work& w, const DevParams& p, int m, int c0, int c1, int max_ns, int digits, int st,
                     cudaStream_t s);
size_t chain_tc_smem(int digits);
// P and Q digit planes (blockIdx.y = 0: P, 1: Q)
void launch_slice_pq(const Work& w, int c0, int c1, int digits, cudaStream_t s);
// adjoint pair matrix and its per-pair contraction on the tcgen05 tensor cores (digits 5 only;
// returns false for another digit count or when a tensor map cannot be encoded)
bool launch_pair_tc(const Work& w, const DevParams& p, int c0, int c1, int max_ns, int digits, cudaStream_t s);
void launch_mbd_adj_pair_oz2(const Work& w, const DevParams& p, int c0, int c1, int max_ns, int digits,
                             cudaStream_t s);

// Raise the dynamic shared-memory limit of a kernel to at least `bytes` (never lowers it: the
// limit is process-wide, and lowering it while another host thread launches the same kernel
// with more shared memory would make that launch fail).
void raise_smem_limit(const void* func, size_t bytes);

// Allocation-free entry point (lmbd_central_polarizabilities_noalloc): scratch lookup and
// the persistent SCS kernel variant, both in k_scs.cu next to the static scratch array.
int noalloc_scratch(void** ptr, size_t* bytes);
void launch_scs_central_noalloc(const Work& w, const DevParams& p, double* bslots, long long slot_doubles,
                                int nslots, int max_n12, int max_n1, cudaStream_t s);
