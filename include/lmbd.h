/* lmbd.h — C ABI of the GB300 (sm_103a) lMBD library.
 *
 * lMBD is the atom-wise, linear-scaling many-body dispersion model of
 * Muhli, Ala-Nissila and Caro, arXiv 2407.06409.  For every atom k ("central
 * atom") the library
 *   1. gathers the sites (atoms and their periodic images) within the cutoffs
 *      (Sec. III.A, sets K; Sec. III.B, sets K1 and K2),
 *   2. builds the short-range dipole tensors T_SR(omega) and solves the local
 *      screening system B_K alpha_K = d_K at omega = 0 and at every quadrature
 *      frequency (Sec. III.B, Eq. local_pol),
 *   3. blends local and central polarisabilities (Eq. full-pol), forms the SCS
 *      radii (Eq. scaled-rvdw) and the long-range tensor T_LR with the cutoff
 *      function f_LR (Sec. III.A),
 *   4. evaluates the local energy E_k as the k-block trace of the truncated
 *      series sum_n c_n G^n, c_n = -1/n, G = sqrt(A) T_LR sqrt(A) (Eq. E_k),
 *      integrated over imaginary frequency by Gauss-Legendre quadrature,
 *   5. optionally returns forces, the exact gradient -d(sum_k w_k E_k)/dR at
 *      fixed Hirshfeld ratios, by a hand-written adjoint of steps 2-4.
 *
 * Units: positions and cell in Angstrom; species parameters in atomic units
 * (alpha0 in bohr^3, C6 in Ha bohr^6, R_vdW in bohr); energies in eV; forces
 * in eV/Angstrom (CODATA 2018 bohr and hartree).
 *
 * Memory: every array argument may be a device pointer or a host pointer; the
 * library asks the CUDA runtime which one it is.  Host arrays are copied to and
 * from the device inside the call (on the given stream, which is then
 * synchronised).  The caller owns every array; the context owns its device
 * workspaces (grown on demand with cudaMalloc) and frees them in lmbd_destroy.
 *
 * Errors: every entry point returns an int status (LMBD_OK = 0); no exception
 * or longjmp crosses the ABI.  After an error the outputs are unspecified and
 * the context stays usable.  A context is not thread-safe: calls on one
 * context must be serialised by the caller.
 */
#ifndef LMBD_H
#define LMBD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LMBD_OK            0
#define LMBD_EINVAL        1  /* bad argument: sizes, NaN input, coincident atoms, bad cutoffs   */
#define LMBD_ENOMEM        2  /* device allocation failed                                         */
#define LMBD_NOT_SPD       3  /* a screening matrix B_K is singular: zero pivot in the LU fallback */
#define LMBD_ECUDA         4  /* a CUDA runtime call failed                                       */
#define LMBD_ECAPACITY     5  /* more sites around one atom than the kernels support             */
#define LMBD_EUNSUPPORTED  6  /* option not supported (e.g. series order out of range)           */
#define LMBD_ESCRATCH      7  /* problem larger than the allocation-free entry point's scratch   */
#define LMBD_EMODEL        8  /* frequency or integrand model not applicable (see below)        */
#define LMBD_ETIMEOUT      9  /* a bounded wait inside a tensor-core kernel ran out; the kernel
                                 drained its own copies, freed its tensor memory and returned   */
#define LMBD_CATASTROPHE  10  /* diagnostic, only with lmbd_set_spectral_check(ctx, 1): the
                                 spectral proxy of G reached 1 for some centre and frequency
                                 (polarisation catastrophe, Sec. III.A); outputs were written  */

#define LMBD_MAX_FREQ      64 /* maximum number of quadrature frequencies                        */
#define LMBD_MAX_ORDER     10 /* maximum series order n_max                                      */

typedef struct lmbd_ctx lmbd_ctx;

/* Free-atom reference data of one species (Sec. II.B, Eq. bar-alpha and after). */
typedef struct {
  double alpha0;   /* static free-atom polarisability alpha^atom, bohr^3     */
  double c6;       /* free-atom C6^atom, Ha bohr^6                            */
  double r0;       /* free-atom vdW radius R_vdW^atom, bohr                   */
} lmbd_species;

/* Model parameters.  Radii in Angstrom.
 *   r_scs     SCS radius: K1 = B(r_SCS), K2 = B(2 r_SCS) \ B(r_SCS)      (Sec. III.B)
 *   r_mbd1    primary MBD radius: couplings of the central atom          (Sec. III.A)
 *   r_mbd2    secondary MBD radius: couplings between other sites        (Sec. III.A)
 *   r_sphere  radius of the local MBD sphere K; <= 0 selects the paper's
 *             r_MBD = r_mbd1 + r_mbd2
 *   r_buf     buffer width r_b of f_SR and f_LR (~0.5 Angstrom)          (Sec. III.A)
 *   r_inner   inner buffer of f_inner (2 Angstrom in the paper)          (Sec. III.B)
 *   beta, d   damping parameters (0.83 and 6)                            (Sec. II.B)
 *   omega_scale  L of the quadrature map omega = L (1 + x) / (1 - x), Ha
 * Requirements: 0 < r_scs <= sphere radius, r_buf > 0, r_inner > 0.           */
typedef struct {
  double r_scs, r_mbd1, r_mbd2, r_sphere, r_buf, r_inner, beta, d, omega_scale;
} lmbd_params;

/* Phases of one call, in launch order (index into the lmbd_stats arrays). */
#define LMBD_PHASE_NEIGHBORS   0  /* free-atom terms, cell list, site lists, offsets          */
#define LMBD_PHASE_SCS         1  /* T_SR assembly + Cholesky + solves, all atoms/frequencies */
#define LMBD_PHASE_PREPARE     2  /* blend, SCS radii, T_LR, first Krylov block               */
#define LMBD_PHASE_CHAIN       3  /* Krylov products v_{m+1} = D T D v_m                       */
#define LMBD_PHASE_ENERGY      4  /* k-block traces and quadrature                            */
#define LMBD_PHASE_ADJ_SERIES  5  /* series adjoint: dL/dalpha~, pair-matrix factors          */
#define LMBD_PHASE_ADJ_PAIR    6  /* pair matrix and dT_LR/dr contraction                     */
#define LMBD_PHASE_ADJ_BLEND   7  /* SCS-radius and blend adjoint                             */
#define LMBD_PHASE_ADJ_SCS     8  /* adjoint SCS solves and dT_SR/dr contraction              */
#define LMBD_PHASE_OUTPUT      9  /* unit conversion and copies of the outputs                */
#define LMBD_NPHASE           10

/* Per-call statistics of the last lmbd_energy_forces call.  flops count the dense
 * linear algebra of each phase from the actual site counts (Cholesky n^3/3, two
 * triangular solves 6 n^2 per frequency, 2 n^2 k per product of an n x n with an
 * n x k matrix); ms are device times from CUDA events on the call's stream and are
 * filled only when profiling is on (lmbd_set_profiling), in batched launch mode. */
typedef struct {
  double flops[LMBD_NPHASE];
  double ms[LMBD_NPHASE];
  int launches[LMBD_NPHASE];
  double bytes_workspace;  /* device workspace in use, bytes                                */
  long long n_sites;       /* total sites over all central atoms (within the list radius)  */
  int max_k1, max_sphere, max_sites; /* largest K1, sphere and site-list capacity           */
  int kernel_launches;     /* kernels launched by the call                                  */
  double bytes_arena;      /* of bytes_workspace: the arena holding the per-wave arrays       */
  int waves_scs;           /* waves of central atoms in the forward SCS stage                 */
  int waves_mbd;           /* waves of central atoms in the MBD stage (energy and adjoint)    */
  int scs_recomputed;      /* 1 when the SCS stage was evaluated again before its adjoint     */
  long long scs_pairs;     /* SCS site pairs over all central atoms (r < r_SCS, K1 x (K1 u K2)) */
  long long scs_adjacency; /* directed K1-K1 pair entries (two per K1-K1 pair)                 */
  double ms_kernel[2];     /* with profiling, one wave: device time of the bucket launches of
                              [0] the SCS factor kernel, [1] the SCS adjoint kernel (all side
                              streams, fork to join; without the pair-list kernels)            */
  long long scs_lu_systems; /* (centre, frequency) screening systems solved by the LU fallback:
                              the FP32 Cholesky met a non-positive pivot (B_K indefinite) or
                              its FP64 refinement did not converge                              */
  int sites_refreshed;     /* 1 if the call refreshed resident site lists (lmbd_set_verlet_skin)
                              instead of building them                                         */
  int reused_forward;      /* 1 if lmbd_forces_kept ran the reverse sweep on the kept forward
                              state instead of a whole call                                    */
  long long spectral_flags; /* (centre, frequency) terms whose spectral proxy reached 1: with
                              M = floor(n_max / 2) >= 2, |G^M e_k|^2 >= |G^(M-1) e_k|^2 (the
                              k-block traces Tr[G^2M]_kk and Tr[G^(2M-2)]_kk); never set when
                              n_max < 4                                                       */
  long long tlr_pairs;     /* site pairs whose T_LR block the call stored: with
                              lmbd_set_sparse_tlr(ctx, 1) the coupled pairs, otherwise every
                              pair of every sphere (sum of ns (ns - 1) / 2)                    */
} lmbd_stats;

/* Fill *out with the defaults r_scs = 5, r_mbd1 = r_mbd2 = r_sphere = 7,
 * r_buf = 0.5, r_inner = 2, beta = 0.83, d = 6, omega_scale = 0.6.          */
int lmbd_default_params(lmbd_params* out);

/* Create a context.  species: n_species entries (host memory, copied).
 * n_freq: quadrature points (1..LMBD_MAX_FREQ); series_order: n_max
 * (2..LMBD_MAX_ORDER).  On success *out receives the context.               */
int lmbd_create(const lmbd_species* species, int n_species, const lmbd_params* params,
                int n_freq, int series_order, lmbd_ctx** out);

/* Per-atom energies and (optionally) forces of one structure.
 *   n_atoms      N >= 0
 *   positions    N x 3 row-major, Angstrom
 *   cell         3 x 3 row-major lattice vectors (rows), Angstrom; NULL = no periodicity
 *   species      N indices into the species table
 *   hirshfeld    N Hirshfeld volume ratios nu_i > 0
 * A species index outside [0, n_species), a non-finite position or a Hirshfeld ratio
 * that is not positive and finite gives LMBD_EINVAL, for host and device arrays alike
 * (device arrays are checked by the first kernel, before any table lookup).
 *   energies     out, N per-atom energies E_k, eV (may be NULL)
 *   forces       out, N x 3, eV/Angstrom, -d(sum_k E_k)/dR; NULL = energies only
 *   stream       cudaStream_t to run on (NULL = legacy default stream)
 * The call is complete (outputs written) when it returns.                   */
int lmbd_energy_forces(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell,
                       const int* species, const double* hirshfeld, double* energies,
                       double* forces, void* stream);

/* As lmbd_energy_forces, but forces = -d(sum_k w_k E_k)/dR for caller weights
 * w (N entries; NULL = all ones).  This is the vector-Jacobian product that
 * a reverse-mode autograd backward needs.                                   */
int lmbd_energy_forces_weighted(lmbd_ctx* ctx, int n_atoms, const double* positions,
                                const double* cell, const int* species,
                                const double* hirshfeld, const double* energy_weights,
                                double* energies, double* forces, void* stream);

/* Energies now, forces later (a reverse-mode autograd: forward, then backward with the upstream
 * gradient as weights).  lmbd_energy_keep computes the energies like lmbd_energy_forces without
 * forces, but lays the workspaces out for forces and keeps the forward state (site lists, SCS
 * factors and solutions, T_LR, Krylov blocks, pair coefficients) on the device.
 * lmbd_forces_kept then gives forces = -d(sum_k w_k E_k)/dR for weights w (NULL = ones) by the
 * reverse sweep alone on that state (the adjoint of Sec. III.D's derivative pieces, exact), when
 * the state is there: the context's last call was lmbd_energy_keep for the same atom count, its
 * state fitted the device as one wave (see lmbd_set_memory_budget), and the positions and species
 * are the same (compared on the device; the cell and Hirshfeld ratios must be the same too: the
 * caller's promise).  Otherwise, or after another call on the context, lmbd_forces_kept makes a
 * whole lmbd_energy_forces_weighted call: the forces are right either way, and
 * lmbd_stats.reused_forward tells which happened.  The kept state serves one reverse sweep.
 * Arguments as lmbd_energy_forces_weighted; energies of lmbd_forces_kept are not written.      */
int lmbd_energy_keep(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell,
                     const int* species, const double* hirshfeld, double* energies, void* stream);
int lmbd_forces_kept(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell,
                     const int* species, const double* hirshfeld, const double* energy_weights,
                     double* forces, void* stream);

/* Launch mode: LMBD_LAUNCH_BATCHED (default) processes all atoms in each
 * kernel launch; LMBD_LAUNCH_PER_ATOM launches every per-atom kernel once per
 * central atom (the plain one-launch-per-atom form, same arithmetic).       */
#define LMBD_LAUNCH_BATCHED  0
#define LMBD_LAUNCH_PER_ATOM 1
int lmbd_set_launch_mode(lmbd_ctx* ctx, int mode);

/* Arithmetic of the two large matrix products (the Krylov chain T_LR W and the adjoint pair
 * matrix P Q^T).  LMBD_PREC_SLICED (default) evaluates them on the bf16 tensor cores from
 * exact 7-bit integer slices of the FP64 operands, recombined in FP64 (6 slices for the
 * products that feed the energies, 5 for those that feed only the forces; truncation error
 * ~S 2^-7S relative to sum |a||b|); LMBD_PREC_FP64 uses FP64 FMA kernels.  Everything
 * else is FP64 (the SCS factorisation is FP32 with FP64 iterative refinement).            */
#define LMBD_PREC_FP64   0
#define LMBD_PREC_SLICED 1
int lmbd_set_precision(lmbd_ctx* ctx, int mode);

/* Tensor-core instruction path of the two sliced products: the Krylov chain T_LR W (Eq. E_k;
 * the matrix-vector products of the series, all frequencies at once) and the adjoint pair
 * matrix P Q^T (the derivative pieces of Sec. III.D).  Same digit slices, same exact integer
 * recombination, so results agree to the last bits (the FP32 accumulation of the
 * lowest-order digit groups may round in another order).
 * LMBD_MMA_TC05 (default): fifth-generation tensor cores, tcgen05.mma issued by one thread
 * per CTA, FP32 accumulators in tensor memory (one per digit order), operands staged in
 * 64-byte swizzled shared memory; 128 x 48 chain tiles, 126 x 96 pair tiles (42 x 32 sites);
 * needs sm_100a/sm_103a.  A device wait that runs out returns LMBD_ETIMEOUT.
 * LMBD_MMA_WARP: warp-level mma.sync, 64 x 48 chain tiles, 48 x 48 pair tiles.
 * Ignored under LMBD_PREC_FP64.
 * Returns LMBD_EINVAL for another value.                                                      */
#define LMBD_MMA_WARP 0
#define LMBD_MMA_TC05 1
int lmbd_set_mma_path(lmbd_ctx* ctx, int path);

/* Bound, in SM clock cycles, of every mbarrier wait in the main loop of the tcgen05 kernels
 * (copies landed, MMAs done, accumulators complete); 0 (default) = 2^32 cycles, about two
 * seconds.  A wait that runs out ends that kernel's tile early: the kernel waits (with the
 * default bound) for its own copies and MMAs in flight, frees its tensor memory and returns,
 * and the call returns LMBD_ETIMEOUT with its outputs undefined; the context stays usable.
 * Small budgets exist to exercise that path.  Returns LMBD_EINVAL for a negative value.     */
int lmbd_set_wait_budget(lmbd_ctx* ctx, long long cycles);

/* Frequency model of the screened polarisabilities.
 * LMBD_FREQ_QUADRATURE (default): the SCS system is solved at omega = 0 and at every
 *   quadrature node.
 * LMBD_FREQ_LORENTZIAN: the paper's Lorentzian model (Sec. III.C, Eqs. alpha_SCS_freq and
 *   char-freq): the SCS system is solved at omega = 0 and omega_ref (Hartree, > 0) only; for
 *   every site the blended polarisability (Eq. full-pol) at the two frequencies defines
 *   omega~_i = omega_ref / sqrt(alpha~(0)/alpha~(omega_ref) - 1), and
 *   alpha~_i(omega) = alpha~_i(0) / (1 + (omega/omega~_i)^2) at the quadrature nodes.  Forces
 *   are the exact gradient of that model.  A call in which some blended polarisability is
 *   larger at omega_ref than at 0 (no real omega~) returns LMBD_EMODEL.  The paper treats
 *   omega_ref as an empirical, element-dependent parameter.
 * lmbd_get_central_polarizabilities then returns N x 2 columns (omega = 0, omega_ref).      */
#define LMBD_FREQ_QUADRATURE 0
#define LMBD_FREQ_LORENTZIAN 1
int lmbd_set_frequency_model(lmbd_ctx* ctx, int model, double omega_ref);

/* Integrand model (Sec. III.C, Eq. integrand and Eq. E_MBD_k).
 * n_fit_nodes = 0 (default): the integrand I(omega) = sum_n c_n Tr{g_k G^(n-2) g_k^T} is
 *   evaluated at every quadrature node and integrated by the quadrature.
 * n_fit_nodes = m, series_order <= m <= LMBD_MAX_FIT_NODES: I is evaluated at omega = 0 and at
 *   m fit nodes omega_j = L (1 + x_j) / (1 - x_j), x_j the m-point Gauss-Legendre nodes and
 *   L = omega_scale (so at n_max + 1 frequencies at least, as the paper asks).  For every
 *   centre, phi(omega) = a / (1 + sum_{n=1}^{n_max} b_n omega^(2n)) is fitted with a, b_n >= 0
 *   to the linearised equations a I(0) - sum_n b_n omega_j^(2n) I(omega_j) = I(omega_j) by
 *   non-negative least squares (Lawson-Hanson active set, chosen on unit-norm columns), and
 *   E_k = I(0) (1/2pi) sum_i w_i phi(omega_i) with the n_freq-point quadrature.  Forces are the
 *   exact gradient of that E_k (the active set is locally constant).  Combines with either
 *   frequency model.  A call in which some centre's fit has a > 0 and every b_n = 0 (phi not
 *   integrable) returns LMBD_EMODEL.  m outside the range returns LMBD_EINVAL. */
#define LMBD_MAX_FIT_NODES 24
int lmbd_set_integrand_fit(lmbd_ctx* ctx, int n_fit_nodes);

/* Series coefficients (Sec. III.A, Eqs. diagonal_appr, eigendecomp and polynomial-fit).
 * lanczos_steps = 0 (default): c_n = -1/n, the Taylor coefficients of ln(1 - lambda).
 * lanczos_steps = m (1..LMBD_MAX_LANCZOS): for every central atom and every frequency of the
 *   integrand, the spectral interval [lambda_min, lambda_max] of the symmetric G = D T_LR D is
 *   estimated by the extreme Ritz values of min(m, 3 n_sphere) Lanczos steps (three-term
 *   recurrence without reorthogonalisation, FP64, start vector u_i = SplitMix64 output i mapped
 *   to [-1, 1) and normalised), and c_1..c_n_max minimise the L2 distance between
 *   sum_n c_n lambda^n and ln(1 - lambda) on that interval (64-point Gauss-Legendre quadrature);
 *   these c_n replace -1/n in the energy.  Forces hold the c_n fixed, as the force expressions of
 *   Sec. III.D do, so they are not the gradient of the c_n's own position dependence.  A call in
 *   which some interval reaches lambda = 1 (ln(1 - lambda) undefined, a polarisation
 *   catastrophe) returns LMBD_EMODEL; one whose sphere exceeds 341 sites returns
 *   LMBD_ECAPACITY in this mode.  Returns LMBD_EINVAL for m outside 0..LMBD_MAX_LANCZOS. */
#define LMBD_MAX_LANCZOS 64
int lmbd_set_series_fit(lmbd_ctx* ctx, int lanczos_steps);

/* Resident site lists for trajectories (MD frames of one structure).  skin (Angstrom) > 0: the
 * site lists hold every atom image within the list radius max(2 r_SCS, sphere) + skin of the
 * frame they were built for, and stay on the device with that frame's positions.  A later call
 * with the same atom count, cell and species whose atoms have all moved by less than skin / 2
 * (positions as given, not wrapped) refreshes them instead of searching again: each stored
 * candidate's displacement is recomputed from the new positions, and the candidates are sorted
 * and counted again.  The sites within the list radius, their order and their bits are those of a
 * fresh search, so results are those of a call without a skin (the Verlet-list argument: an atom
 * now within the radius was within radius + skin).  Any other call searches again and becomes
 * the new reference.  lmbd_stats.sites_refreshed tells which happened.  skin = 0 (default)
 * turns it off.  The skin widens the lists (and their memory) by ((r + skin) / r)^3.  Returns
 * LMBD_EINVAL for a negative or non-finite skin.                                             */
int lmbd_set_verlet_skin(lmbd_ctx* ctx, double skin);

/* Log mode (Sec. III.A, Eq. series-expansion: the n_max -> infinity limit of the series, the
 * k-block trace of ln(1 - G) that the truncated series and the polynomial fit approximate).
 * lanczos_steps = 0 (default): the truncated series.  lanczos_steps = m (1..LMBD_MAX_LANCZOS):
 * for every central atom, frequency of the integrand and direction alpha of the centre's
 * three rows, m steps of the Lanczos recurrence on G = D T_LR D (FP64, no reorthogonalisation)
 * from the unit vector e_alpha give a tridiagonal J; its eigenvalues theta_i and the first
 * components z_i of its eigenvectors (implicit QL) form the Gauss rule
 * e_alpha^T ln(1 - G) e_alpha ~ sum_i z_i^2 ln(1 - theta_i), exact once the Krylov space is
 * exhausted (the recurrence stops when beta falls below 1e-13 of the largest coefficient) and
 * converging geometrically in m otherwise; the three directions sum to [ln(1 - G)]_kk, which
 * replaces the series in the integrand (quadrature or fitted integrand, either frequency
 * model).  Energies only: a call with forces returns LMBD_EUNSUPPORTED; combined with
 * lmbd_set_series_fit it returns LMBD_EINVAL; a sphere beyond 341 sites returns
 * LMBD_ECAPACITY.  An eigenvalue theta >= 1 (polarisation catastrophe) gives a NaN energy.
 * Returns LMBD_EINVAL for m outside 0..LMBD_MAX_LANCZOS.                                    */
int lmbd_set_log_mode(lmbd_ctx* ctx, int lanczos_steps);

/* Spectral check (Sec. III.A: the truncated series and ln(1 - G) need the eigenvalues of
 * G = sqrt(A) T_LR sqrt(A) inside (-1, 1); beyond, the polarisation catastrophe).  Every call
 * counts the (centre, frequency) terms whose proxy |G^M e_k|^2 / |G^(M-1) e_k|^2 (M =
 * floor(n_max / 2) >= 2) reaches 1 in lmbd_stats.spectral_flags.  fail = 0 (default): the call
 * returns LMBD_OK regardless; fail = 1: it returns LMBD_CATASTROPHE when the count is not zero
 * (outputs still written).  Returns LMBD_EINVAL for another value.                          */
int lmbd_set_spectral_check(lmbd_ctx* ctx, int fail);

/* Block-sparse T_LR (Sec. III.A, Fig. sparsity: the central row and column of T_LR,K couple
 * the sites within r_MBD,1 of the central atom, every other pair only the sites within r_MBD,2
 * of each other, so with r_MBD,2 < r_MBD,1 most blocks of a large sphere are zero).
 * on = 0 (default): T_LR,K is stored dense per central atom (3 ns x 3 ns) and the Krylov chain
 *   and the adjoint pair products run over all blocks (lmbd_set_precision selects their
 *   arithmetic).
 * on = 1: per central atom only the coupled site pairs are stored (found by an FP32 distance
 *   test with a relative slack of 2e-4 on rc^2; a listed pair whose FP64 distance is not below
 *   its cutoff has a zero block, as on the dense path), and the chain steps
 *   v_{m+1} = D T_LR D v_m and the pair products M_st = P_s Q_t^T run over those pairs alone,
 *   in float-float arithmetic (pairs of FP32 numbers, about 2^-46 relative per product) with
 *   FP64 results; lmbd_set_precision does not apply to them.  Spheres up to 4096 sites
 *   (LMBD_ECAPACITY beyond).  Serves the series energy and the exact forces: a call with log
 *   mode, polynomial-fit coefficients or the paper's force model returns LMBD_EUNSUPPORTED.
 *   lmbd_stats.tlr_pairs counts the stored pairs.
 * Returns LMBD_EINVAL for another value of on.                                               */
int lmbd_set_sparse_tlr(lmbd_ctx* ctx, int on);

/* Force model (Sec. III.D).
 * LMBD_FORCES_EXACT (default): forces = -d(sum_k w_k E_k)/dR, the exact gradient of the
 *   returned energies at fixed Hirshfeld ratios.
 * LMBD_FORCES_PAPER: the paper's approximate forces, F_k = -dE^{k,tot}/dr_k of the total
 *   energy of atom k's own sphere (Eq. E_k_tot, full traces, every image of k in the sphere
 *   moving with it), with the central polarisabilities held fixed (Eq. full-pol-grad), the full
 *   derivative in the n = 2 term and, for n >= 3, the derivative of G kept only in the row and
 *   column of the central atom (Eq. cent-appr).  The frequency integral is the quadrature; with
 *   lmbd_set_integrand_fit(m) it is the paper's fitted force integrand instead: the force
 *   integrand F(nu_j) of every atom and component at omega = 0 and the m fit nodes (one pass of
 *   the reverse sweep per sample, so m + 1 passes), the fit theta(omega) =
 *   sum_{i<=M} u_i (-omega)^i / (1 + sum_{l<=K} v_l omega^(2l)), u, v >= 0, M = K = min(m/2, 5),
 *   to the ratios F(nu_j) / F(0) by non-negative least squares (a fit whose numerator does not
 *   grow two orders slower than its denominator is repeated with M lowered by one, until theta
 *   decays at least as omega^-2), and F = F(0) times the integral of theta / (2 pi) by the n_freq-point
 *   quadrature (LMBD_EMODEL if no fitted theta of some component is integrable).  Energies are unchanged; with per-atom weights (lmbd_energy_forces_weighted)
 *   E^{k,tot} is multiplied by w_k. */
#define LMBD_FORCES_EXACT 0
#define LMBD_FORCES_PAPER 1
int lmbd_set_force_model(lmbd_ctx* ctx, int model);

/* Autotuner of the SCS launch shapes.  The local SCS systems are launched in buckets of
 * central atoms whose |K1| lies within a width w (shared memory, and with it the blocks per
 * SM, is sized for the largest system of a bucket; narrow buckets waste less shared memory,
 * wide ones launch less often).  lmbd_autotune runs the given structure (the arguments of
 * lmbd_energy_forces; forces may be NULL) twice for each w in {2, 3, 4, 6, 8, 12, 16}, times the
 * SCS and SCS-adjoint phases with CUDA events on the stream, keeps the fastest w in the
 * context for later calls and returns it in *bucket_width (if not NULL).  Results do not depend
 * on w.  The outputs hold the last call's values.  Batched launch mode only (LMBD_EINVAL
 * otherwise).  Default w = 6. */
int lmbd_autotune(lmbd_ctx* ctx, int n_atoms, const double* positions, const double* cell, const int* species,
                  const double* hirshfeld_ratios, double* energies, double* forces, void* cuda_stream,
                  int* bucket_width);

/* Device memory budget of the context in bytes (0 = the default: the device's free
 * memory at each call less 1 GiB).  Central atoms are processed in contiguous waves whose
 * per-centre arrays fit the budget: the SCS stage of every centre first (its central
 * polarisabilities feed every sphere that contains the atom), then the MBD energy and its
 * adjoint wave by wave, then the SCS adjoint wave by wave.  When the SCS arrays of all
 * centres do not fit beside one MBD wave, each SCS adjoint wave first evaluates its SCS
 * stage again (same arithmetic, same results).  Results do not depend on the waves up to
 * the order of floating-point atomic additions in the forces.  A budget too small for one
 * central atom gives LMBD_ENOMEM.                                                          */
int lmbd_set_memory_budget(lmbd_ctx* ctx, size_t bytes);

/* Free every device workspace of the context except its species table (the next call
 * allocates again); results of the last call are no longer available.  For a server that
 * must return memory held by an idle context.                                          */
int lmbd_release_workspace(lmbd_ctx* ctx);

/* Device bytes the context holds now (*out, host). */
int lmbd_held_bytes(const lmbd_ctx* ctx, size_t* out);

/* Per-phase device timing with CUDA events (0 = off, the default; reported only when
 * every stage ran as a single wave). */
int lmbd_set_profiling(lmbd_ctx* ctx, int on);

/* Central polarisabilities alpha_I,k(omega) of the last call (Sec. III.B):
 * N x (n_freq + 1) row-major; column 0 is omega = 0, then the quadrature
 * nodes in increasing order (N x 2: omega = 0, omega_ref with the Lorentzian
 * frequency model).  out: device or host.                                   */
int lmbd_get_central_polarizabilities(lmbd_ctx* ctx, double* out, void* stream);

/* Site counts of the last call, N x 4 int32 row-major:
 * |K1| (r < r_SCS, includes the atom), |sphere| (r < sphere radius),
 * |K1 u K2| (r < 2 r_SCS), all sites within max(2 r_SCS, sphere radius).   */
int lmbd_get_site_counts(lmbd_ctx* ctx, int* out, void* stream);

/* Quadrature nodes (Ha) and weights of the context; host arrays of n_freq. */
int lmbd_get_quadrature(const lmbd_ctx* ctx, double* omega, double* weight);

/* Statistics of the last call (host struct). */
int lmbd_get_stats(const lmbd_ctx* ctx, lmbd_stats* out);

/* Destroy the context and free its device memory.  NULL is accepted. */
int lmbd_destroy(lmbd_ctx* ctx);

/* Allocation-free central polarisabilities.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory — plug-ins of an MD engine that owns the device memory pool,
 * and embedded runtimes that forbid allocation after start-up.  It computes the same central
 * polarisabilities alpha_I,k(omega) as lmbd_energy_forces (site search and one local
 * SCS solve per atom and frequency, Sec. III.B), without a context and without
 * calling cudaMalloc, cudaFree or any allocating routine: every scratch buffer is
 * carved from one fixed array of LMBD_NOALLOC_SCRATCH_BYTES that is part of the
 * library image, so every GPU that loads the library holds it until the process exits.
 *   species_params/n_species  as lmbd_create (host, n_species <= 64)
 *   params, n_freq            as lmbd_create
 *   n_atoms ... hirshfeld     as lmbd_energy_forces (device or host pointers)
 *   alpha_central             out, n_atoms x (n_freq + 1), column 0 is omega = 0
 *   stream                    cudaStream_t (NULL = legacy default stream); the call
 *                             synchronises it before returning
 * Limits: n_atoms <= LMBD_NOALLOC_MAX_ATOMS, at most LMBD_NOALLOC_SITE_CAP sites within
 * max(2 r_SCS, sphere radius) of any atom, at most LMBD_NOALLOC_MAX_K1 sites within
 * r_SCS; larger problems return LMBD_ESCRATCH before any device work on them.
 * The call reads the site counts back to the host before the solves, so it cannot run
 * on a stream that is being captured into a CUDA graph: such a stream gets
 * LMBD_EUNSUPPORTED before anything is issued on it.  Device-resident species indices
 * outside [0, n_species), non-finite positions and non-positive Hirshfeld ratios give
 * LMBD_EINVAL (host arrays are checked before any copy).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls
 * share the one array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU (other streams or threads) race on it and must be serialised. */
#define LMBD_NOALLOC_SCRATCH_BYTES (32u << 20)
#define LMBD_NOALLOC_MAX_ATOMS     256
#define LMBD_NOALLOC_SITE_CAP      512
#define LMBD_NOALLOC_MAX_K1        64
int lmbd_central_polarizabilities_noalloc(const lmbd_species* species_params, int n_species,
                                          const lmbd_params* params, int n_freq, int n_atoms,
                                          const double* positions, const double* cell,
                                          const int* species, const double* hirshfeld,
                                          double* alpha_central, void* stream);

/* Static, human-readable text for a status code. */
const char* lmbd_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* LMBD_H */
