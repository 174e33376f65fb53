"""Plain CPU oracle for the lMBD local-cluster problem (arXiv 2407.06409).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or runs
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` do.  It shares no code with the CUDA path.

Everything is float64 PyTorch on the CPU and follows the paper's equations in
the paper's order, one atom (one "central atom k") at a time:

* free-atom polarisability, characteristic frequency, Gaussian width and
  vdW radius (Sec. II.B, Eq. bar-alpha and the definitions after Eq. h-func);
* the short-range dipole tensor T_SR = (1 - f) d_i d_j [erf(r/sigma)/r]
  written as -T g + h (Eq. T_SR, Eqs. g-func / h-func) with the cutoff
  functions f_SR and f_inner (Sec. III.B);
* the local SCS system B_K alpha_K = d_K over the coupled set K1 = B(r_SCS)
  with the uncoupled shell K2 = B(2 r_SCS) minus B(r_SCS) (Eq. local_pol),
  solved with a library dense solve;
* central polarisabilities alpha_I (each atom in its own sphere) and the
  range-separated blend with f_SCS (Eq. full-pol);
* SCS radii (Eq. scaled-rvdw), T_LR with f_LR and the primary/secondary radii
  (Sec. III.A), G = sqrt(A) T_LR sqrt(A) (Eq. G_frequency);
* the local energy as the truncated series Tr{g_k G^(n-2) g_k^T} with
  c_n = -1/n (Eq. mbd-local / Eq. E_k) or, in "log mode", the k-block of
  ln(1 - G) from a symmetric eigendecomposition (Eq. series-expansion);
* the frequency integral by Gauss-Legendre quadrature mapped to [0, inf);
* optionally (omega_ref set) the Lorentzian frequency model of Sec. III.C: SCS solves at
  omega = 0 and omega_ref only, alpha~(omega) at the nodes from Eqs. char-freq and
  alpha_SCS_freq applied to the blended polarisabilities;
* optionally (fit_nodes set) the fitted integrand of Sec. III.C: the integrand I(omega) of
  Eq. integrand at omega = 0 and a few fit nodes, the rational phi(omega) = a / (1 + sum_n
  b_n omega^(2n)) with a, b_n >= 0 from non-negative least squares (Lawson-Hanson active set)
  on the linearised equations, and E_k = I(0) times the integral of phi (Eq. E_MBD_k);
* optionally (lanczos_steps set) the polynomial-fit coefficients of Sec. III.A: per centre and
  frequency, lambda_min and lambda_max of G from m Lanczos steps (Ritz values of the tridiagonal
  matrix), c_n from the least-squares fit of ln(1 - lambda) by sum_{n=1}^{n_max} c_n lambda^n on
  [lambda_min, lambda_max] (Eq. diagonal_appr), used in place of -1/n (Eq. polynomial-fit) and
  held fixed in the forces.

The paper's approximate forces (Sec. III.D) are a separate driver, ``System.paper_forces``:
F_k = -dE^{k,tot}/dr_k of the total energy of atom k's own sphere (Eq. E_k_tot, full trace)
with dalpha_I/dr = 0 (Eq. full-pol-grad), the full dG/dr_k in the n = 2 term and, for n >= 3,
dG/dr_k kept only in the row and column of the central atom (Eqs. mbd-forces, cent-appr).

Forces are -d(sum_k w_k E_k)/dR by PyTorch autograd (reverse mode), applied to
the two phases separately so that memory stays bounded: first E_k with the
other atoms' central polarisabilities as leaves, then those central
polarisabilities with the accumulated seeds (exact chain rule).

Readings where the paper is silent or inconsistent (the design notes list
them): energy sign per Eq. E_MBD (c_n = -1/n, dispersion energy negative);
MBD sphere radius r_sphere (default r_MBD,1 + r_MBD,2); every periodic image
within a radius is a distinct site; set membership by strict r < r_c with r
measured in Angstrom from the central atom; Gauss-Legendre nodes mapped by
omega = L (1 + x)/(1 - x); positions in Angstrom, species parameters in
atomic units, outputs in eV and eV/Angstrom with CODATA 2018 constants.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np
import torch

BOHR_ANGSTROM = 0.529177210903       # CODATA 2018
HARTREE_EV = 27.211386245988         # CODATA 2018
_DT = torch.float64


@dataclass(frozen=True)
class Params:
    """Cutoffs in Angstrom; beta and d from Sec. II.B (beta = 0.83, d = 6)."""
    r_scs: float = 5.0
    r_mbd1: float = 7.0
    r_mbd2: float = 7.0
    r_sphere: float = 7.0          # <= 0 means r_mbd1 + r_mbd2 (the paper's B_{r_MBD})
    r_buf: float = 0.5             # buffer width r_b of f_SR and f_LR (Sec. III.A)
    r_inner: float = 2.0           # r_inner of f_inner (Sec. III.B: hard-coded 2 Angstrom)
    beta: float = 0.83
    d: float = 6.0
    n_freq: int = 12
    series_order: int | None = 6   # None = log mode (the n_max -> infinity limit)
    omega_scale: float = 0.6       # L of the frequency mapping, Hartree
    # None: SCS solved at omega = 0 and at every quadrature node.  A value (Hartree): the
    # Lorentzian model of Sec. III.C -- SCS at omega = 0 and omega_ref only, then
    # alpha~_i(omega) = alpha~_i(0) / (1 + (omega / omega~_i)^2) (Eq. alpha_SCS_freq) with
    # omega~_i from the two solves (Eq. char-freq)
    omega_ref: float | None = None
    # None: the integrand is evaluated at every quadrature node.  m > 0: the fitted integrand
    # of Sec. III.C -- I(omega) at omega = 0 and m fit nodes (m >= series_order, so at least
    # n_max + 1 values), phi fitted by NNLS, E_k = I(0) * integral of phi, the integral by the
    # n_freq-point quadrature
    fit_nodes: int | None = None
    # None: c_n = -1/n.  m > 0: c_n per centre and frequency from the polynomial fit of
    # ln(1 - lambda) on the Lanczos estimate (m steps) of G's spectral interval (Sec. III.A);
    # forces hold the c_n fixed, as the force expressions of Sec. III.D do
    lanczos_steps: int | None = None

    @property
    def sphere(self) -> float:
        return self.r_sphere if self.r_sphere > 0 else self.r_mbd1 + self.r_mbd2

    @property
    def r_list(self) -> float:
        return max(2.0 * self.r_scs, self.sphere)


# ----------------------------------------------------------------------------------------
# frequency grid (Eq. E_MBD integral over imaginary frequency)
# ----------------------------------------------------------------------------------------
def quadrature(n_freq: int, omega_scale: float) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre nodes on [-1, 1] mapped to [0, inf): omega = L(1+x)/(1-x)."""
    x, w = np.polynomial.legendre.leggauss(n_freq)
    omega = omega_scale * (1.0 + x) / (1.0 - x)
    weight = 2.0 * omega_scale * w / (1.0 - x) ** 2
    return omega, weight


def fit_node_frequencies(m: int, omega_scale: float) -> np.ndarray:
    """Frequencies at which the fitted integrand is sampled: omega = 0, then the m-point
    Gauss-Legendre nodes under the same mapping as the quadrature (the paper leaves the
    sample frequencies open)."""
    x, _ = np.polynomial.legendre.leggauss(m)
    return np.concatenate([[0.0], omega_scale * (1.0 + x) / (1.0 - x)])


def frequencies(p: Params) -> tuple[torch.Tensor, torch.Tensor]:
    """Column 0 is omega = 0 (needed for the SCS radii), then the nodes at which the
    integrand is evaluated: the quadrature nodes with their weights, or with fit_nodes set the
    fit frequencies (weights unused, zero)."""
    if p.fit_nodes:
        nodes = fit_node_frequencies(p.fit_nodes, p.omega_scale)
        omega = torch.tensor(np.concatenate([[0.0], nodes]), dtype=_DT)
        return omega, torch.zeros_like(omega)
    om, w = quadrature(p.n_freq, p.omega_scale)
    omega = torch.tensor(np.concatenate([[0.0], om]), dtype=_DT)
    weight = torch.tensor(np.concatenate([[0.0], w]), dtype=_DT)
    return omega, weight


def scs_frequencies(p: Params) -> torch.Tensor:
    """Frequencies of the SCS solves: every column of `frequencies`, or 0 and omega_ref."""
    if p.omega_ref is None:
        return frequencies(p)[0]
    return torch.tensor([0.0, p.omega_ref], dtype=_DT)


def lorentzian(alpha0, alpha_ref, omega_ref, omega):
    """Sec. III.C: omega~ = omega_ref / sqrt(alpha~(0)/alpha~(omega_ref) - 1) (Eq. char-freq),
    alpha~(omega) = alpha~(0) / (1 + (omega/omega~)^2) (Eq. alpha_SCS_freq).

    alpha0, alpha_ref: (n,); omega: (Q,).  Returns (n, Q).
    """
    omega_t = omega_ref / torch.sqrt(alpha0 / alpha_ref - 1.0)
    return alpha0[:, None] / (1.0 + (omega[None, :] / omega_t[:, None]) ** 2)


# ----------------------------------------------------------------------------------------
# fitted integrand (Sec. III.C, Eq. integrand and the phi(omega) fit, Eq. E_MBD_k)
# ----------------------------------------------------------------------------------------
def nnls_passive(A: np.ndarray, y: np.ndarray) -> tuple[list[int], np.ndarray]:
    """Non-negative least squares min |A x - y|, x >= 0, by the Lawson-Hanson active-set
    method (Lawson and Hanson, Solving Least Squares Problems, 1974, ch. 23), the method the
    paper names for its fits.

    A has unit-norm columns (the caller scales them).  Returns the passive set (sorted column
    indices with x > 0) and x.  Tolerance: a column enters only if its gradient component
    exceeds 1e-13 |y|; at most 3 C outer steps.
    """
    R, C = A.shape
    x = np.zeros(C)
    passive = np.zeros(C, dtype=bool)
    ny = float(np.sqrt((y * y).sum()))
    if ny == 0.0:
        return [], x
    tol = 1e-13 * ny
    for _ in range(3 * C):
        grad = A.T @ (y - A @ x)
        cand = [c for c in range(C) if not passive[c]]
        if not cand:
            break
        t = max(cand, key=lambda c: (grad[c], -c))
        if grad[t] <= tol:
            break
        passive[t] = True
        while True:
            idx = np.nonzero(passive)[0]
            z = np.zeros(C)
            z[idx] = np.linalg.lstsq(A[:, idx], y, rcond=None)[0]
            if np.all(z[idx] > 0.0):
                x = z
                break
            # step from x towards z until the first passive component reaches zero
            neg = [c for c in idx if z[c] <= 0.0]
            steps = [x[c] / (x[c] - z[c]) for c in neg]
            j = int(np.argmin(steps))
            x = x + steps[j] * (z - x)
            x[neg[j]] = 0.0
            for c in idx:
                if x[c] <= 0.0:
                    x[c] = 0.0
                    passive[c] = False
            if not passive.any():
                break
    return [int(c) for c in np.nonzero(passive)[0]], x


def phi_fit(I: torch.Tensor, nodes: np.ndarray, order: int) -> tuple[torch.Tensor, torch.Tensor]:
    """Coefficients of phi(omega) = a / (1 + sum_{n=1}^{order} b_n omega^(2n)) with a, b >= 0.

    I: integrand values at `nodes` (nodes[0] = 0).  The fit of Sec. III.C, I(omega) ~ phi(omega)
    I(0), is made linear by multiplying out the denominator: for every node
    a I(0) - sum_n b_n omega^(2n) I(omega) = I(omega), solved in the least-squares sense under
    a, b >= 0.  The active set is chosen on unit-norm columns; the returned coefficients are
    the plain least-squares solution on that set (differentiable through I).
    """
    J = I.shape[0]
    nu = torch.as_tensor(nodes, dtype=_DT)
    cols = [I[0] * torch.ones(J, dtype=_DT)] + [-(nu ** (2 * n)) * I for n in range(1, order + 1)]
    A = torch.stack(cols, dim=1)
    An = A.detach().numpy()
    sc = np.sqrt((An * An).sum(0))
    sc[sc == 0.0] = 1.0
    passive, _ = nnls_passive(An / sc, I.detach().numpy())
    x = torch.zeros(order + 1, dtype=_DT)
    if passive:
        sP = torch.as_tensor(sc[passive], dtype=_DT)
        Q, R = torch.linalg.qr(A[:, passive] / sP)
        zP = torch.linalg.solve_triangular(R, (Q.T @ I)[:, None], upper=True)[:, 0]
        x = x.index_put((torch.tensor(passive),), zP / sP)
    a, b = x[0], x[1:]
    if float(a.detach()) > 0.0 and not bool((b.detach() > 0).any()):
        raise ValueError("fitted integrand has no decaying term: phi is not integrable")
    return a, b


def phi_integral(a, b, omega: np.ndarray, weight: np.ndarray) -> torch.Tensor:
    """Integral over [0, inf) of phi(omega) / (2 pi) by the given quadrature."""
    om = torch.as_tensor(omega, dtype=_DT)
    den = torch.ones_like(om)
    for n in range(1, b.shape[0] + 1):
        den = den + b[n - 1] * om ** (2 * n)
    return (torch.as_tensor(weight, dtype=_DT) * a / den).sum() / (2.0 * math.pi)


def theta_orders(m: int) -> tuple[int, int]:
    """Orders (M, K) of the force-integrand fit from m fit nodes: M = K = min(floor(m/2), 5),
    so that the M + K + 1 coefficients need at most the m + 1 samples (omega = 0 and the nodes)."""
    k = min(m // 2, 5)
    return k, k


def theta_fit(R: np.ndarray, nodes: np.ndarray, M: int, K: int) -> tuple[np.ndarray, np.ndarray]:
    """Coefficients of the force-integrand fit of Sec. III.D,
    theta(omega) = sum_{j=0}^{M} u_j (-omega)^j / (1 + sum_{l=1}^{K} v_l omega^(2l)), u, v >= 0
    (the paper prints the exponent of the denominator as 2n; read as 2l), fitted to the ratios
    R_i = F(nu_i) / F(0) of the force integrand at the sample frequencies nu_i (nu_0 = 0): the
    denominator is multiplied out, sum_j u_j (-nu_i)^j - R_i sum_l v_l nu_i^(2l) = R_i, and the
    system is solved by non-negative least squares (Lawson-Hanson on unit-norm columns, as for
    phi); the coefficients are the plain least-squares solution on the final passive set.  The
    integral over [0, inf) needs the numerator to grow two orders slower than the denominator:
    when the fitted theta does not (the NNLS may leave the highest v at zero), the numerator
    order M is lowered by one and the fit repeated (a reading; the paper leaves M and K open).
    Returns (u, v) with len(u) = M + 1 of the original M (trailing zeros if lowered)."""
    nu = np.asarray(nodes, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    for Mc in range(M, -1, -1):
        cols = [(-nu) ** j for j in range(Mc + 1)] + [-R * nu ** (2 * l) for l in range(1, K + 1)]
        A = np.stack(cols, axis=1)
        sc = np.sqrt((A * A).sum(0))
        sc[sc == 0.0] = 1.0
        passive, _ = nnls_passive(A / sc, R)
        x = np.zeros(Mc + 1 + K)
        if passive:
            x[passive] = np.linalg.lstsq(A[:, passive] / sc[passive], R, rcond=None)[0] / sc[passive]
        u, v = x[:Mc + 1], x[Mc + 1:]
        ju = max([j for j in range(Mc + 1) if u[j] > 0.0], default=-1)
        lv = max([l for l in range(1, K + 1) if v[l - 1] > 0.0], default=0)
        if ju < 0 or 2 * lv >= ju + 2:
            return np.concatenate([u, np.zeros(M - Mc)]), v
    raise ValueError("fitted force integrand is not integrable")


def theta_integral(u, v, omega: np.ndarray, weight: np.ndarray) -> float:
    """Integral over [0, inf) of theta(omega) / (2 pi) by the given quadrature."""
    om = np.asarray(omega, dtype=np.float64)
    num = sum(u[j] * (-om) ** j for j in range(len(u)))
    den = 1.0 + sum(v[l - 1] * om ** (2 * l) for l in range(1, len(v) + 1))
    return float((np.asarray(weight) * num / den).sum() / (2.0 * math.pi))


# ----------------------------------------------------------------------------------------
# polynomial-fit series coefficients (Sec. III.A, Eqs. diagonal_appr, eigendecomp,
# polynomial-fit)
# ----------------------------------------------------------------------------------------
def splitmix64_unit(count: int) -> np.ndarray:
    """Start vector of the Lanczos iteration: entries in [-1, 1) from the SplitMix64 generator
    (Steele, Lea and Flood 2014; Vigna's reference constants), counter 0, 1, 2, ..."""
    out = np.empty(count)
    m64 = (1 << 64) - 1
    for i in range(count):
        z = ((i + 1) * 0x9E3779B97F4A7C15) & m64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m64
        z ^= z >> 31
        out[i] = (z >> 11) * 2.0 ** -52 - 1.0
    return out


def lanczos_interval(G: np.ndarray, steps: int) -> tuple[float, float]:
    """Smallest and largest Ritz value after min(steps, dim) Lanczos steps on the symmetric G
    (Lanczos 1950; three-term recurrence, no reorthogonalisation), started from the SplitMix64
    vector.  An exhausted Krylov space (beta = 0) ends the iteration early."""
    n = G.shape[0]
    m = min(steps, n)
    v = splitmix64_unit(n)
    v = v / np.sqrt(v @ v)
    v_prev = np.zeros(n)
    beta = 0.0
    alphas, betas = [], []
    for j in range(m):
        w = G @ v
        a = float(v @ w)
        w = w - a * v - beta * v_prev
        alphas.append(a)
        b = float(np.sqrt(w @ w))
        if j == m - 1 or b == 0.0:
            break
        betas.append(b)
        v_prev, v, beta = v, w / b, b
    Tm = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
    ev = np.linalg.eigvalsh(Tm)
    return float(ev[0]), float(ev[-1])


def log_fit_coefficients(lo: float, hi: float, order: int, target=None) -> np.ndarray:
    """c_1..c_order of the least-squares polynomial sum_n c_n lambda^n (no constant term, since
    ln(1 - 0) = 0) closest to target(lambda) = ln(1 - lambda) in L2 on [lo, hi], the integral
    taken by 64-point Gauss-Legendre quadrature.  Returns c_0..c_order (c_0 = 0).  A degenerate
    interval gives the Taylor coefficients -1/n."""
    c = np.zeros(order + 1)
    if not hi - lo > 1e-12:
        c[1:] = [-1.0 / n for n in range(1, order + 1)]
        return c
    if target is None:
        if hi >= 1.0:
            raise ValueError("spectral interval reaches 1: ln(1 - lambda) is not defined")
        target = lambda lam: np.log1p(-lam)
    x, w = np.polynomial.legendre.leggauss(64)
    lam = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
    sw = np.sqrt(0.5 * (hi - lo) * w)
    rho = max(abs(lo), abs(hi))                   # columns in lambda / rho for conditioning
    V = np.stack([(lam / rho) ** n for n in range(1, order + 1)], axis=1) * sw[:, None]
    d = np.linalg.lstsq(V, target(lam) * sw, rcond=None)[0]
    c[1:] = d / rho ** np.arange(1, order + 1)
    return c


# ----------------------------------------------------------------------------------------
# free-atom quantities (Sec. II.B)
# ----------------------------------------------------------------------------------------
def free_atom(species, nu, table, omega):
    """alpha_bar_i(omega) (Eq. bar-alpha), sigma_i(omega), R_vdW,i.

    omega_i = 4 C6 / (3 alpha0^2); alpha_bar = alpha0 nu / (1 + (omega/omega_i)^2);
    sigma_i = (sqrt(2/pi) alpha_bar / 3)^(1/3); R_vdW,i = R0 nu^(1/3).
    """
    tab = torch.as_tensor(table, dtype=_DT)
    sp = torch.as_tensor(np.asarray(species), dtype=torch.long)
    nu = torch.as_tensor(nu, dtype=_DT)
    a0, c6, r0 = tab[sp, 0], tab[sp, 1], tab[sp, 2]
    om_i = 4.0 * c6 / (3.0 * a0 * a0)
    alpha_bar = (a0 * nu)[:, None] / (1.0 + (omega[None, :] / om_i[:, None]) ** 2)
    sigma = (math.sqrt(2.0 / math.pi) * alpha_bar / 3.0) ** (1.0 / 3.0)
    r_vdw = r0 * nu ** (1.0 / 3.0)
    return alpha_bar, sigma, r_vdw, a0, r0


# ----------------------------------------------------------------------------------------
# pair functions (Sec. II.B and III)
# ----------------------------------------------------------------------------------------
def fermi(r, s, d):
    """Damping f(r, S) = 1 / (1 + exp[-d (r/S - 1)]) (Eq. damping-function)."""
    return 1.0 / (1.0 + torch.exp(-d * (r / s - 1.0)))


def cutoff_buffer(r, rc, rb):
    """f_SR / f_LR: 1 below rc - rb, 1 - 3t^2 + 2t^3 in the buffer, 0 beyond rc."""
    t = (r - rc + rb) / rb
    mid = 1.0 - 3.0 * t * t + 2.0 * t * t * t
    return torch.where(r < rc - rb, torch.ones_like(r), torch.where(r < rc, mid, torch.zeros_like(r)))


def f_inner(r, r_in):
    """f_inner = 3 (r/r_in)^2 - 2 (r/r_in)^3 below r_in, else 1 (Sec. III.B)."""
    u = r / r_in
    return torch.where(r < r_in, 3.0 * u * u - 2.0 * u * u * u, torch.ones_like(r))


def f_scs(r, r_scs):
    """f_SCS = 3 (r/r_SCS)^2 - 2 (r/r_SCS)^3 (Eq. full-pol)."""
    u = r / r_scs
    return 3.0 * u * u - 2.0 * u * u * u


def dipole_T(rvec):
    """T_ij = d/dr d/dr (1/r) = (3 r r^T - delta r^2) / r^5, rvec = r_j - r_i (bohr)."""
    r2 = (rvec * rvec).sum(-1)
    r = torch.sqrt(r2)
    outer = rvec[..., :, None] * rvec[..., None, :]
    eye = torch.eye(3, dtype=_DT)
    return (3.0 * outer - r2[..., None, None] * eye) / (r ** 5)[..., None, None]


def dipole_T_sr_bare(rvec, sigma_ij):
    """d/dr_i d/dr_j [erf(r/sigma)/r] = -T g + h (Eqs. T_SR, g-func, h-func), undamped."""
    r2 = (rvec * rvec).sum(-1)
    r = torch.sqrt(r2)
    x = r / sigma_ij
    ex = torch.exp(-x * x)
    g = torch.special.erf(x) - 2.0 / math.sqrt(math.pi) * x * ex
    hfac = 4.0 / math.sqrt(math.pi) * x ** 3 * ex
    outer = rvec[..., :, None] * rvec[..., None, :]
    h = hfac[..., None, None] * outer / (r ** 5)[..., None, None]
    return -dipole_T(rvec) * g[..., None, None] + h


# ----------------------------------------------------------------------------------------
# sites: every periodic image within r_list of the central atom is its own site
# ----------------------------------------------------------------------------------------
@dataclass
class Sites:
    atom: torch.Tensor      # (n,) long
    shift: torch.Tensor     # (n, 3) long lattice shift
    r_ang: torch.Tensor     # (n,) distance to the centre, Angstrom (no grad)
    n1: int                 # |K1| = #sites with r < r_SCS (prefix)
    ns: int                 # #sites with r < r_sphere (prefix)
    n12: int                # #sites with r < 2 r_SCS (prefix; K2 = [n1, n12))


def enumerate_sites(positions: np.ndarray, cell: np.ndarray | None, k: int, p: Params) -> Sites:
    """Brute force over all atoms and all lattice shifts; sorted by (r, atom, shift)."""
    pos = np.asarray(positions, dtype=np.float64)
    n = pos.shape[0]
    rl = p.r_list
    if cell is None:
        shifts = np.zeros((1, 3), dtype=np.int64)
    else:
        cell = np.asarray(cell, dtype=np.float64)
        inv = np.linalg.inv(cell)
        frac = pos @ inv
        dfrac = frac - frac[k]
        vol = abs(np.linalg.det(cell))
        width = np.array([vol / np.linalg.norm(np.cross(cell[(i + 1) % 3], cell[(i + 2) % 3]))
                          for i in range(3)])
        reach = rl / width
        lo = np.floor(-reach - dfrac.max(axis=0)).astype(np.int64) - 1
        hi = np.ceil(reach - dfrac.min(axis=0)).astype(np.int64) + 1
        grids = np.meshgrid(*[np.arange(lo[i], hi[i] + 1) for i in range(3)], indexing="ij")
        shifts = np.stack([g.ravel() for g in grids], axis=1)
    atoms = np.repeat(np.arange(n), shifts.shape[0])
    sh = np.tile(shifts, (n, 1))
    if cell is None:
        disp = pos[atoms] - pos[k]
    else:
        disp = pos[atoms] + sh @ cell - pos[k]
    r2 = np.einsum("ij,ij->i", disp, disp)
    keep = r2 < rl * rl
    atoms, sh, r2 = atoms[keep], sh[keep], r2[keep]
    order = np.lexsort((sh[:, 2], sh[:, 1], sh[:, 0], atoms, r2))
    atoms, sh, r2 = atoms[order], sh[order], r2[order]
    if atoms[0] != k or r2[0] != 0.0 or (len(r2) > 1 and r2[1] == 0.0):
        raise ValueError("central atom must be the unique site at distance zero")
    n1 = int(np.sum(r2 < p.r_scs ** 2))
    ns = int(np.sum(r2 < p.sphere ** 2))
    n12 = int(np.sum(r2 < (2.0 * p.r_scs) ** 2))
    return Sites(torch.as_tensor(atoms), torch.as_tensor(sh), torch.as_tensor(np.sqrt(r2)), n1, ns, n12)


def site_positions(P: torch.Tensor, cell, s: Sites, k: int) -> torch.Tensor:
    """Site displacement from the central atom, in bohr (differentiable in P, Angstrom)."""
    if cell is None:
        disp = P[s.atom] - P[k]
    else:
        disp = P[s.atom] + s.shift.to(_DT) @ torch.as_tensor(cell, dtype=_DT) - P[k]
    return disp / BOHR_ANGSTROM


# ----------------------------------------------------------------------------------------
# local SCS solve (Sec. III.B, Eq. local_pol)
# ----------------------------------------------------------------------------------------
def scs_local(x, s: Sites, alpha_bar, sigma, r_vdw, p: Params):
    """Solve B_K alpha_K = d_K for all frequencies.

    x: (n_sites, 3) bohr displacements of the sites.  Returns X with shape
    (Q, 3 n1, 3) and alpha_K (Q, n1) = Tr(X_i)/3 (Eq. after Eq. polarizabilities).
    """
    n1, n12 = s.n1, s.n12
    r_scs = p.r_scs / BOHR_ANGSTROM
    r_b = p.r_buf / BOHR_ANGSTROM
    r_in = p.r_inner / BOHR_ANGSTROM
    Q = alpha_bar.shape[1]
    a = alpha_bar[s.atom]          # (n_sites, Q)
    sg = sigma[s.atom]
    rv = r_vdw[s.atom]

    # coupled pairs i != j inside K1
    ii, jj = torch.meshgrid(torch.arange(n1), torch.arange(n1), indexing="ij")
    off = ii != jj
    ii, jj = ii[off], jj[off]
    diag = 1.0 / a[:n1].T                                   # (Q, n1): 1/alpha_bar_i on the diagonal
    eye3 = torch.eye(3, dtype=_DT)
    B = torch.diag_embed(diag.repeat_interleave(3, dim=1))
    if len(ii):
        rvec = x[jj] - x[ii]
        r = torch.sqrt((rvec * rvec).sum(-1))
        s_ij = p.beta * (rv[ii] + rv[jj])
        damp = (1.0 - fermi(r, s_ij, p.d)) * cutoff_buffer(r, r_scs, r_b)
        sig_ij = torch.sqrt(sg[ii] ** 2 + sg[jj] ** 2)          # (npair, Q)
        tsr = dipole_T_sr_bare(rvec[:, None, :].expand(-1, Q, -1), sig_ij) * damp[:, None, None, None]
        blocks = torch.zeros(Q, n1, n1, 3, 3, dtype=_DT)
        blocks = blocks.index_put((torch.arange(Q)[:, None], ii[None, :], jj[None, :]),
                                  tsr.permute(1, 0, 2, 3))
        B = B + blocks.permute(0, 1, 3, 2, 4).reshape(Q, 3 * n1, 3 * n1)

    # right-hand side d_i = 1 - sum_{j in K2} T_SR,ij alpha_bar_j
    d = eye3.repeat(n1, 1)[None].expand(Q, -1, -1).clone()
    n2 = n12 - n1
    if n2 > 0:
        ii, jj = torch.meshgrid(torch.arange(n1), torch.arange(n1, n12), indexing="ij")
        ii, jj = ii.reshape(-1), jj.reshape(-1)
        rvec = x[jj] - x[ii]
        r = torch.sqrt((rvec * rvec).sum(-1))
        s_ij = p.beta * (rv[ii] + rv[jj])
        damp = (1.0 - fermi(r, s_ij, p.d)) * cutoff_buffer(r, r_scs, r_b) * f_inner(r, r_in)
        sig_ij = torch.sqrt(sg[ii] ** 2 + sg[jj] ** 2)
        tsr = dipole_T_sr_bare(rvec[:, None, :].expand(-1, Q, -1), sig_ij) * damp[:, None, None, None]
        contrib = tsr * a[jj][:, :, None, None]              # (npair, Q, 3, 3)
        acc = torch.zeros(n1, Q, 3, 3, dtype=_DT).index_add(0, ii, contrib)
        d = d - acc.permute(1, 0, 2, 3).reshape(Q, 3 * n1, 3)

    X = torch.linalg.solve(B, d)
    alpha_K = X.reshape(Q, n1, 3, 3).diagonal(dim1=-2, dim2=-1).sum(-1) / 3.0
    return X, alpha_K, B, d


# ----------------------------------------------------------------------------------------
# local energy (Sec. III.A, Eq. E_k)
# ----------------------------------------------------------------------------------------
def blend(alpha_K, alpha_I_sites, r_bohr, p: Params):
    """Eq. full-pol: (1 - f_SCS) alpha_K + f_SCS alpha_I inside r_SCS, alpha_I outside.

    alpha_K: (Q, n1) for the K1 prefix; alpha_I_sites: (n, Q); r_bohr: (n,).
    """
    n = alpha_I_sites.shape[0]
    n1 = alpha_K.shape[1]
    r_scs = p.r_scs / BOHR_ANGSTROM
    out = alpha_I_sites.clone()
    m = min(n1, n)
    fs = f_scs(r_bohr[:m], r_scs)[:, None]
    out[:m] = (1.0 - fs) * alpha_K.T[:m] + fs * alpha_I_sites[:m]
    return out


def t_lr(x, alpha0_tilde, a0, r0, p: Params):
    """T_LR,K (3n x 3n): f_LR(r; r_MBD,p) f(r, S~) T with p = 1 on the central row/column."""
    n = x.shape[0]
    r_b = p.r_buf / BOHR_ANGSTROM
    r1 = p.r_mbd1 / BOHR_ANGSTROM
    r2c = p.r_mbd2 / BOHR_ANGSTROM
    r_t = r0 * (alpha0_tilde / a0) ** (1.0 / 3.0)            # Eq. scaled-rvdw
    ii, jj = torch.meshgrid(torch.arange(n), torch.arange(n), indexing="ij")
    off = ii != jj
    ii, jj = ii[off], jj[off]
    T = torch.zeros(n, n, 3, 3, dtype=_DT)
    if len(ii):
        rvec = x[jj] - x[ii]
        r = torch.sqrt((rvec * rvec).sum(-1))
        s_t = p.beta * (r_t[ii] + r_t[jj])
        central = (ii == 0) | (jj == 0)
        rc = torch.where(central, torch.full_like(r, r1), torch.full_like(r, r2c))
        flr = cutoff_buffer(r, rc, r_b)
        blk = dipole_T(rvec) * (flr * fermi(r, s_t, p.d))[:, None, None]
        T = T.index_put((ii, jj), blk)
    return T.permute(0, 2, 1, 3).reshape(3 * n, 3 * n)


def local_energy(T, alpha_tilde, weight, p: Params):
    """E_k in Hartree: sum_q w_q/(2 pi) sum_n c_n Tr{g_k G^(n-2) g_k^T}, c_n = -1/n.

    The central site is site 0, so g_k is rows 0..2 of G = sqrt(A) T sqrt(A).
    In log mode the k-block trace of ln(1 - G) from eigh replaces the series.
    With lanczos_steps set, c_n of this centre and frequency come from the polynomial fit.
    With fit_nodes set, the values at the nodes are the integrand I(omega_j) of the fit and
    E_k = I(0) * integral of phi (Sec. III.C).
    """
    terms = []
    for q in range(1, alpha_tilde.shape[1]):
        dq = torch.sqrt(alpha_tilde[:, q]).repeat_interleave(3)
        G = dq[:, None] * T * dq[None, :]
        if p.series_order is None:
            lam, V = torch.linalg.eigh(G)
            term = (V[:3, :] ** 2 * torch.log1p(-lam)[None, :]).sum()
        else:
            if p.lanczos_steps:
                lo, hi = lanczos_interval(G.detach().numpy(), p.lanczos_steps)
                cn = log_fit_coefficients(lo, hi, p.series_order)
            else:
                cn = [0.0, 0.0] + [-1.0 / n for n in range(2, p.series_order + 1)]
            gk = G[:3, :]
            y = gk.T
            term = torch.zeros((), dtype=_DT)
            for n in range(2, p.series_order + 1):
                term = term + float(cn[n]) * torch.trace(gk @ y)
                y = G @ y
        terms.append(term)
    if p.fit_nodes:
        I = torch.stack(terms)
        a, b = phi_fit(I, fit_node_frequencies(p.fit_nodes, p.omega_scale), p.series_order)
        om, w = quadrature(p.n_freq, p.omega_scale)
        return I[0] * phi_integral(a, b, om, w)
    e = torch.zeros((), dtype=_DT)
    for q, term in enumerate(terms, start=1):
        e = e + weight[q] / (2.0 * math.pi) * term
    return e


def spectral_ratios(T, alpha_tilde, p: Params) -> list[float]:
    """Proxy of the polarisation catastrophe (Sec. III.A: the series of Eq. E_k converges only
    when the eigenvalues of G lie inside (-1, 1)): for every integrand frequency, with
    M = floor(n_max / 2), the ratio |G^M e_k|^2 / |G^(M-1) e_k|^2 of the Frobenius norms of the
    centre's columns of G^M and G^(M-1), from explicit matrix powers.  As M grows it tends to
    the largest lambda^2 that the centre's block sees.  Empty when M < 2."""
    M = (p.series_order or 0) // 2
    if M < 2:
        return []
    out = []
    for q in range(1, alpha_tilde.shape[1]):
        dq = torch.sqrt(alpha_tilde[:, q]).repeat_interleave(3)
        G = dq[:, None] * T * dq[None, :]
        Gm1 = torch.linalg.matrix_power(G, M - 1)[:, :3]
        Gm = G @ Gm1
        out.append(float((Gm * Gm).sum() / (Gm1 * Gm1).sum()))
    return out


# ----------------------------------------------------------------------------------------
# drivers
# ----------------------------------------------------------------------------------------
class System:
    """Holds the inputs and caches site lists."""

    def __init__(self, positions, cell, species, hirshfeld, table, params: Params):
        self.pos = np.asarray(positions, dtype=np.float64)
        self.cell = None if cell is None else np.asarray(cell, dtype=np.float64)
        self.species = np.asarray(species)
        self.nu = np.asarray(hirshfeld, dtype=np.float64)
        self.table = np.asarray(table, dtype=np.float64)
        self.p = params
        self.omega, self.weight = frequencies(params)
        self.omega_s = scs_frequencies(params)
        self._sites: dict[int, Sites] = {}

    @property
    def n(self) -> int:
        return self.pos.shape[0]

    def sites(self, k: int) -> Sites:
        if k not in self._sites:
            self._sites[k] = enumerate_sites(self.pos, self.cell, k, self.p)
        return self._sites[k]

    def free(self):
        """Free-atom quantities at the SCS frequencies."""
        return free_atom(self.species, self.nu, self.table, self.omega_s)

    def central_alpha(self, atoms, P=None) -> dict[int, torch.Tensor]:
        """alpha_I,a(omega) for the listed atoms: the centre block of each atom's own solve."""
        P = torch.as_tensor(self.pos) if P is None else P
        ab, sg, rv, _, _ = self.free()
        out = {}
        for a in atoms:
            s = self.sites(a)
            x = site_positions(P, self.cell, s, a)
            _, aK, _, _ = scs_local(x, s, ab, sg, rv, self.p)
            out[a] = aK[:, 0]
        return out

    def energy_of_centre(self, k, P, alpha_I: dict[int, torch.Tensor]):
        ab, sg, rv, a0, r0 = self.free()
        s = self.sites(k)
        x = site_positions(P, self.cell, s, k)
        _, aK, _, _ = scs_local(x, s, ab, sg, rv, self.p)
        ns = s.ns
        aI = torch.stack([alpha_I[int(a)] for a in s.atom[:ns]])
        # distance to the centre (site 0 sits at the origin; keep sqrt away from zero)
        rb = torch.cat([torch.zeros(1, dtype=_DT), torch.sqrt((x[1:ns] * x[1:ns]).sum(-1))])
        at = blend(aK, aI, rb, self.p)
        T = t_lr(x[:ns], at[:, 0], a0[s.atom[:ns]], r0[s.atom[:ns]], self.p)
        if self.p.omega_ref is not None:
            # Lorentzian model: alpha~ at the quadrature nodes from its values at 0 and omega_ref
            at = lorentzian(at[:, 0], at[:, 1], self.p.omega_ref, self.omega)
        return local_energy(T, at, self.weight, self.p) * HARTREE_EV

    def spectral_ratios_of_centre(self, k, alpha_I) -> list[float]:
        """spectral_ratios of centre k's sphere at the integrand frequencies."""
        ab, sg, rv, a0, r0 = self.free()
        s = self.sites(k)
        P = torch.as_tensor(self.pos)
        x = site_positions(P, self.cell, s, k)
        _, aK, _, _ = scs_local(x, s, ab, sg, rv, self.p)
        ns = s.ns
        aI = torch.stack([alpha_I[int(a)] for a in s.atom[:ns]])
        rb = torch.cat([torch.zeros(1, dtype=_DT), torch.sqrt((x[1:ns] * x[1:ns]).sum(-1))])
        at = blend(aK, aI, rb, self.p)
        T = t_lr(x[:ns], at[:, 0], a0[s.atom[:ns]], r0[s.atom[:ns]], self.p)
        if self.p.omega_ref is not None:
            at = lorentzian(at[:, 0], at[:, 1], self.p.omega_ref, self.omega)
        return spectral_ratios(T, at, self.p)

    def spectral_flags(self, centres=None) -> int:
        """Number of (centre, integrand frequency) terms whose spectral ratio is >= 1."""
        centres = list(range(self.n)) if centres is None else [int(c) for c in centres]
        need = sorted({int(a) for k in centres for a in self.sites(k).atom[: self.sites(k).ns]})
        with torch.no_grad():
            aI = self.central_alpha(need)
            return sum(sum(1 for r in self.spectral_ratios_of_centre(k, aI) if r >= 1.0) for k in centres)

    def energies(self, centres=None) -> np.ndarray:
        """Per-atom energies E_k in eV for the listed centres (default all)."""
        centres = list(range(self.n)) if centres is None else [int(c) for c in centres]
        need = sorted({int(a) for k in centres for a in self.sites(k).atom[: self.sites(k).ns]})
        P = torch.as_tensor(self.pos)
        with torch.no_grad():
            aI = self.central_alpha(need, P)
            return np.array([float(self.energy_of_centre(k, P, aI)) for k in centres])

    def paper_forces(self, centres=None) -> np.ndarray:
        """The paper's approximate forces (Sec. III.D); see the module function."""
        return paper_forces(self, centres)

    def energies_forces(self, centres=None, weights=None):
        """Energies (eV) of the centres and F = -d(sum_k w_k E_k)/dR (eV/Angstrom), all atoms."""
        centres = list(range(self.n)) if centres is None else [int(c) for c in centres]
        w = np.ones(len(centres)) if weights is None else np.asarray(weights, dtype=np.float64)
        need = sorted({int(a) for k in centres for a in self.sites(k).atom[: self.sites(k).ns]})
        P0 = torch.as_tensor(self.pos)
        with torch.no_grad():
            aI0 = self.central_alpha(need, P0)
        grad = torch.zeros_like(P0)
        seed = {a: torch.zeros_like(aI0[a]) for a in need}
        energies = []
        for k, wk in zip(centres, w):
            P = P0.clone().requires_grad_(True)
            leaves = {a: aI0[a].clone().requires_grad_(True) for a in
                      {int(b) for b in self.sites(k).atom[: self.sites(k).ns]}}
            e = self.energy_of_centre(k, P, leaves)
            energies.append(float(e.detach()))
            if wk == 0.0:
                continue
            (wk * e).backward()
            grad += P.grad
            for a, t in leaves.items():
                if t.grad is not None:
                    seed[a] += t.grad
        for a in need:
            if torch.count_nonzero(seed[a]) == 0:
                continue
            P = P0.clone().requires_grad_(True)
            aI = self.central_alpha([a], P)[a]
            if not aI.requires_grad:       # no SCS neighbours: alpha_I does not move
                continue
            (aI * seed[a]).sum().backward()
            grad += P.grad
        return np.array(energies), (-grad).numpy()


def _paper_total(T, alpha_tilde, weight, p: Params):
    """E^{k,tot} of Eq. E_k_tot in Hartree with the central-atom approximation of Sec. III.D
    built into its derivative: the n = 2 term sees every block of G, the n >= 3 terms only the
    blocks in the row and column of the central site (the others enter as constants)."""
    n3 = T.shape[0]
    central = torch.zeros(n3, n3, dtype=torch.bool)
    central[:3, :] = True
    central[:, :3] = True
    e = torch.zeros((), dtype=_DT)
    for q in range(1, alpha_tilde.shape[1]):
        dq = torch.sqrt(alpha_tilde[:, q]).repeat_interleave(3)
        G = dq[:, None] * T * dq[None, :]
        if p.lanczos_steps:
            lo, hi = lanczos_interval(G.detach().numpy(), p.lanczos_steps)
            cn = log_fit_coefficients(lo, hi, p.series_order)
        else:
            cn = [0.0, 0.0] + [-1.0 / n for n in range(2, p.series_order + 1)]
        term = float(cn[2]) * torch.trace(G @ G)
        Gm = torch.where(central, G, G.detach())
        Y = Gm @ Gm
        for n in range(3, p.series_order + 1):
            Y = Y @ Gm
            term = term + float(cn[n]) * torch.trace(Y)
        e = e + weight[q] / (2.0 * math.pi) * term
    return e


def paper_forces(sysm: "System", centres=None) -> np.ndarray:
    """The paper's approximate forces (Sec. III.D) in eV/Angstrom: for every atom k,
    F_k = -dE^{k,tot}/dr_k of its own sphere (every image of k in the sphere moves with it),
    with alpha_I held fixed (Eq. full-pol-grad) and the central-atom approximation for n >= 3
    (Eq. cent-appr).  The frequency integral is the quadrature; with fit_nodes set it is the
    paper's fitted force integrand instead: the force integrand F_k(nu_i) (the same derivative of
    the bare integrand at one frequency) at omega = 0 and the fit nodes, per Cartesian component
    the fit theta of the ratios F(nu_i) / F(0) (theta_fit), and F_k = F_k(0) times the integral
    of theta / (2 pi) (the integrand of Eq. mbd-forces-sym with its frequency dependence fitted)."""
    p = sysm.p
    if p.series_order is None:
        raise ValueError("paper forces need the truncated series")
    centres = list(range(sysm.n)) if centres is None else [int(c) for c in centres]
    need = sorted({int(a) for k in centres for a in sysm.sites(k).atom[: sysm.sites(k).ns]})
    P0 = torch.as_tensor(sysm.pos)
    with torch.no_grad():
        aI0 = sysm.central_alpha(need, P0)
    ab, sg, rv, a0, r0 = sysm.free()
    F = np.zeros((sysm.n, 3))
    for k in centres:
        P = P0.clone().requires_grad_(True)
        s = sysm.sites(k)
        x = site_positions(P, sysm.cell, s, k)
        _, aK, _, _ = scs_local(x, s, ab, sg, rv, p)
        ns = s.ns
        aI = torch.stack([aI0[int(a)] for a in s.atom[:ns]])
        rb = torch.cat([torch.zeros(1, dtype=_DT), torch.sqrt((x[1:ns] * x[1:ns]).sum(-1))])
        at = blend(aK, aI, rb, p)
        T = t_lr(x[:ns], at[:, 0], a0[s.atom[:ns]], r0[s.atom[:ns]], p)
        if p.omega_ref is not None:
            at = lorentzian(at[:, 0], at[:, 1], p.omega_ref, sysm.omega)
        if not p.fit_nodes:
            e = _paper_total(T, at, sysm.weight, p) * HARTREE_EV
            g = torch.autograd.grad(e, P)[0]
            F[k] = -g[k].numpy()
            continue
        # force integrand at each sample frequency (columns 1.. of alpha~): the bare integrand
        # (weight 2 pi at that column only), differentiated like the quadrature form
        nq = at.shape[1]
        Fs = []
        for q in range(1, nq):
            wq = torch.zeros(nq, dtype=_DT)
            wq[q] = 2.0 * math.pi
            e = _paper_total(T, at, wq, p) * HARTREE_EV
            g = torch.autograd.grad(e, P, retain_graph=q < nq - 1)[0]
            Fs.append(-g[k].numpy())
        Fs = np.array(Fs)                                  # (samples, 3)
        nodes = fit_node_frequencies(p.fit_nodes, p.omega_scale)
        M, K = theta_orders(p.fit_nodes)
        om, w = quadrature(p.n_freq, p.omega_scale)
        for gam in range(3):
            if Fs[0, gam] == 0.0:
                continue
            u, v = theta_fit(Fs[:, gam] / Fs[0, gam], nodes, M, K)
            F[k, gam] = Fs[0, gam] * theta_integral(u, v, om, w)
    return F


def with_params(p: Params, **kw) -> Params:
    return replace(p, **kw)
