"""Thin ctypes binding of the lMBD C ABI (include/lmbd.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``liblmbd.so``.  Arrays may be torch tensors (CUDA or CPU) or numpy
arrays; CUDA tensors are passed as device pointers, everything else as host
pointers (the library copies host arrays itself).  If the shared library has
not been built this module raises at import time: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblmbd.so")

LMBD_OK, LMBD_EINVAL, LMBD_ENOMEM, LMBD_NOT_SPD, LMBD_ECUDA, LMBD_ECAPACITY, LMBD_EUNSUPPORTED = range(7)
LMBD_ESCRATCH, LMBD_EMODEL, LMBD_ETIMEOUT, LMBD_CATASTROPHE = 7, 8, 9, 10
FREQ_QUADRATURE, FREQ_LORENTZIAN = 0, 1
FORCES_EXACT, FORCES_PAPER = 0, 1
LAUNCH_BATCHED, LAUNCH_PER_ATOM = 0, 1
PREC_FP64, PREC_SLICED = 0, 1
MMA_WARP, MMA_TC05 = 0, 1


class Species(ctypes.Structure):
    _fields_ = [("alpha0", ctypes.c_double), ("c6", ctypes.c_double), ("r0", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("r_scs", "r_mbd1", "r_mbd2", "r_sphere", "r_buf", "r_inner", "beta", "d", "omega_scale")]


PHASES = ("neighbors", "scs", "prepare", "chain", "energy", "adj_series", "adj_pair", "adj_blend",
          "adj_scs", "output")
NPHASE = len(PHASES)


class Stats(ctypes.Structure):
    _fields_ = [("flops", ctypes.c_double * NPHASE), ("ms", ctypes.c_double * NPHASE),
                ("launches", ctypes.c_int * NPHASE), ("bytes_workspace", ctypes.c_double),
                ("n_sites", ctypes.c_longlong), ("max_k1", ctypes.c_int), ("max_sphere", ctypes.c_int),
                ("max_sites", ctypes.c_int), ("kernel_launches", ctypes.c_int), ("bytes_arena", ctypes.c_double),
                ("waves_scs", ctypes.c_int), ("waves_mbd", ctypes.c_int), ("scs_recomputed", ctypes.c_int),
                ("scs_pairs", ctypes.c_longlong), ("scs_adjacency", ctypes.c_longlong),
                ("ms_kernel", ctypes.c_double * 2), ("scs_lu_systems", ctypes.c_longlong),
                ("sites_refreshed", ctypes.c_int), ("reused_forward", ctypes.c_int),
                ("spectral_flags", ctypes.c_longlong), ("tlr_pairs", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            if k in ("flops", "ms", "launches"):
                d[k] = {ph: v[i] for i, ph in enumerate(PHASES)}
            elif k == "ms_kernel":
                d[k] = {"scs_factor": v[0], "scs_adjoint": v[1]}
            else:
                d[k] = v
        return d


class LmbdError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {lib().lmbd_status_string(status).decode()} (status {status})")
        self.status = status


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2407_06409_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.lmbd_status_string.restype = ctypes.c_char_p
        L.lmbd_status_string.argtypes = [ctypes.c_int]
        L.lmbd_default_params.argtypes = [ctypes.POINTER(Params)]
        L.lmbd_create.argtypes = [ctypes.POINTER(Species), ctypes.c_int, ctypes.POINTER(Params), ctypes.c_int,
                                  ctypes.c_int, ctypes.POINTER(_P)]
        L.lmbd_energy_forces.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]
        L.lmbd_energy_forces_weighted.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P]
        L.lmbd_energy_keep.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P]
        L.lmbd_forces_kept.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]
        L.lmbd_set_launch_mode.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_profiling.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_precision.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_mma_path.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_wait_budget.argtypes = [_P, ctypes.c_longlong]
        L.lmbd_set_memory_budget.argtypes = [_P, ctypes.c_size_t]
        L.lmbd_set_frequency_model.argtypes = [_P, ctypes.c_int, ctypes.c_double]
        L.lmbd_set_integrand_fit.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_series_fit.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_force_model.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_spectral_check.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_sparse_tlr.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_log_mode.argtypes = [_P, ctypes.c_int]
        L.lmbd_set_verlet_skin.argtypes = [_P, ctypes.c_double]
        L.lmbd_autotune.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int)]
        L.lmbd_release_workspace.argtypes = [_P]
        L.lmbd_held_bytes.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t)]
        L.lmbd_get_central_polarizabilities.argtypes = [_P, _P, _P]
        L.lmbd_get_site_counts.argtypes = [_P, _P, _P]
        L.lmbd_get_quadrature.argtypes = [_P, _D, _D]
        L.lmbd_get_stats.argtypes = [_P, ctypes.POINTER(Stats)]
        L.lmbd_destroy.argtypes = [_P]
        for f in ("lmbd_default_params", "lmbd_create", "lmbd_energy_forces", "lmbd_energy_forces_weighted",
                  "lmbd_energy_keep", "lmbd_forces_kept",
                  "lmbd_set_launch_mode", "lmbd_set_profiling", "lmbd_set_precision", "lmbd_set_mma_path", "lmbd_set_wait_budget", "lmbd_set_memory_budget", "lmbd_set_frequency_model",
                  "lmbd_set_integrand_fit", "lmbd_set_series_fit", "lmbd_set_force_model", "lmbd_set_spectral_check",
                  "lmbd_set_log_mode", "lmbd_set_verlet_skin", "lmbd_set_sparse_tlr",
                  "lmbd_autotune",
                  "lmbd_release_workspace", "lmbd_held_bytes",
                  "lmbd_get_central_polarizabilities", "lmbd_get_site_counts",
                  "lmbd_get_quadrature", "lmbd_get_stats", "lmbd_destroy"):
            getattr(L, f).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(status: int, what: str) -> None:
    if status != LMBD_OK:
        raise LmbdError(status, what)


def default_params(**kw) -> Params:
    p = Params()
    _check(lib().lmbd_default_params(ctypes.byref(p)), "lmbd_default_params")
    for k, v in kw.items():
        setattr(p, k, float(v))
    return p


def _torch():
    import torch
    return torch


def _as_arg(x, dtype):
    """(pointer, keepalive) for a torch tensor / numpy array / None."""
    if x is None:
        return None, None
    torch = _torch()
    if isinstance(x, torch.Tensor):
        t = x.detach().to(dtype).contiguous()
        return ctypes.c_void_p(t.data_ptr()), t
    a = np.ascontiguousarray(x, dtype={torch.float64: np.float64, torch.int32: np.int32}[dtype])
    return ctypes.c_void_p(a.ctypes.data), a


def _stream_ptr(stream, device):
    """The given stream; else the current stream of a CUDA device; else the legacy stream."""
    torch = _torch()
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream)
    if device.type != "cuda":
        return None
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class LMBD:
    """One library context: species table, model parameters, quadrature and series order."""

    def __init__(self, table, params: Params | None = None, n_freq: int = 12, series_order: int = 6):
        table = np.asarray(table, dtype=np.float64).reshape(-1, 3)
        sp = (Species * len(table))(*[Species(*row) for row in table])
        self.params = params if params is not None else default_params()
        self.n_freq = int(n_freq)
        self.series_order = int(series_order)
        h = _P()
        _check(lib().lmbd_create(sp, len(table), ctypes.byref(self.params), self.n_freq, self.series_order,
                                 ctypes.byref(h)), "lmbd_create")
        self._h = h
        self.last_status = LMBD_OK

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().lmbd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_launch_mode(self, mode: int) -> None:
        _check(lib().lmbd_set_launch_mode(self._h, int(mode)), "lmbd_set_launch_mode")

    def set_precision(self, mode: int) -> None:
        _check(lib().lmbd_set_precision(self._h, int(mode)), "lmbd_set_precision")

    def set_mma_path(self, path: int) -> None:
        """Tensor-core path of the sliced products: MMA_TC05 (tcgen05, default) or MMA_WARP (mma.sync)."""
        _check(lib().lmbd_set_mma_path(self._h, int(path)), "lmbd_set_mma_path")

    def set_wait_budget(self, cycles: int) -> None:
        """Bound (SM cycles) of each wait in the tcgen05 kernels' main loop; 0 = default (~2 s)."""
        _check(lib().lmbd_set_wait_budget(self._h, int(cycles)), "lmbd_set_wait_budget")

    def set_memory_budget(self, nbytes: int) -> None:
        """Device bytes this context may hold (0 = free memory less 1 GiB); larger inputs run in waves."""
        _check(lib().lmbd_set_memory_budget(self._h, int(nbytes)), "lmbd_set_memory_budget")

    def set_frequency_model(self, model: int, omega_ref: float = 0.0) -> None:
        """FREQ_QUADRATURE (SCS at every node) or FREQ_LORENTZIAN (SCS at 0 and omega_ref, Ha)."""
        _check(lib().lmbd_set_frequency_model(self._h, int(model), float(omega_ref)), "lmbd_set_frequency_model")
        self._lorentz = model == FREQ_LORENTZIAN
        self._update_scs_columns()

    def set_integrand_fit(self, n_fit_nodes: int) -> None:
        """0: integrand at every quadrature node.  m >= series_order: the fitted integrand of
        Sec. III.C -- I(omega) at 0 and m fit nodes, phi(omega) by non-negative least squares,
        E_k = I(0) times the quadrature of phi."""
        _check(lib().lmbd_set_integrand_fit(self._h, int(n_fit_nodes)), "lmbd_set_integrand_fit")
        self._fit_nodes = int(n_fit_nodes)
        self._update_scs_columns()

    def set_series_fit(self, lanczos_steps: int) -> None:
        """0: c_n = -1/n.  m > 0: c_n per centre and frequency from the least-squares fit of
        ln(1 - lambda) on the m-step Lanczos estimate of G's spectral interval (Sec. III.A)."""
        _check(lib().lmbd_set_series_fit(self._h, int(lanczos_steps)), "lmbd_set_series_fit")

    def set_verlet_skin(self, skin: float) -> None:
        """Resident site lists across frames of one structure (Angstrom; 0 = search every call)."""
        _check(lib().lmbd_set_verlet_skin(self._h, float(skin)), "lmbd_set_verlet_skin")

    def set_log_mode(self, lanczos_steps: int) -> None:
        """0: truncated series; m > 0: [ln(1 - G)]_kk from m-step Lanczos Gauss rules (energies only)."""
        _check(lib().lmbd_set_log_mode(self._h, int(lanczos_steps)), "lmbd_set_log_mode")

    def set_sparse_tlr(self, on: bool) -> None:
        """True: block-sparse T_LR (coupled site pairs only, float-float chain and pair products)."""
        _check(lib().lmbd_set_sparse_tlr(self._h, 1 if on else 0), "lmbd_set_sparse_tlr")

    def set_spectral_check(self, fail: bool) -> None:
        """True: calls whose spectral proxy reached 1 return LMBD_CATASTROPHE (outputs written)."""
        _check(lib().lmbd_set_spectral_check(self._h, 1 if fail else 0), "lmbd_set_spectral_check")

    def set_force_model(self, model: int) -> None:
        """FORCES_EXACT (gradient of the energies) or FORCES_PAPER (Sec. III.D approximations)."""
        _check(lib().lmbd_set_force_model(self._h, int(model)), "lmbd_set_force_model")

    def _update_scs_columns(self) -> None:
        # SCS solves: 0 and omega_ref, or omega = 0 and every frequency at which the integrand
        # is evaluated (the quadrature nodes, or 0 and the fit nodes)
        fit = getattr(self, "_fit_nodes", 0)
        nodes = fit + 1 if fit else self.n_freq
        self._scs_columns = 2 if getattr(self, "_lorentz", False) else nodes + 1

    def release_workspace(self) -> None:
        """Free the context's device workspaces (the next call allocates again)."""
        _check(lib().lmbd_release_workspace(self._h), "lmbd_release_workspace")

    def held_bytes(self) -> int:
        out = ctypes.c_size_t(0)
        _check(lib().lmbd_held_bytes(self._h, ctypes.byref(out)), "lmbd_held_bytes")
        return int(out.value)

    def set_profiling(self, on: bool) -> None:
        _check(lib().lmbd_set_profiling(self._h, 1 if on else 0), "lmbd_set_profiling")

    def energy_forces(self, positions, cell, species, hirshfeld, forces: bool = True, weights=None,
                      stream=None, allow_not_spd: bool = False, allow_catastrophe: bool = False):
        """Per-atom energies (eV) and forces (eV/Angstrom) as torch tensors.

        Outputs live on the device of ``positions`` (CPU tensors / numpy -> CPU).
        ``weights`` (N) turns forces into -d(sum_k w_k E_k)/dR.
        """
        torch = _torch()
        dev = positions.device if isinstance(positions, torch.Tensor) else torch.device("cpu")
        n = int(positions.shape[0])
        pp, k1 = _as_arg(positions, torch.float64)
        cp, k2 = _as_arg(cell, torch.float64)
        sp, k3 = _as_arg(species, torch.int32)
        hp, k4 = _as_arg(hirshfeld, torch.float64)
        wp, k5 = _as_arg(weights, torch.float64)
        e = torch.empty(n, dtype=torch.float64, device=dev)
        f = torch.empty((n, 3), dtype=torch.float64, device=dev) if forces else None
        st = _stream_ptr(stream, dev)
        status = lib().lmbd_energy_forces_weighted(
            self._h, n, pp, cp, sp, hp, wp, ctypes.c_void_p(e.data_ptr()),
            ctypes.c_void_p(f.data_ptr()) if f is not None else None, st)
        self.last_status = status
        if not (status == LMBD_OK or (allow_not_spd and status == LMBD_NOT_SPD)
                or (allow_catastrophe and status == LMBD_CATASTROPHE)):
            raise LmbdError(status, "lmbd_energy_forces")
        del k1, k2, k3, k4, k5
        return e, f

    def energy_keep(self, positions, cell, species, hirshfeld, stream=None):
        """Energies (lmbd_energy_keep), keeping the forward state for forces_kept."""
        torch = _torch()
        dev = positions.device if isinstance(positions, torch.Tensor) else torch.device("cpu")
        n = int(positions.shape[0])
        pp, k1 = _as_arg(positions, torch.float64)
        cp, k2 = _as_arg(cell, torch.float64)
        sp, k3 = _as_arg(species, torch.int32)
        hp, k4 = _as_arg(hirshfeld, torch.float64)
        e = torch.empty(n, dtype=torch.float64, device=dev)
        st = _stream_ptr(stream, dev)
        status = lib().lmbd_energy_keep(self._h, n, pp, cp, sp, hp, ctypes.c_void_p(e.data_ptr()), st)
        self.last_status = status
        _check(status, "lmbd_energy_keep")
        del k1, k2, k3, k4
        return e

    def forces_kept(self, positions, cell, species, hirshfeld, weights=None, stream=None):
        """-d(sum_k w_k E_k)/dR (lmbd_forces_kept): the reverse sweep on the kept forward state
        when it matches these inputs, else a whole call."""
        torch = _torch()
        dev = positions.device if isinstance(positions, torch.Tensor) else torch.device("cpu")
        n = int(positions.shape[0])
        pp, k1 = _as_arg(positions, torch.float64)
        cp, k2 = _as_arg(cell, torch.float64)
        sp, k3 = _as_arg(species, torch.int32)
        hp, k4 = _as_arg(hirshfeld, torch.float64)
        wp, k5 = _as_arg(weights, torch.float64)
        f = torch.empty((n, 3), dtype=torch.float64, device=dev)
        st = _stream_ptr(stream, dev)
        status = lib().lmbd_forces_kept(self._h, n, pp, cp, sp, hp, wp, ctypes.c_void_p(f.data_ptr()), st)
        self.last_status = status
        _check(status, "lmbd_forces_kept")
        del k1, k2, k3, k4, k5
        return f

    def autotune(self, positions, cell, species, hirshfeld, forces: bool = True, stream=None) -> int:
        """Pick the SCS bucket width for this kind of structure (lmbd_autotune); returns it."""
        torch = _torch()
        dev = positions.device if isinstance(positions, torch.Tensor) else torch.device("cpu")
        n = int(positions.shape[0])
        pp, k1 = _as_arg(positions, torch.float64)
        cp, k2 = _as_arg(cell, torch.float64)
        sp, k3 = _as_arg(species, torch.int32)
        hp, k4 = _as_arg(hirshfeld, torch.float64)
        e = torch.empty(n, dtype=torch.float64, device=dev)
        f = torch.empty((n, 3), dtype=torch.float64, device=dev) if forces else None
        width = ctypes.c_int(0)
        _check(lib().lmbd_autotune(self._h, n, pp, cp, sp, hp, ctypes.c_void_p(e.data_ptr()),
                                   ctypes.c_void_p(f.data_ptr()) if f is not None else None,
                                   _stream_ptr(stream, dev), ctypes.byref(width)), "lmbd_autotune")
        del k1, k2, k3, k4
        return int(width.value)

    def central_polarizabilities(self, n: int, device="cpu"):
        torch = _torch()
        out = torch.empty((n, getattr(self, "_scs_columns", self.n_freq + 1)), dtype=torch.float64, device=device)
        st = _stream_ptr(None, out.device)
        _check(lib().lmbd_get_central_polarizabilities(self._h, ctypes.c_void_p(out.data_ptr()), st),
               "lmbd_get_central_polarizabilities")
        return out

    def site_counts(self, n: int):
        out = np.empty((n, 4), dtype=np.int32)
        _check(lib().lmbd_get_site_counts(self._h, ctypes.c_void_p(out.ctypes.data), None), "lmbd_get_site_counts")
        return out

    def quadrature(self):
        om = np.empty(self.n_freq)
        w = np.empty(self.n_freq)
        _check(lib().lmbd_get_quadrature(self._h, om.ctypes.data_as(_D), w.ctypes.data_as(_D)),
               "lmbd_get_quadrature")
        return om, w

    def stats(self) -> dict:
        s = Stats()
        _check(lib().lmbd_get_stats(self._h, ctypes.byref(s)), "lmbd_get_stats")
        return s.as_dict()


def _make_energy_function():
    torch = _torch()

    class LmbdEnergy(torch.autograd.Function):
        """Per-atom lMBD energies with the hand-written adjoint as backward.

        forward(positions, model, cell, species, hirshfeld) -> E (N) with the forward state kept
        on the device; backward runs the library's reverse sweep on it for weights w = dL/dE:
        dL/dR = -F(w).
        """

        @staticmethod
        def forward(ctx, positions, model, cell, species, hirshfeld):
            # the library keeps the forward state (factors, T_LR, Krylov blocks) for the backward
            e = model.energy_keep(positions.detach(), cell, species, hirshfeld)
            ctx.model = model
            ctx.save_for_backward(positions)
            ctx.extra = (cell, species, hirshfeld)
            return e

        @staticmethod
        def backward(ctx, grad_e):
            (positions,) = ctx.saved_tensors
            cell, species, hirshfeld = ctx.extra
            # the reverse sweep alone on the kept state (a whole call if it is gone)
            f = ctx.model.forces_kept(positions.detach(), cell, species, hirshfeld, weights=grad_e.contiguous())
            return -f, None, None, None, None

    return LmbdEnergy


_ENERGY_FN = None


def lmbd_energy(positions, model: LMBD, cell, species, hirshfeld):
    """Differentiable per-atom energies (torch.autograd)."""
    global _ENERGY_FN
    if _ENERGY_FN is None:
        _ENERGY_FN = _make_energy_function()
    return _ENERGY_FN.apply(positions, model, cell, species, hirshfeld)
