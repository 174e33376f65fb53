"""CPU oracle for the lMBD hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product package.
"""
from .lmbd_oracle import (BOHR_ANGSTROM, HARTREE_EV, Params, System, quadrature, frequencies,
                          free_atom, fermi, cutoff_buffer, f_inner, f_scs, dipole_T,
                          dipole_T_sr_bare, enumerate_sites, scs_local, t_lr, local_energy,
                          blend, site_positions, with_params, fit_node_frequencies, nnls_passive,
                          phi_fit, phi_integral, lorentzian, splitmix64_unit, lanczos_interval,
                          log_fit_coefficients, spectral_ratios, theta_orders, theta_fit,
                          theta_integral, paper_forces)

__all__ = ["BOHR_ANGSTROM", "HARTREE_EV", "Params", "System", "quadrature", "frequencies",
           "free_atom", "fermi", "cutoff_buffer", "f_inner", "f_scs", "dipole_T",
           "dipole_T_sr_bare", "enumerate_sites", "scs_local", "t_lr", "local_energy", "blend",
           "site_positions", "with_params", "fit_node_frequencies", "nnls_passive", "phi_fit",
           "phi_integral", "lorentzian", "splitmix64_unit", "lanczos_interval", "log_fit_coefficients",
           "spectral_ratios", "theta_orders", "theta_fit", "theta_integral", "paper_forces"]
