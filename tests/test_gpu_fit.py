"""Fitted integrand of Sec. III.C on the GPU against the oracle's fit.

The integrand I(omega) of Eq. integrand at omega = 0 and m fit nodes, phi(omega) = a / (1 +
sum_n b_n omega^(2n)) fitted per centre by non-negative least squares, E_k = I(0) times the
quadrature of phi (Eq. E_MBD_k); forces are the exact gradient through the fit.  Energies
within 1e-10 relative and forces within 1e-8 eV/Angstrom of the oracle, alone and combined
with the Lorentzian frequency model (the paper's own fast path).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_06409_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    from paper_2407_06409_gb300 import build, lmbd
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lmbd


def _op(p, **kw):
    return oracle.Params(r_scs=p.r_scs, r_mbd1=p.r_mbd1, r_mbd2=p.r_mbd2, r_sphere=p.r_sphere, r_buf=p.r_buf,
                         r_inner=p.r_inner, beta=p.beta, d=p.d, n_freq=12, series_order=6,
                         omega_scale=p.omega_scale, **kw)


def _dev(s):
    cell = None if s.cell is None else torch.tensor(s.cell, device="cuda")
    return (torch.tensor(s.positions, device="cuda"), cell,
            torch.tensor(s.species, dtype=torch.int32, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"))


def test_cluster_energies_with_per_node_scs(lm):
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_integrand_fit(6)
    e, _ = model.energy_forces(*_dev(s), forces=False)
    so = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _op(p, fit_nodes=6))
    ref = so.energies()
    assert np.max(np.abs(e.cpu().numpy() - ref) / np.abs(ref)) < 1e-10
    # SCS at omega = 0, then at the integrand's frequencies (0 again and the 6 fit nodes)
    aI = model.central_polarizabilities(s.n_atoms).numpy()
    assert aI.shape == (24, 8)
    ca = so.central_alpha(range(24))
    for a, v in ca.items():
        assert np.allclose(aI[a], v.numpy(), rtol=1e-12, atol=0)
    # switching the fit off gives the quadrature energies again
    model.set_integrand_fit(0)
    e_q, _ = model.energy_forces(*_dev(s), forces=False)
    ref_q = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _op(p)).energies()
    assert np.max(np.abs(e_q.cpu().numpy() - ref_q) / np.abs(ref_q)) < 1e-10
    assert np.max(np.abs(e.cpu().numpy() - ref_q) / np.abs(ref_q)) > 1e-6


@pytest.mark.parametrize("omega_ref", [None, 4.0])
def test_box_forces_match_oracle(lm, omega_ref):
    s = inputs.box(110, seed=1, jitter=0.05)
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    if omega_ref is not None:
        model.set_frequency_model(lm.FREQ_LORENTZIAN, omega_ref)
    model.set_integrand_fit(6)
    e, f = model.energy_forces(*_dev(s), forces=True)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table,
                       _op(p, omega_ref=omega_ref, fit_nodes=6))
    e_ref, f_ref = so.energies_forces()
    assert np.max(np.abs(e.cpu().numpy() - e_ref) / np.abs(e_ref)) < 1e-10
    assert np.abs(f.cpu().numpy() - f_ref).max() < 1e-8
    # memory-bounded waves give the same result in this mode
    st = model.stats()
    mb = lm.LMBD(s.table, p, 12, 6)
    if omega_ref is not None:
        mb.set_frequency_model(lm.FREQ_LORENTZIAN, omega_ref)
    mb.set_integrand_fit(6)
    mb.set_memory_budget(int(st["bytes_workspace"] - st["bytes_arena"] + 0.1 * st["bytes_arena"]))
    e2, f2 = mb.energy_forces(*_dev(s), forces=True)
    assert mb.stats()["waves_mbd"] > 1
    assert torch.equal(e2, e)
    assert (f2 - f).abs().max().item() < 1e-12


def test_fit_settings_are_checked(lm):
    s = inputs.cluster(12, seed=2)
    model = lm.LMBD(s.table, lm.default_params(r_scs=4.0, r_mbd1=4.0, r_mbd2=4.0, r_sphere=4.0), 12, 6)
    for bad in (-1, 5, 25):
        with pytest.raises(lm.LmbdError) as err:
            model.set_integrand_fit(bad)
        assert err.value.status == lm.LMBD_EINVAL
    model.set_integrand_fit(24)
    e, f = model.energy_forces(*_dev(s), forces=True)
    assert torch.isfinite(e).all() and torch.isfinite(f).all()
