"""Polynomial-fit series coefficients of Sec. III.A on the GPU against the oracle.

Per central atom and frequency, the Lanczos estimate of the spectral interval of G and the
least-squares fit of ln(1 - lambda) on it give c_n in place of -1/n (Eqs. diagonal_appr and
polynomial-fit); forces hold the c_n fixed.  Energies within 1e-10 relative and forces within
1e-8 eV/Angstrom of the oracle, alone and with the paper's fitted frequency path.
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


def test_cluster_energies(lm):
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_series_fit(20)
    e, _ = model.energy_forces(*_dev(s), forces=False)
    ref = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _op(p, lanczos_steps=20)).energies()
    assert np.max(np.abs(e.cpu().numpy() - ref) / np.abs(ref)) < 1e-10
    model.set_series_fit(0)
    e0, _ = model.energy_forces(*_dev(s), forces=False)
    assert np.max(np.abs(e.cpu().numpy() - e0.cpu().numpy()) / np.abs(ref)) > 1e-9


@pytest.mark.parametrize("fast_path", [False, True])
def test_box_forces_match_oracle(lm, fast_path):
    s = inputs.box(110, seed=1, jitter=0.05)
    p = lm.default_params()
    kw = dict(lanczos_steps=12)
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_series_fit(12)
    if fast_path:   # with the Lorentzian model and the fitted integrand as well
        model.set_frequency_model(lm.FREQ_LORENTZIAN, 4.0)
        model.set_integrand_fit(6)
        kw.update(omega_ref=4.0, fit_nodes=6)
    e, f = model.energy_forces(*_dev(s), forces=True)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p, **kw))
    e_ref, f_ref = so.energies_forces()
    assert np.max(np.abs(e.cpu().numpy() - e_ref) / np.abs(e_ref)) < 1e-10
    assert np.abs(f.cpu().numpy() - f_ref).max() < 1e-8
    st = model.stats()
    mb = lm.LMBD(s.table, p, 12, 6)
    mb.set_series_fit(12)
    if fast_path:
        mb.set_frequency_model(lm.FREQ_LORENTZIAN, 4.0)
        mb.set_integrand_fit(6)
    mb.set_memory_budget(int(st["bytes_workspace"] - st["bytes_arena"] + 0.1 * st["bytes_arena"]))
    e2, f2 = mb.energy_forces(*_dev(s), forces=True)
    assert mb.stats()["waves_mbd"] > 1
    assert torch.equal(e2, e)
    assert (f2 - f).abs().max().item() < 1e-12


def test_series_fit_settings_are_checked(lm):
    s = inputs.cluster(12, seed=2)
    model = lm.LMBD(s.table, lm.default_params(r_scs=4.0, r_mbd1=4.0, r_mbd2=4.0, r_sphere=4.0), 12, 6)
    for bad in (-1, 65):
        with pytest.raises(lm.LmbdError) as err:
            model.set_series_fit(bad)
        assert err.value.status == lm.LMBD_EINVAL
    # more steps than the Krylov space has: the iteration stops at its dimension
    model.set_series_fit(64)
    e, f = model.energy_forces(*_dev(s), forces=True)
    ref = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table,
                        _op(lm.default_params(r_scs=4.0, r_mbd1=4.0, r_mbd2=4.0, r_sphere=4.0),
                            lanczos_steps=64)).energies()
    # (an atom without neighbours inside the 4 Angstrom sphere has E_k = 0 on both sides)
    assert np.all(np.abs(e.cpu().numpy() - ref) <= 1e-10 * np.abs(ref))
    assert torch.isfinite(f).all()
