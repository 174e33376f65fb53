"""The paper's approximate forces (Sec. III.D) on the GPU against the oracle's.

F_k = -dE^{k,tot}/dr_k of atom k's own sphere with alpha_I held and, for n >= 3, the
derivative kept in the central row and column only (Eqs. full-pol-grad, mbd-forces,
cent-appr); within 1e-8 eV/Angstrom of the oracle, alone and with the Lorentzian model and the
polynomial-fit coefficients, and with the fitted force integrand theta(omega) of Sec. III.D.
Energies are those of the exact mode.
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


def test_cluster_paper_forces(lm):
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    model = lm.LMBD(s.table, p, 12, 6)
    e_x, f_x = model.energy_forces(*_dev(s), forces=True)
    model.set_force_model(lm.FORCES_PAPER)
    e, f = model.energy_forces(*_dev(s), forces=True)
    assert torch.equal(e, e_x)
    so = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _op(p))
    f_ref = so.paper_forces()
    assert np.abs(f.cpu().numpy() - f_ref).max() < 1e-8
    # the approximation differs from the exact forces
    assert (f - f_x).abs().max().item() > 1e-4


@pytest.mark.parametrize("variant", ["plain", "lorentz_series_fit"])
def test_box_paper_forces(lm, variant):
    s = inputs.box(110, seed=1, jitter=0.05)
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_force_model(lm.FORCES_PAPER)
    kw = {}
    if variant != "plain":
        model.set_frequency_model(lm.FREQ_LORENTZIAN, 4.0)
        model.set_series_fit(12)
        kw = dict(omega_ref=4.0, lanczos_steps=12)
    e, f = model.energy_forces(*_dev(s), forces=True)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p, **kw))
    e_ref = so.energies()
    f_ref = so.paper_forces()
    assert np.max(np.abs(e.cpu().numpy() - e_ref) / np.abs(e_ref)) < 1e-10
    assert np.abs(f.cpu().numpy() - f_ref).max() < 1e-8
    # memory-bounded waves give the same forces
    st = model.stats()
    mb = lm.LMBD(s.table, p, 12, 6)
    mb.set_force_model(lm.FORCES_PAPER)
    if variant != "plain":
        mb.set_frequency_model(lm.FREQ_LORENTZIAN, 4.0)
        mb.set_series_fit(12)
    mb.set_memory_budget(int(st["bytes_workspace"] - st["bytes_arena"] + 0.1 * st["bytes_arena"]))
    _, f2 = mb.energy_forces(*_dev(s), forces=True)
    assert mb.stats()["waves_mbd"] > 1
    assert (f2 - f).abs().max().item() < 1e-12


def test_force_model_settings(lm):
    s = inputs.cluster(12, seed=2)
    model = lm.LMBD(s.table, lm.default_params(r_scs=4.0, r_mbd1=4.0, r_mbd2=4.0, r_sphere=4.0), 12, 6)
    with pytest.raises(lm.LmbdError) as err:
        model.set_force_model(2)
    assert err.value.status == lm.LMBD_EINVAL


@pytest.mark.parametrize("omega_ref", [None, 4.0])
def test_paper_forces_with_fitted_force_integrand(lm, omega_ref):
    # the paper's fast path end to end (Sec. III.C-D): fitted energy integrand phi and fitted
    # force integrand theta (one reverse pass per sample frequency, then the theta fit)
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_integrand_fit(6)
    kw = dict(fit_nodes=6)
    if omega_ref is not None:
        model.set_frequency_model(lm.FREQ_LORENTZIAN, omega_ref)
        kw["omega_ref"] = omega_ref
    e_x, _ = model.energy_forces(*_dev(s), forces=False)
    model.set_force_model(lm.FORCES_PAPER)
    e, f = model.energy_forces(*_dev(s), forces=True)
    assert torch.equal(e, e_x)
    so = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _op(p, **kw))
    f_ref = so.paper_forces()
    assert np.abs(f.cpu().numpy() - f_ref).max() < 1e-8
    # close to, but not the same as, the quadrature of the force integrand
    mq = lm.LMBD(s.table, p, 12, 6)
    mq.set_force_model(lm.FORCES_PAPER)
    if omega_ref is not None:
        mq.set_frequency_model(lm.FREQ_LORENTZIAN, omega_ref)
    _, fq = mq.energy_forces(*_dev(s), forces=True)
    d = (f - fq).abs().max().item()
    assert 1e-8 < d < 0.1 * fq.abs().max().item()
