"""Log mode of Sec. III.A on the GPU against the oracle's eigendecomposition.

The n_max -> infinity limit of the series, the k-block trace of ln(1 - G) per frequency, from
Lanczos Gauss rules (three start vectors per centre and frequency, implicit QL of the
tridiagonal matrices) on the GPU, and from a full symmetric eigendecomposition in the oracle.
Energies within 1e-10 relative: on a small cluster whose Krylov spaces are exhausted (the
Gauss rules are exact), on a production-size periodic box (3 n_s ~ 435, converged Gauss rules),
and with the Lorentzian frequency model.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_06409_gb300 import inputs

pytestmark = pytest.mark.gpu

E_RTOL = 1e-10


@pytest.fixture(scope="module")
def lm():
    from paper_2407_06409_gb300 import build, lmbd
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lmbd


def _op(p, **kw):
    return oracle.Params(r_scs=p.r_scs, r_mbd1=p.r_mbd1, r_mbd2=p.r_mbd2, r_sphere=p.r_sphere, r_buf=p.r_buf,
                         r_inner=p.r_inner, beta=p.beta, d=p.d, n_freq=12, series_order=None,
                         omega_scale=p.omega_scale, **kw)


def _dev(s):
    cell = None if s.cell is None else torch.tensor(s.cell, device="cuda")
    return (torch.tensor(s.positions, device="cuda"), cell,
            torch.tensor(s.species, dtype=torch.int32, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"))


def test_cluster_log_mode_matches_eigendecomposition(lm):
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_log_mode(64)
    e, _ = model.energy_forces(*_dev(s), forces=False)
    e = e.cpu().numpy()
    so = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _op(p))
    ref = so.energies()
    assert np.max(np.abs(e - ref) / np.abs(ref)) < E_RTOL
    # the log limit differs from the n_max = 6 series (the series is truncated)
    model.set_log_mode(0)
    e6, _ = model.energy_forces(*_dev(s), forces=False)
    assert np.max(np.abs(e6.cpu().numpy() - e) / np.abs(ref)) > 1e-9
    # with the Lorentzian frequency model
    model.set_log_mode(64)
    model.set_frequency_model(lm.FREQ_LORENTZIAN, 6.0)
    el, _ = model.energy_forces(*_dev(s), forces=False)
    refl = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _op(p, omega_ref=6.0)).energies()
    assert np.max(np.abs(el.cpu().numpy() - refl) / np.abs(refl)) < E_RTOL


def test_box_log_mode_at_production_cutoffs(lm):
    s = inputs.box(110, seed=1, jitter=0.05)
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_log_mode(48)
    e, _ = model.energy_forces(*_dev(s), forces=False)
    e = e.cpu().numpy()
    assert model.stats()["max_sphere"] >= 120
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    sample = list(range(0, s.n_atoms, 11))
    ref = so.energies(sample)
    assert np.max(np.abs(e[sample] - ref) / np.abs(ref)) < E_RTOL


def test_log_mode_refuses_forces_and_the_series_fit(lm):
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_log_mode(16)
    with pytest.raises(lm.LmbdError) as ex:
        model.energy_forces(*_dev(s), forces=True)
    assert ex.value.status == lm.LMBD_EUNSUPPORTED
    model.set_series_fit(12)
    with pytest.raises(lm.LmbdError) as ex:
        model.energy_forces(*_dev(s), forces=False)
    assert ex.value.status == lm.LMBD_EINVAL
    with pytest.raises(lm.LmbdError):
        model.set_log_mode(65)
