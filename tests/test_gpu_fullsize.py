"""Parity at the benchmark sizes, in the launch configuration bench.py times.

* 4096-atom periodic box (0.1 atoms/A^3, r_SCS 5 A, sphere 7 A, 12 frequencies, n_max 6),
  batched launch, sliced tensor-core products: per-atom energies of sampled atoms against the
  oracle, and the full gradient of one sampled local energy E_k (forces with one-hot weights)
  against the oracle's autograd gradient.
* 512-atom box with 0.05 A jitter: adjoint forces against central finite differences of the
  GPU energies (h = 1e-4 A, FP64 products so that rounding noise stays far below 1e-8 eV/A),
  sliced against FP64 products, and weighted forces against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_06409_gb300 import inputs

pytestmark = pytest.mark.gpu

E_RTOL = 1e-10
F_ATOL = 1e-8


@pytest.fixture(scope="module")
def lm():
    from paper_2407_06409_gb300 import build, lmbd
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lmbd


def _op(p):
    return oracle.Params(r_scs=p.r_scs, r_mbd1=p.r_mbd1, r_mbd2=p.r_mbd2, r_sphere=p.r_sphere, r_buf=p.r_buf,
                         r_inner=p.r_inner, beta=p.beta, d=p.d, n_freq=12, series_order=6,
                         omega_scale=p.omega_scale)


def _dev(s):
    return (torch.tensor(s.positions, device="cuda"), torch.tensor(s.cell, device="cuda"),
            torch.tensor(s.species, dtype=torch.int32, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"))


@pytest.fixture(scope="module")
def box4096():
    return inputs.box(4096, seed=0)


def test_box4096_sampled_energies(lm, box4096):
    s = box4096
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    e, f = model.energy_forces(*_dev(s), forces=True)
    e = e.cpu().numpy()
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(f.cpu().numpy()))
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    sample = [0, 1777, 4095]
    ref = so.energies(sample)
    rel = np.abs(e[sample] - ref) / np.abs(ref)
    assert np.all(rel < E_RTOL), rel
    # translation invariance of the total force
    assert np.abs(f.cpu().numpy().sum(0)).max() < 1e-9


def test_box4096_gradient_of_one_local_energy(lm, box4096):
    s = box4096
    p = lm.default_params()
    k = 2048
    w = np.zeros(s.n_atoms)
    w[k] = 1.0
    model = lm.LMBD(s.table, p, 12, 6)
    _, f = model.energy_forces(*_dev(s), forces=True, weights=torch.tensor(w, device="cuda"))
    f = f.cpu().numpy()
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    _, f_ref = so.energies_forces(centres=[k], weights=[1.0])
    assert np.abs(f - f_ref).max() < F_ATOL
    # -dE_k/dR is local: atoms beyond sphere + 2 r_SCS (17 A) feel nothing
    assert np.count_nonzero(np.abs(f).max(1) > 0) < s.n_atoms


@pytest.fixture(scope="module")
def box512():
    return inputs.box(512, seed=3, jitter=0.05)


def _site_key(model, n):
    return model.site_counts(n).copy()


def test_box512_forces_match_finite_differences(lm, box512):
    s = box512
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_precision(lm.PREC_FP64)
    pos, cell, sp, nu = _dev(s)
    e0, f = model.energy_forces(pos, cell, sp, nu, forces=True)
    f = f.cpu().numpy()
    key0 = _site_key(model, s.n_atoms)
    h = 1e-4
    rng = np.random.default_rng(7)
    checked = 0
    for a in rng.choice(s.n_atoms, 12, replace=False):
        for g in range(3):
            es = []
            same = True
            for sgn in (1.0, -1.0):
                pp = pos.clone()
                pp[a, g] += sgn * h
                e, _ = model.energy_forces(pp, cell, sp, nu, forces=False)
                if not np.array_equal(_site_key(model, s.n_atoms), key0):
                    same = False
                es.append(e.sum().item())
            if not same:
                continue
            fd = -(es[0] - es[1]) / (2 * h)
            assert abs(fd - f[a, g]) < F_ATOL + 1e-6 * abs(f[a, g]), (a, g, fd, f[a, g])
            checked += 1
    assert checked >= 24


def test_box512_sliced_products_match_fp64(lm, box512):
    s = box512
    p = lm.default_params()
    args = _dev(s)
    m64 = lm.LMBD(s.table, p, 12, 6)
    m64.set_precision(lm.PREC_FP64)
    e64, f64 = m64.energy_forces(*args)
    msl = lm.LMBD(s.table, p, 12, 6)
    esl, fsl = msl.energy_forces(*args)
    assert ((esl - e64).abs() / e64.abs()).max().item() < E_RTOL
    assert (fsl - f64).abs().max().item() < F_ATOL


def test_box512_weighted_forces_match_oracle(lm, box512):
    s = box512
    p = lm.default_params()
    rng = np.random.default_rng(11)
    centres = rng.choice(s.n_atoms, 4, replace=False)
    w = np.zeros(s.n_atoms)
    w[centres] = rng.uniform(0.5, 1.5, 4)
    model = lm.LMBD(s.table, p, 12, 6)
    e, f = model.energy_forces(*_dev(s), forces=True, weights=torch.tensor(w, device="cuda"))
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    e_ref, f_ref = so.energies_forces(centres=centres, weights=w[centres])
    rel = np.abs(e.cpu().numpy()[centres] - e_ref) / np.abs(e_ref)
    assert np.all(rel < E_RTOL)
    assert np.abs(f.cpu().numpy() - f_ref).max() < F_ATOL


def test_box4096_waves_under_budget_match_single_wave(lm, box4096):
    s = box4096
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    e0, f0 = model.energy_forces(*_dev(s))
    st = model.stats()
    whole = st["bytes_workspace"] - st["bytes_arena"]
    for frac, recompute in ((0.5, 0), (0.12, 1)):
        mb = lm.LMBD(s.table, p, 12, 6)
        mb.set_memory_budget(int(whole + frac * st["bytes_arena"]))
        e, f = mb.energy_forces(*_dev(s))
        sb = mb.stats()
        assert sb["waves_mbd"] > 1 and sb["scs_recomputed"] == recompute
        assert sb["bytes_workspace"] <= whole + frac * st["bytes_arena"]
        assert torch.equal(e, e0)
        assert (f - f0).abs().max().item() < 1e-12
