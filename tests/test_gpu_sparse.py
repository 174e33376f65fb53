"""Block-sparse T_LR (Sec. III.A, the secondary cutoff r_MBD,2) through the C ABI, against the
oracle and against the dense path.

Tolerances as on the dense path: per-atom energies within 1e-10 relative, forces within
1e-8 eV/Angstrom.  The sparse chain and pair products run in float-float arithmetic; against
the dense path with FP64 products the two agree to 1e-11 relative (energies) and 1e-9 eV/A.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import BOHR_ANGSTROM as BOHR
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


def _op(p, n_freq=12, order=6):
    return oracle.Params(r_scs=p.r_scs, r_mbd1=p.r_mbd1, r_mbd2=p.r_mbd2, r_sphere=p.r_sphere,
                         r_buf=p.r_buf, r_inner=p.r_inner, beta=p.beta, d=p.d, n_freq=n_freq,
                         series_order=order, omega_scale=p.omega_scale)


def _dev(s):
    cell = None if s.cell is None else torch.tensor(s.cell, device="cuda")
    return (torch.tensor(s.positions, device="cuda"), cell,
            torch.tensor(s.species, dtype=torch.int32, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"))


def _model(lm, s, p, sparse, n_freq=12, order=6, fp64=False):
    m = lm.LMBD(s.table, p, n_freq, order)
    if sparse:
        m.set_sparse_tlr(True)
    if fp64:
        m.set_precision(lm.PREC_FP64)
    return m


def _pair_count_bounds(so, p, centres):
    """Coupled site pairs of the given centres by brute force (exact), and the pairs whose
    distance lies within 1e-4 relative above their cutoff (which the FP32 pattern test may
    list as explicit zero blocks)."""
    exact = band = 0
    for k in centres:
        st = so.sites(k)
        x = oracle.site_positions(torch.as_tensor(so.pos), so.cell, st, k)[:st.ns].numpy() * BOHR
        d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
        lower = np.tril(np.ones_like(d, dtype=bool), -1)
        rc = np.full_like(d, p.r_mbd2)
        rc[:, 0] = rc[0, :] = p.r_mbd1
        exact += int(np.sum(lower & (d < rc)))
        band += int(np.sum(lower & (d >= rc) & (d < rc * (1 + 1e-4))))
    return exact, band


# ---------------------------------------------------------------------------------------
# 200-atom periodic box, r_MBD,1 = 6, r_MBD,2 = 3, sphere r_MBD,1 + r_MBD,2 = 9 Angstrom:
# ~300 sites per sphere, ~3 % of the site pairs coupled
# ---------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def box200():
    return inputs.box(200, seed=12, jitter=0.05)


def _p200(lm):
    return lm.default_params(r_scs=3.5, r_mbd1=6.0, r_mbd2=3.0, r_sphere=0.0)


def test_sparse_energies_forces_match_oracle(lm, box200):
    s = box200
    p = _p200(lm)
    rng = np.random.default_rng(3)
    centres = rng.choice(s.n_atoms, 5, replace=False)
    w = np.zeros(s.n_atoms)
    w[centres] = rng.uniform(0.5, 1.5, 5)
    m = _model(lm, s, p, sparse=True)
    e, f = m.energy_forces(*_dev(s), forces=True, weights=torch.tensor(w, device="cuda"))
    e, f = e.cpu().numpy(), f.cpu().numpy()
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(f))
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    e_ref, f_ref = so.energies_forces(centres=centres, weights=w[centres])
    rel = np.abs(e[centres] - e_ref) / np.abs(e_ref)
    assert np.all(rel < E_RTOL), rel.max()
    assert np.abs(f - f_ref).max() < F_ATOL
    # the stored pairs: every coupled pair, plus at most those just beyond a cutoff
    st = m.stats()
    exact, band = _pair_count_bounds(so, p, range(s.n_atoms))
    assert exact <= st["tlr_pairs"] <= exact + band, (st["tlr_pairs"], exact, band)
    ns = m.site_counts(s.n_atoms)[:, 1].astype(np.int64)
    assert st["tlr_pairs"] < 0.15 * np.sum(ns * (ns - 1) // 2)


def test_sparse_matches_dense_every_atom(lm, box200):
    s = box200
    p = _p200(lm)
    args = _dev(s)
    e64, f64 = _model(lm, s, p, sparse=False, fp64=True).energy_forces(*args)
    msp = _model(lm, s, p, sparse=True)
    esp, fsp = msp.energy_forces(*args)
    assert ((esp - e64).abs() / e64.abs()).max().item() < 1e-11
    assert (fsp - f64).abs().max().item() < 1e-9
    # deterministic energies: the same call again, and one launch per atom
    e2, _ = msp.energy_forces(*args)
    assert torch.equal(e2, esp)
    msp.set_launch_mode(lm.LAUNCH_PER_ATOM)
    e3, f3 = msp.energy_forces(*args)
    assert torch.equal(e3, esp)
    assert (f3 - fsp).abs().max().item() < 1e-12


def test_sparse_waves_under_budget_match_single_wave(lm, box200):
    s = box200
    p = _p200(lm)
    args = _dev(s)
    m0 = _model(lm, s, p, sparse=True)
    e0, f0 = m0.energy_forces(*args)
    st = m0.stats()
    whole = st["bytes_workspace"] - st["bytes_arena"]
    mb = _model(lm, s, p, sparse=True)
    mb.set_memory_budget(int(whole + 0.3 * st["bytes_arena"]))
    e, f = mb.energy_forces(*args)
    assert mb.stats()["waves_mbd"] > 1
    assert torch.equal(e, e0)
    assert (f - f0).abs().max().item() < 1e-12


@pytest.mark.parametrize("order,n_freq", [(2, 6), (3, 8), (7, 12)])
def test_sparse_series_orders(lm, order, n_freq):
    s = inputs.box(60, seed=4)
    p = lm.default_params(r_scs=3.0, r_mbd1=5.5, r_mbd2=2.5, r_sphere=0.0)
    m = _model(lm, s, p, sparse=True, n_freq=n_freq, order=order)
    e, f = m.energy_forces(*_dev(s))
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p, n_freq, order))
    centres = [0, 17, 42]
    e_ref = so.energies(centres)
    rel = np.abs(e.cpu().numpy()[centres] - e_ref) / np.abs(e_ref)
    assert np.all(rel < E_RTOL), rel.max()
    e64, f64 = _model(lm, s, p, sparse=False, n_freq=n_freq, order=order, fp64=True).energy_forces(*_dev(s))
    assert (f - f64).abs().max().item() < 1e-9


def test_sparse_central_row_only(lm):
    # r_MBD,2 below the minimum separation: only the central row and column couple
    s = inputs.box(80, seed=8)
    p = lm.default_params(r_scs=3.0, r_mbd1=5.0, r_mbd2=0.8, r_sphere=5.0)
    m = _model(lm, s, p, sparse=True)
    e, _ = m.energy_forces(*_dev(s), forces=True)
    ns = m.site_counts(s.n_atoms)[:, 1].astype(np.int64)
    assert m.stats()["tlr_pairs"] == int(np.sum(ns - 1))
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    centres = [0, 5, 33]
    rel = np.abs(e.cpu().numpy()[centres] - so.energies(centres)) / np.abs(so.energies(centres))
    assert np.all(rel < E_RTOL)


def test_sparse_edge_cases(lm):
    table = np.array([[9.0, 30.0, 3.5], [6.0, 20.0, 3.2]])
    p = lm.default_params(r_scs=4.0, r_mbd1=6.0, r_mbd2=2.0, r_sphere=0.0)
    m = lm.LMBD(table, p, 12, 6)
    m.set_sparse_tlr(True)
    e, f = m.energy_forces(torch.zeros((0, 3), device="cuda", dtype=torch.float64), None,
                           torch.zeros(0, dtype=torch.int32, device="cuda"),
                           torch.zeros(0, device="cuda", dtype=torch.float64))
    assert e.numel() == 0 and f.shape == (0, 3)
    # one atom, two atoms beyond every cutoff (no coupled pair at all): zero energy and force
    for pos in ([[0.0, 0.0, 0.0]], [[0.0, 0.0, 0.0], [0.0, 0.0, 30.0]]):
        n = len(pos)
        e, f = m.energy_forces(torch.tensor(pos, device="cuda", dtype=torch.float64), None,
                               torch.zeros(n, dtype=torch.int32, device="cuda"),
                               torch.full((n,), 0.8, device="cuda", dtype=torch.float64))
        assert torch.all(e == 0) and torch.all(f == 0)
        assert m.stats()["tlr_pairs"] == 0
    # a trimer: the pair (1, 2) lies beyond r_MBD,2, the central pairs within r_MBD,1
    pos = np.array([[0.0, 0.0, 0.0], [3.1, 0.0, 0.0], [0.0, 3.3, 0.4]])
    sp = np.array([0, 1, 0], dtype=np.int32)
    nu = np.array([0.9, 0.7, 0.8])
    e, f = m.energy_forces(torch.tensor(pos, device="cuda"), None, torch.tensor(sp, device="cuda"),
                           torch.tensor(nu, device="cuda"))
    assert m.stats()["tlr_pairs"] == 3 * 2
    so = oracle.System(pos, None, sp, nu, table, _op(p))
    e_ref, f_ref = so.energies_forces()
    assert np.all(np.abs(e.cpu().numpy() - e_ref) / np.abs(e_ref) < E_RTOL)
    assert np.abs(f.cpu().numpy() - f_ref).max() < F_ATOL


def test_sparse_rejects_dense_only_modes(lm, box200):
    s = box200
    p = _p200(lm)
    args = _dev(s)
    for setup, forces in ((lambda m: m.set_log_mode(8), False), (lambda m: m.set_series_fit(8), False),
                          (lambda m: m.set_force_model(lm.FORCES_PAPER), True)):
        m = _model(lm, s, p, sparse=True)
        setup(m)
        with pytest.raises(lm.LmbdError) as ei:
            m.energy_forces(*args, forces=forces)
        assert ei.value.status == lm.LMBD_EUNSUPPORTED
        m.set_sparse_tlr(False)
        m.energy_forces(*args, forces=forces)


def test_sparse_sphere_beyond_the_dense_capacity(lm):
    # sphere r_MBD,1 + r_MBD,2 = 14 Angstrom, ~1150 sites: beyond the dense kernels' 1024
    s = inputs.box(160, seed=21)
    p = lm.default_params(r_scs=3.0, r_mbd1=11.5, r_mbd2=2.5, r_sphere=0.0)
    args = _dev(s)
    with pytest.raises(lm.LmbdError) as ei:
        _model(lm, s, p, sparse=False).energy_forces(*args, forces=False)
    assert ei.value.status == lm.LMBD_ECAPACITY
    m = _model(lm, s, p, sparse=True)
    e, f = m.energy_forces(*args, forces=True)
    assert m.stats()["max_sphere"] > 1024
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    centres = [0, 77]
    e_ref = so.energies(centres)
    rel = np.abs(e.cpu().numpy()[centres] - e_ref) / np.abs(e_ref)
    assert np.all(rel < E_RTOL), rel.max()
    # forces against central differences of the total energy (no site set changes)
    pos = args[0]
    key = m.site_counts(s.n_atoms).copy()
    f = f.cpu().numpy()
    h = 1e-4
    checked = 0
    for a, g in ((3, 0), (50, 1), (120, 2), (7, 1)):
        es = []
        for sgn in (1.0, -1.0):
            pp = pos.clone()
            pp[a, g] += sgn * h
            e1, _ = m.energy_forces(pp, *args[1:], forces=False)
            es.append(e1.sum().item() if np.array_equal(m.site_counts(s.n_atoms), key) else None)
        if None in es:
            continue
        fd = -(es[0] - es[1]) / (2 * h)
        assert abs(fd - f[a, g]) < F_ATOL + 1e-6 * abs(f[a, g]), (a, g, fd, f[a, g])
        checked += 1
    assert checked >= 2


# ---------------------------------------------------------------------------------------
# the bench line's split-cutoff workload at full size: the 4096-atom benchmark box with
# r_MBD,1 = 6, r_MBD,2 = 3 A (sphere 9 A, ~300 sites), every atom against the dense path with
# FP64 products, sampled centres and one one-hot gradient against the oracle
# ---------------------------------------------------------------------------------------
def test_box4096_split_cutoffs_sparse(lm):
    s = inputs.box(4096, seed=0)
    p = lm.default_params(r_mbd1=6.0, r_mbd2=3.0, r_sphere=0.0)
    args = _dev(s)
    msp = _model(lm, s, p, sparse=True)
    esp, fsp = msp.energy_forces(*args)
    counts = msp.site_counts(s.n_atoms)
    e64, f64 = _model(lm, s, p, sparse=False, fp64=True).energy_forces(*args)
    assert ((esp - e64).abs() / e64.abs()).max().item() < 1e-11
    assert (fsp - f64).abs().max().item() < 1e-9
    # oracle centres: the largest |K1| and sphere, and centres within 4 A of the former (their
    # spheres share most of the central polarisabilities the oracle must solve for)
    n1, ns = counts[:, 0], counts[:, 1]
    k0 = int(np.argmax(n1))
    d = s.positions - s.positions[k0]
    box = np.diag(s.cell)
    d -= box * np.round(d / box)
    near = np.argsort((d * d).sum(1))[1:6]
    centres = [k0, int(np.argmax(ns))] + [int(c) for c in near if int(c) != int(np.argmax(ns))]
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    e_ref = so.energies(centres)
    rel = np.abs(esp.cpu().numpy()[centres] - e_ref) / np.abs(e_ref)
    assert np.all(rel < E_RTOL), (rel.max(), centres[int(np.argmax(rel))])
    w = np.zeros(s.n_atoms)
    w[k0] = 1.0
    _, f_ref = so.energies_forces(centres=[k0], weights=np.array([1.0]))
    _, f = msp.energy_forces(*args, forces=True, weights=torch.tensor(w, device="cuda"))
    assert np.abs(f.cpu().numpy() - f_ref).max() < F_ATOL
