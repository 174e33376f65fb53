"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances: per-atom energies within 1e-10 relative, forces within 1e-8 eV/Angstrom,
central polarisabilities within 1e-12 relative, site sets exactly.
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


def _oracle_params(p, n_freq=12, order=6):
    return oracle.Params(r_scs=p.r_scs, r_mbd1=p.r_mbd1, r_mbd2=p.r_mbd2, r_sphere=p.r_sphere,
                         r_buf=p.r_buf, r_inner=p.r_inner, beta=p.beta, d=p.d, n_freq=n_freq,
                         series_order=order, omega_scale=p.omega_scale)


def _run(lm, s, p, n_freq=12, order=6, forces=True, weights=None, device="cuda"):
    model = lm.LMBD(s.table, p, n_freq, order)
    pos = torch.tensor(s.positions, device=device)
    cell = None if s.cell is None else torch.tensor(s.cell, device=device)
    sp = torch.tensor(s.species, dtype=torch.int32, device=device)
    nu = torch.tensor(s.hirshfeld, device=device)
    w = None if weights is None else torch.tensor(weights, device=device)
    e, f = model.energy_forces(pos, cell, sp, nu, forces=forces, weights=w)
    return model, e.cpu().numpy(), None if f is None else f.cpu().numpy()


def _check_e(e_gpu, e_ref):
    rel = np.abs(e_gpu - e_ref) / np.maximum(np.abs(e_ref), 1e-300)
    assert np.all(rel < E_RTOL), (rel.max(), np.argmax(rel))


def _check_f(f_gpu, f_ref):
    err = np.abs(f_gpu - f_ref).max()
    assert err < F_ATOL, err


def _gap_ok(s, p):
    """No pair distance within 1e-9 (relative) of a set radius, so both sides agree on sets."""
    radii = [p.r_scs, 2 * p.r_scs, p.r_sphere if p.r_sphere > 0 else p.r_mbd1 + p.r_mbd2]
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _oracle_params(p))
    for k in range(min(s.n_atoms, 8)):
        r = so.sites(k).r_ang.numpy()
        for rc in radii:
            assert np.min(np.abs(r - rc)) > 1e-9 * rc


# ---------------------------------------------------------------------------------------
# 24-atom cluster, cutoff 5 Angstrom (energy only, and with forces)
# ---------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cluster24():
    return inputs.cluster(24, seed=0)


def test_cluster24_energies_polarizabilities_sites(lm, cluster24):
    s = cluster24
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    _gap_ok(s, p)
    model, e, _ = _run(lm, s, p, forces=False)
    so = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _oracle_params(p))
    _check_e(e, so.energies())
    aI = model.central_polarizabilities(s.n_atoms).numpy()
    ref = so.central_alpha(range(s.n_atoms))
    for a in range(s.n_atoms):
        assert np.allclose(aI[a], ref[a].numpy(), rtol=1e-12, atol=0)
    cnt = model.site_counts(s.n_atoms)
    for k in range(s.n_atoms):
        st = so.sites(k)
        assert tuple(cnt[k]) == (st.n1, st.ns, st.n12, len(st.atom))
    om, w = model.quadrature()
    om_ref, w_ref = oracle.quadrature(12, 0.6)
    assert np.allclose(om, om_ref, rtol=1e-14) and np.allclose(w, w_ref, rtol=1e-13)


def test_cluster24_forces(lm, cluster24):
    s = cluster24
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    _, e, f = _run(lm, s, p, forces=True)
    so = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _oracle_params(p))
    e_ref, f_ref = so.energies_forces()
    _check_e(e, e_ref)
    _check_f(f, f_ref)
    assert np.abs(f.sum(0)).max() < 1e-11


# ---------------------------------------------------------------------------------------
# periodic boxes at 0.1 atoms/A^3 with the production cutoffs (r_SCS = 5, sphere 7):
# ~420 sites per atom including periodic images; 3 n1 ~ 160 and 3 ns ~ 435 span
# several 16/64-row tiles with ragged tails
# ---------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def box110():
    return inputs.box(110, seed=1, jitter=0.05)


@pytest.fixture(scope="module")
def box110_ref(box110, lm):
    s = box110
    p = lm.default_params()
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _oracle_params(p))
    e_ref, f_ref = so.energies_forces()
    return so, e_ref, f_ref


def test_box110_energies_and_forces(lm, box110, box110_ref):
    s = box110
    so, e_ref, f_ref = box110_ref
    p = lm.default_params()
    _gap_ok(s, p)
    model, e, f = _run(lm, s, p, forces=True)
    _check_e(e, e_ref)
    _check_f(f, f_ref)
    aI = model.central_polarizabilities(s.n_atoms).numpy()
    ref = so.central_alpha(range(0, s.n_atoms, 9))
    for a, v in ref.items():
        assert np.allclose(aI[a], v.numpy(), rtol=1e-12, atol=0)
    cnt = model.site_counts(s.n_atoms)
    for k in range(0, s.n_atoms, 7):
        st = so.sites(k)
        assert tuple(cnt[k]) == (st.n1, st.ns, st.n12, len(st.atom))
    st = model.stats()
    assert st["max_k1"] >= 40 and st["max_sphere"] >= 120 and st["flops"]["scs"] > 0


def test_box110_weighted_forces_are_vector_jacobian_products(lm, box110):
    s = box110
    p = lm.default_params()
    rng = np.random.default_rng(0)
    w = np.zeros(s.n_atoms)
    w[rng.choice(s.n_atoms, 5, replace=False)] = rng.normal(size=5)
    _, e, f = _run(lm, s, p, forces=True, weights=w)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _oracle_params(p))
    nz = np.nonzero(w)[0]
    _, f_ref = so.energies_forces(centres=nz, weights=w[nz])
    _check_f(f, f_ref)


def test_per_atom_launches_match_batched(lm, box110):
    s = box110
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    args = (torch.tensor(s.positions, device="cuda"), torch.tensor(s.cell, device="cuda"),
            torch.tensor(s.species, dtype=torch.int32, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"))
    e0, f0 = model.energy_forces(*args)
    model.set_launch_mode(lm.LAUNCH_PER_ATOM)
    e1, f1 = model.energy_forces(*args)
    assert torch.equal(e0, e1)
    assert (f0 - f1).abs().max().item() < 1e-12


def test_host_and_device_pointers_agree(lm, box110):
    s = box110
    p = lm.default_params()
    _, e_dev, f_dev = _run(lm, s, p, forces=True)
    model = lm.LMBD(s.table, p, 12, 6)
    e_host, f_host = model.energy_forces(s.positions, s.cell, s.species, s.hirshfeld, forces=True)
    assert np.array_equal(e_host.numpy(), e_dev)
    assert np.abs(f_host.numpy() - f_dev).max() < 1e-12


@pytest.mark.parametrize("order", [2, 3, 5, 7])
def test_series_orders(lm, order):
    s = inputs.box(60, seed=4)
    p = lm.default_params(r_scs=4.0, r_mbd1=5.5, r_mbd2=4.5, r_sphere=6.0)
    _, e, f = _run(lm, s, p, n_freq=8, order=order, forces=True)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _oracle_params(p, 8, order))
    e_ref, f_ref = so.energies_forces()
    _check_e(e, e_ref)
    _check_f(f, f_ref)


def test_paper_default_sphere_r1_plus_r2(lm):
    # r_sphere <= 0 selects the paper's sphere radius r_MBD,1 + r_MBD,2
    s = inputs.box(50, seed=6)
    p = lm.default_params(r_scs=3.0, r_mbd1=3.5, r_mbd2=2.5, r_sphere=0.0)
    _, e, f = _run(lm, s, p, n_freq=6, order=4, forces=True)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _oracle_params(p, 6, 4))
    e_ref, f_ref = so.energies_forces()
    _check_e(e, e_ref)
    _check_f(f, f_ref)


# ---------------------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------------------
def test_empty_and_isolated(lm):
    table = np.array([[6.0, 20.0, 3.2]])
    model = lm.LMBD(table, lm.default_params(), 12, 6)
    e, f = model.energy_forces(torch.zeros((0, 3), device="cuda", dtype=torch.float64), None,
                               torch.zeros(0, dtype=torch.int32, device="cuda"),
                               torch.zeros(0, device="cuda", dtype=torch.float64))
    assert e.numel() == 0 and f.shape == (0, 3)
    # one atom, and two atoms beyond every cutoff: zero energy and force
    for pos in ([[0.0, 0.0, 0.0]], [[0.0, 0.0, 0.0], [0.0, 0.0, 30.0]]):
        n = len(pos)
        e, f = model.energy_forces(torch.tensor(pos, device="cuda", dtype=torch.float64), None,
                                   torch.zeros(n, dtype=torch.int32, device="cuda"),
                                   torch.full((n,), 0.8, device="cuda", dtype=torch.float64))
        assert torch.all(e == 0) and torch.all(f == 0)


def test_dimer_matches_oracle_and_coincident_atoms_rejected(lm):
    table = np.array([[9.0, 30.0, 3.5], [6.0, 20.0, 3.2]])
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 1.1, 1.9]])
    p = lm.default_params(r_scs=3.0, r_mbd1=4.0, r_mbd2=4.0, r_sphere=4.0)
    s = inputs.Structure(pos, None, np.array([0, 1], dtype=np.int32), np.array([0.9, 0.7]), table)
    _, e, f = _run(lm, s, p, forces=True)
    so = oracle.System(pos, None, s.species, s.hirshfeld, table, _oracle_params(p))
    e_ref, f_ref = so.energies_forces()
    _check_e(e, e_ref)
    _check_f(f, f_ref)
    model = lm.LMBD(table, p, 12, 6)
    bad = torch.tensor([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]], device="cuda", dtype=torch.float64)
    with pytest.raises(lm.LmbdError) as ex:
        model.energy_forces(bad, None, torch.zeros(2, dtype=torch.int32, device="cuda"),
                            torch.ones(2, device="cuda", dtype=torch.float64))
    assert ex.value.status == lm.LMBD_EINVAL


def _indefinite_chain():
    """A periodic chain of strongly polarisable atoms 1.4 Angstrom apart (jittered): at omega = 0
    every atom's screening matrix B_K has a negative eigenvalue (polarisation catastrophe,
    Sec. III.A), so the FP32 Cholesky meets a non-positive pivot, while every screened
    polarisability stays positive and the energies are finite."""
    n = 6
    rng = np.random.default_rng(7)
    pos = np.zeros((n, 3))
    pos[:, 2] = 1.4 * np.arange(n)
    pos[:, 0], pos[:, 1] = 1.0, 2.0
    pos += rng.normal(scale=0.03, size=pos.shape)
    cell = np.diag([20.0, 20.0, 1.4 * n])
    table = np.array([[90.0, 30.0, 3.0]])
    return inputs.Structure(pos, cell, np.zeros(n, dtype=np.int32), np.ones(n), table)


def test_indefinite_screening_is_solved_by_the_lu_fallback(lm):
    s = _indefinite_chain()
    p = lm.default_params(r_scs=4.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _oracle_params(p, 4, 4))
    ab, sg, rv, _, _ = so.free()
    for k in range(s.n_atoms):
        st = so.sites(k)
        x = oracle.site_positions(torch.as_tensor(s.positions), s.cell, st, k)
        B = oracle.scs_local(x, st, ab, sg, rv, so.p)[2]
        assert torch.linalg.eigvalsh(B[0]).min().item() < 0          # indefinite at omega = 0
        assert torch.linalg.eigvalsh(B[1:]).min().item() > 0         # definite elsewhere
    e_ref, f_ref = so.energies_forces()
    model, e, f = _run(lm, s, p, n_freq=4, order=4, forces=True)
    assert model.stats()["scs_lu_systems"] == s.n_atoms              # one per atom, at omega = 0
    _check_e(e, e_ref)
    _check_f(f, f_ref)
    a_ref = np.stack([v.numpy() for v in so.central_alpha(range(s.n_atoms)).values()])
    a = model.central_polarizabilities(s.n_atoms).numpy()
    assert np.allclose(a, a_ref, rtol=1e-12, atol=0)
    # the same through the one-launch-per-atom form
    m2 = lm.LMBD(s.table, p, 4, 4)
    m2.set_launch_mode(lm.LAUNCH_PER_ATOM)
    e2, f2 = m2.energy_forces(torch.tensor(s.positions, device="cuda"), torch.tensor(s.cell, device="cuda"),
                              torch.tensor(s.species, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"))
    _check_e(e2.cpu().numpy(), e_ref)
    _check_f(f2.cpu().numpy(), f_ref)


def _strongly_coupled_cluster():
    s = inputs.cluster(10, radius=3.0, min_sep=1.3, n_species=2, seed=2)
    table = np.array([[30.0, 300.0, 1.6], [24.0, 250.0, 1.5]])
    return inputs.Structure(s.positions, None, (s.species % 2).astype(np.int32), np.ones(10), table)


def test_spectral_flags_match_the_oracle(lm):
    # terms (centre, frequency) whose proxy |G^3 e_k|^2 / |G^2 e_k|^2 reaches 1 (Sec. III.A):
    # an integer decided in FP64 on both sides, away from ties (every ratio differs from 1 by
    # more than 5 %), so the counts agree exactly
    s = _strongly_coupled_cluster()
    p = lm.default_params(r_scs=2.5, r_mbd1=6.0, r_mbd2=6.0, r_sphere=6.0)
    so = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _oracle_params(p, 6, 6))
    with torch.no_grad():
        aI = so.central_alpha(range(s.n_atoms))
        ratios = np.array([so.spectral_ratios_of_centre(k, aI) for k in range(s.n_atoms)])
    assert np.min(np.abs(ratios - 1)) > 0.05
    n_ref = int((ratios >= 1).sum())
    assert 0 < n_ref < ratios.size
    model, e, _ = _run(lm, s, p, n_freq=6, order=6, forces=False)
    assert model.stats()["spectral_flags"] == n_ref
    _check_e(e, so.energies())
    # with the check switched on the call reports it and still writes the energies
    model.set_spectral_check(True)
    e2, _ = model.energy_forces(torch.tensor(s.positions, device="cuda"), None,
                                torch.tensor(s.species, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"),
                                forces=False, allow_catastrophe=True)
    assert model.last_status == lm.LMBD_CATASTROPHE
    assert np.array_equal(e2.cpu().numpy(), e)
    # a benign structure raises no flag
    c = inputs.cluster(24, seed=0)
    pc = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    mc, _, _ = _run(lm, c, pc, forces=False)
    assert mc.stats()["spectral_flags"] == 0 and mc.stats()["scs_lu_systems"] == 0


def test_autograd_function(lm, box110):
    s = box110
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    pos = torch.tensor(s.positions, device="cuda", requires_grad=True)
    cell = torch.tensor(s.cell, device="cuda")
    sp = torch.tensor(s.species, dtype=torch.int32, device="cuda")
    nu = torch.tensor(s.hirshfeld, device="cuda")
    e = lm.lmbd_energy(pos, model, cell, sp, nu)
    w = torch.linspace(-1, 2, s.n_atoms, device="cuda", dtype=torch.float64)
    (g,) = torch.autograd.grad((e * w).sum(), pos)
    assert model.stats()["reused_forward"] == 1       # backward ran the reverse sweep alone
    _, f = model.energy_forces(pos.detach(), cell, sp, nu, forces=True, weights=w)
    assert (g + f).abs().max().item() < 1e-13
    e2, _ = model.energy_forces(pos.detach(), cell, sp, nu, forces=False)
    assert torch.equal(e.detach(), e2)


def test_kept_forward_state_falls_back_when_stale(lm, box110):
    s = box110
    model = lm.LMBD(s.table, lm.default_params(), 12, 6)
    pos = torch.tensor(s.positions, device="cuda")
    cell = torch.tensor(s.cell, device="cuda")
    sp = torch.tensor(s.species, dtype=torch.int32, device="cuda")
    nu = torch.tensor(s.hirshfeld, device="cuda")
    w = torch.linspace(0.5, 1.5, s.n_atoms, device="cuda", dtype=torch.float64)
    _, f_ref = model.energy_forces(pos, cell, sp, nu, forces=True, weights=w)
    model.energy_keep(pos, cell, sp, nu)
    f = model.forces_kept(pos, cell, sp, nu, weights=w)
    assert model.stats()["reused_forward"] == 1 and (f - f_ref).abs().max().item() < 1e-12
    # the kept state serves one reverse sweep: a second one is a whole call, same forces
    f2 = model.forces_kept(pos, cell, sp, nu, weights=w)
    assert model.stats()["reused_forward"] == 0 and (f2 - f_ref).abs().max().item() < 1e-12
    # other positions than the kept ones: a whole call for the new positions
    model.energy_keep(pos, cell, sp, nu)
    moved = pos.clone()
    moved[3, 1] += 0.01
    _, f_moved = model.energy_forces(moved, cell, sp, nu, forces=True, weights=w)
    model.energy_keep(pos, cell, sp, nu)
    f3 = model.forces_kept(moved, cell, sp, nu, weights=w)
    assert model.stats()["reused_forward"] == 0 and (f3 - f_moved).abs().max().item() < 1e-12


def test_fp64_product_mode_matches_oracle(lm, box110, box110_ref):
    # the exact FP64 kernels for the two large products stay available and correct
    s = box110
    so, e_ref, f_ref = box110_ref
    model = lm.LMBD(s.table, lm.default_params(), 12, 6)
    model.set_precision(lm.PREC_FP64)
    e, f = model.energy_forces(torch.tensor(s.positions, device="cuda"), torch.tensor(s.cell, device="cuda"),
                               torch.tensor(s.species, dtype=torch.int32, device="cuda"),
                               torch.tensor(s.hirshfeld, device="cuda"))
    _check_e(e.cpu().numpy(), e_ref)
    _check_f(f.cpu().numpy(), f_ref)


def test_device_inputs_out_of_range_are_rejected(lm, cluster24):
    # device-resident inputs are validated by the first kernel: a species index outside the
    # table, a non-finite position or a non-positive Hirshfeld ratio gives LMBD_EINVAL (never
    # an out-of-bounds table read), and the context stays usable afterwards
    s = cluster24
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    model = lm.LMBD(s.table, p, 12, 6)
    pos = torch.tensor(s.positions, device="cuda")
    sp = torch.tensor(s.species, dtype=torch.int32, device="cuda")
    nu = torch.tensor(s.hirshfeld, device="cuda")
    for what in ("species_high", "species_negative", "nan_position", "zero_nu"):
        pos_b, sp_b, nu_b = pos.clone(), sp.clone(), nu.clone()
        if what == "species_high":
            sp_b[5] = len(s.table)
        elif what == "species_negative":
            sp_b[11] = -1
        elif what == "nan_position":
            pos_b[3, 1] = float("nan")
        else:
            nu_b[17] = 0.0
        with pytest.raises(lm.LmbdError) as ex:
            model.energy_forces(pos_b, None, sp_b, nu_b, forces=True)
        assert ex.value.status == lm.LMBD_EINVAL, what
    _, e_ref, f_ref = _run(lm, s, p, forces=True)
    e, f = model.energy_forces(pos, None, sp, nu, forces=True)
    assert np.array_equal(e.cpu().numpy(), e_ref)
    assert np.abs(f.cpu().numpy() - f_ref).max() < 1e-12


def test_site_capacity_grows_for_a_dense_clump(lm):
    # the first site-list capacity comes from the mean density; a dense clump in a dilute
    # periodic box overflows it, and the call must grow the lists and finish (a truncated
    # list is a capacity overflow, not a coincident-atom error)
    rng = np.random.default_rng(11)
    clump = inputs.cluster(200, radius=6.0, min_sep=1.1, n_species=2, seed=11)
    far = rng.uniform(12.0, 38.0, size=(40, 3))
    pos = np.concatenate([clump.positions + 6.0, far])
    keep = [0]
    for i in range(1, len(pos)):
        d = pos[keep] - pos[i]
        d -= 40.0 * np.round(d / 40.0)
        if np.min(np.sum(d * d, axis=1)) > 1.21:
            keep.append(i)
    pos = pos[keep]
    n = len(pos)
    s = inputs.Structure(pos, np.diag([40.0, 40.0, 40.0]), (np.arange(n) % 2).astype(np.int32),
                         rng.uniform(0.6, 1.0, n), clump.table)
    p = lm.default_params(r_scs=4.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    model, e, _ = _run(lm, s, p, n_freq=6, order=4, forces=False)
    st = model.stats()
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _oracle_params(p, 6, 4))
    counts = model.site_counts(n)
    assert st["max_sites"] >= counts[:, 3].max()
    for k in (0, 1, 60, n - 1):
        assert so.sites(k).n1 == counts[k, 0] and so.sites(k).ns == counts[k, 1]
    _check_e(e[[0, 1, 60, n - 1]], so.energies([0, 1, 60, n - 1]))
