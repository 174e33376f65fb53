"""Parity at the benchmark sizes, in the launch configuration bench.py times.

* 4096-atom periodic box (0.1 atoms/A^3, r_SCS 5 A, sphere 7 A, 12 frequencies, n_max 6),
  autotuned SCS buckets, batched launch, sliced tensor-core products: per-atom energies of
  sampled centres against the oracle (the extremes of |K1| and of the sphere, one centre per
  distinct |K1|, the smallest ragged tensor-core tile tails, random ones), and the full gradients
  of four single local energies E_k (forces with one-hot weights) against the oracle's autograd
  gradients (the four oracle gradients in a spawn process pool, oracle_pool).
* 512-atom box with 0.05 A jitter: adjoint forces against central finite differences of the
  GPU energies (h = 1e-4 A, FP64 products so that rounding noise stays far below 1e-8 eV/A),
  sliced against FP64 products, and weighted forces against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle_pool
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


@pytest.fixture(scope="module")
def box4096_run(lm, box4096):
    """The bench configuration: autotuned SCS buckets, batched launch, tcgen05 sliced products."""
    s = box4096
    p = lm.default_params()
    model = lm.LMBD(s.table, p, 12, 6)
    width = model.autotune(*_dev(s))
    e, f = model.energy_forces(*_dev(s), forces=True)
    counts = model.site_counts(s.n_atoms)
    return model, width, e.cpu().numpy(), f.cpu().numpy(), counts


def _sample_centres(s, counts, rng, radius=6.0):
    """Centres that reach the kernels' edge cases: the largest and smallest |K1| (SCS shared
    memory and bucket limits) and sphere (the last, ragged 128-row tcgen05 tile), and, among the
    centres within `radius` of the largest-|K1| centre (so that their spheres share most of the
    central polarisabilities the oracle must evaluate): one centre per distinct |K1| (bucket
    edges of any width), the smallest ragged tails of the 128-row tiles (3 n_s mod 128) and
    random ones."""
    n1, ns = counts[:, 0], counts[:, 1]
    tail = (3 * ns) % 128
    tail[tail == 0] = 128
    k0 = int(np.argmax(n1))
    d = s.positions - s.positions[k0]
    box = np.diag(s.cell)
    d -= box * np.round(d / box)
    near = np.flatnonzero(np.sqrt((d * d).sum(1)) < radius)
    pick = [k0, int(np.argmax(ns)), int(np.argmin(n1)), int(np.argmin(ns))]
    for v in np.unique(n1[near]):
        pick.append(int(near[np.flatnonzero(n1[near] == v)[0]]))
    pick += [int(i) for i in near[np.argsort(tail[near], kind="stable")[:4]]]
    pick += [int(i) for i in rng.choice(near, 6, replace=False)]
    out = []
    for c in pick:
        if c not in out:
            out.append(c)
    return out


def test_box4096_sampled_energies(lm, box4096, box4096_run):
    s = box4096
    p = lm.default_params()
    model, width, e, f, counts = box4096_run
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(f))
    centres = _sample_centres(s, counts, np.random.default_rng(5))
    assert len(centres) >= 32, len(centres)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _op(p))
    # the oracle's own site enumeration agrees with the device lists for every sampled centre
    for c in centres:
        st = so.sites(c)
        assert (st.n1, st.ns, st.n12) == tuple(int(v) for v in counts[c, :3])
    ref = so.energies(centres)
    rel = np.abs(e[centres] - ref) / np.abs(ref)
    assert np.all(rel < E_RTOL), (rel.max(), centres[int(np.argmax(rel))])
    # translation invariance of the total force
    assert np.abs(f.sum(0)).max() < 1e-9


def test_box4096_gradients_of_extreme_local_energies(lm, box4096, box4096_run):
    # one-hot weights: the full gradient of single local energies E_k, for the centres with the
    # largest |K1|, the largest sphere, the smallest ragged tile tail and a middle one
    s = box4096
    p = lm.default_params()
    model, width, _, _, counts = box4096_run
    n1, ns = counts[:, 0], counts[:, 1]
    tail = (3 * ns) % 128
    tail[tail == 0] = 128
    centres = []
    for c in (int(np.argmax(n1)), int(np.argmax(ns)), int(np.argmin(tail)), 2048):
        if c not in centres:
            centres.append(c)
    refs = oracle_pool.gradients(s, _op(p), centres)
    for k, f_ref in zip(centres, refs):
        w = np.zeros(s.n_atoms)
        w[k] = 1.0
        _, f = model.energy_forces(*_dev(s), forces=True, weights=torch.tensor(w, device="cuda"))
        f = f.cpu().numpy()
        assert np.abs(f - f_ref).max() < F_ATOL, k
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
