"""Krylov-chain product on the fifth-generation tensor cores (tcgen05, TMEM accumulators).

The tcgen05 path (lmbd_set_mma_path(LMBD_MMA_TC05)) slices T_LR and W into the same digit
planes as the warp-level mma.sync path and recombines the digit groups exactly, so the two
agree to the last bits (only the FP32 accumulation order of the lowest-order groups differs);
both are checked against the CPU oracle at the stated tolerances (energies 1e-10 relative,
forces 1e-8 eV/Angstrom).  Cases: spheres spanning several 128-row tiles and two K chunks
with ragged tails, one-stage and few-stage K loops (dimer, small cluster), series orders that
use 6- and 5-digit steps, energy-only calls, wave partitions, and the 4096-atom box in the
launch configuration of the benchmark.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_06409_gb300 import inputs

pytestmark = pytest.mark.gpu

E_RTOL = 1e-10
F_ATOL = 1e-8
# agreement of the two tensor-core paths (same digits, same integer recombination)
E_PATH_RTOL = 1e-13
F_PATH_ATOL = 1e-12


@pytest.fixture(scope="module")
def lm():
    from paper_2407_06409_gb300 import build, lmbd
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lmbd


def _args(s):
    cell = None if s.cell is None else torch.tensor(s.cell, device="cuda")
    return (torch.tensor(s.positions, device="cuda"), cell,
            torch.tensor(s.species, dtype=torch.int32, device="cuda"), torch.tensor(s.hirshfeld, device="cuda"))


def _both(lm, s, p, n_freq=12, order=6, forces=True, budget=None):
    out = {}
    for path in (lm.MMA_WARP, lm.MMA_TC05):
        model = lm.LMBD(s.table, p, n_freq, order)
        model.set_mma_path(path)
        if budget is not None:
            model.set_memory_budget(budget)
        e, f = model.energy_forces(*_args(s), forces=forces)
        torch.cuda.synchronize()
        out[path] = (e.cpu().numpy(), None if f is None else f.cpu().numpy(), model.stats())
    return out[lm.MMA_WARP], out[lm.MMA_TC05]


def _same(a, b):
    (ew, fw, _), (et, ft, _) = a, b
    rel = np.abs(et - ew) / np.maximum(np.abs(ew), 1e-300)
    assert rel.max() < E_PATH_RTOL, (rel.max(), np.argmax(rel))
    if fw is not None:
        assert np.abs(ft - fw).max() < F_PATH_ATOL, np.abs(ft - fw).max()


def _oracle_params(p, n_freq=12, order=6):
    return oracle.Params(r_scs=p.r_scs, r_mbd1=p.r_mbd1, r_mbd2=p.r_mbd2, r_sphere=p.r_sphere,
                         r_buf=p.r_buf, r_inner=p.r_inner, beta=p.beta, d=p.d, n_freq=n_freq,
                         series_order=order, omega_scale=p.omega_scale)


def test_tc05_box110_matches_oracle_and_warp_path(lm):
    s = inputs.box(110, seed=1, jitter=0.05)
    p = lm.default_params()
    warp, tc = _both(lm, s, p)
    st = tc[2]
    # spheres of ~120-150 sites: 3 ns > 256, so four 128-row tiles (the last ragged) and two
    # K chunks, the second ragged
    assert 3 * st["max_sphere"] > 256
    _same(warp, tc)
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table, _oracle_params(p))
    e_ref, f_ref = so.energies_forces()
    rel = np.abs(tc[0] - e_ref) / np.abs(e_ref)
    assert rel.max() < E_RTOL, rel.max()
    assert np.abs(tc[1] - f_ref).max() < F_ATOL


@pytest.mark.parametrize("order", [3, 4, 6, 8])
def test_tc05_series_orders_small_spheres(lm, order):
    # 24-atom cluster, 5 Angstrom spheres: a few to ~24 sites (one to three K stages); order 8
    # runs 6-digit and 5-digit chain steps
    s = inputs.cluster(24, seed=0)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    warp, tc = _both(lm, s, p, order=order)
    _same(warp, tc)
    warp, tc = _both(lm, s, p, order=order, forces=False)
    _same(warp, tc)


def test_tc05_dimer_single_stage(lm):
    # two sites: 3 ns = 6, one K stage of 32 with zero fill, one ragged row tile
    s = inputs.Structure(np.array([[0.0, 0.0, 0.0], [3.1, 0.4, -0.2]]), None, np.array([0, 1], dtype=np.int32),
                         np.array([0.8, 0.9]), inputs.cluster(24, seed=0).table)
    p = lm.default_params(r_scs=5.0, r_mbd1=5.0, r_mbd2=5.0, r_sphere=5.0)
    warp, tc = _both(lm, s, p)
    _same(warp, tc)
    so = oracle.System(s.positions, None, s.species, s.hirshfeld, s.table, _oracle_params(p))
    e_ref, f_ref = so.energies_forces()
    assert np.max(np.abs(tc[0] - e_ref) / np.abs(e_ref)) < E_RTOL
    assert np.abs(tc[1] - f_ref).max() < F_ATOL


def test_tc05_waves_match_single_wave(lm):
    s = inputs.box(110, seed=1, jitter=0.05)
    p = lm.default_params()
    warp, tc = _both(lm, s, p)
    st = tc[2]
    whole = st["bytes_workspace"] - st["bytes_arena"]
    _, tcw = _both(lm, s, p, budget=int(whole + 0.15 * st["bytes_arena"]))
    assert tcw[2]["waves_mbd"] > 1
    assert np.array_equal(tcw[0], tc[0])
    assert np.abs(tcw[1] - tc[1]).max() < F_PATH_ATOL


def test_tc05_box4096_matches_warp_path(lm):
    # the benchmark structure in the batched launch configuration
    s = inputs.box(4096, density=0.1, min_sep=1.1, n_species=4, seed=0)
    p = lm.default_params()
    warp, tc = _both(lm, s, p)
    assert 3 * tc[2]["max_sphere"] > 384
    _same(warp, tc)


def test_tc05_wait_that_runs_out_is_reported_and_the_context_recovers(lm):
    # A one-cycle budget makes the first wait for a slot's copies run out (the bulk copies were
    # issued just before it).  The kernels then wait for their own copies and MMAs in flight,
    # free tensor memory and return; the call reports LMBD_ETIMEOUT.  With the default budget the
    # same context gives the results of a fresh one, bit for bit.
    s = inputs.box(110, seed=1, jitter=0.05)
    p = lm.default_params()
    ref = lm.LMBD(s.table, p, 12, 6)
    e0, f0 = ref.energy_forces(*_args(s))
    model = lm.LMBD(s.table, p, 12, 6)
    model.set_wait_budget(1)
    with pytest.raises(lm.LmbdError) as err:
        model.energy_forces(*_args(s))
    assert err.value.status == lm.LMBD_ETIMEOUT
    model.set_wait_budget(0)
    e1, f1 = model.energy_forces(*_args(s))
    assert torch.equal(e1, e0)
    assert (f1 - f0).abs().max().item() < F_PATH_ATOL
    with pytest.raises(lm.LmbdError):
        model.set_wait_budget(-1)
