"""Continuous batching on the GPU: each result is the same alone and in the mix.

Requests of different sizes (some MD frames of earlier ones) run concurrently on three
library contexts with their own streams, under an HBM cap small enough that the larger
requests run in memory-bounded waves.  Every request is then computed alone on a fresh
context without a budget: per-atom energies must agree bit for bit (same arithmetic in
any wave, on any stream) and forces to rounding (floating-point atomic order).
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


def test_results_same_alone_and_in_the_mix(lm):
    from paper_2407_06409_gb300 import serve
    table, items = inputs.serving_workload(14, rate=50.0, lo=50, hi=700, seed=5)
    assert any(it.frame > 0 for it in items)
    engines = [serve.LmbdEngine(table) for _ in range(3)]
    fp = serve.Footprint(min_wave=64)
    hbm = 4e9
    srv = serve.Server(engines, hbm_bytes=hbm, footprint=fp)
    res = srv.serve(items, realtime=False)
    assert all(r.error is None for r in res), [r.error for r in res if r.error]
    assert srv.peak_accounted <= hbm
    assert any(r.waves != (1, 1) for r in res)
    alone = lm.LMBD(table, lm.default_params(), 12, 6)
    for it, r in zip(items, res):
        s = it.structure
        e, f = alone.energy_forces(s.positions, s.cell, s.species, s.hirshfeld, forces=True)
        assert np.array_equal(e.numpy(), r.energies), it.rid
        assert np.abs(f.numpy() - r.forces).max() < 1e-12, it.rid
    # one small request against the oracle
    small = min(items, key=lambda it: it.structure.n_atoms)
    s = small.structure
    p = lm.default_params()
    so = oracle.System(s.positions, s.cell, s.species, s.hirshfeld, s.table,
                       oracle.Params(r_scs=p.r_scs, r_mbd1=p.r_mbd1, r_mbd2=p.r_mbd2, r_sphere=p.r_sphere,
                                     r_buf=p.r_buf, r_inner=p.r_inner, beta=p.beta, d=p.d, n_freq=12,
                                     series_order=6, omega_scale=p.omega_scale))
    sample = [0, s.n_atoms // 2, s.n_atoms - 1]
    ref = so.energies(sample)
    e_small = res[items.index(small)].energies
    assert np.all(np.abs(e_small[sample] - ref) / np.abs(ref) < 1e-10)
    for e in engines:
        e.close()


def test_realtime_serving_reports_latency(lm):
    from paper_2407_06409_gb300 import serve
    table, items = inputs.serving_workload(24, rate=40.0, lo=50, hi=400, seed=9)
    engines = [serve.LmbdEngine(table) for _ in range(2)]
    srv = serve.Server(engines, hbm_bytes=20e9)
    res = srv.serve(items, realtime=True)
    s = serve.summarize(res)
    assert s["errors"] == 0 and s["requests"] == 24
    assert 0 < s["p50_s"] <= s["p99_s"] < 60
    assert s["atoms_per_s"] > 0
    for e in engines:
        e.close()


def test_resident_site_lists_across_md_frames(lm):
    # frames of one trajectory on one context with a Verlet skin: while no atom has moved by
    # half the skin the site lists are refreshed in place (one atom even crosses the periodic
    # boundary), and every frame's energies equal, bit for bit, those of a fresh context
    base = inputs.box(300, seed=21)
    box = float(base.cell[0, 0])
    pos0 = base.positions.copy()
    pos0[0, 0] = box - 0.004                      # at the boundary: the jitter moves it across
    rng = np.random.default_rng(5)
    frames = [pos0]
    for _ in range(3):
        f = frames[-1] + rng.normal(scale=0.02, size=pos0.shape) * 0.5
        frames.append(f)
    frames[1][0, 0] = box + 0.004                 # crossed (positions are not wrapped)
    frames.append(frames[-1] + 0.2 * rng.normal(size=pos0.shape))   # a large move: search again
    p = lm.default_params()
    res = lm.LMBD(base.table, p, 12, 6)
    res.set_verlet_skin(0.5)
    refreshed = []
    for f in frames:
        s = inputs.Structure(f, base.cell, base.species, base.hirshfeld, base.table)
        e, fo = res.energy_forces(f, base.cell, base.species, base.hirshfeld, forces=True)
        refreshed.append(res.stats()["sites_refreshed"])
        fresh = lm.LMBD(base.table, p, 12, 6)
        e0, f0 = fresh.energy_forces(f, base.cell, base.species, base.hirshfeld, forces=True)
        assert np.array_equal(res.site_counts(s.n_atoms)[:, :3], fresh.site_counts(s.n_atoms)[:, :3])
        assert torch.equal(e, e0)
        assert (fo - f0).abs().max().item() < 1e-12
        fresh.close()
    assert refreshed == [0, 1, 1, 1, 0]
