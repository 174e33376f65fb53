"""Host logic of the continuous-batching server, with a fake engine (no GPU).

Checks admission under the HBM cap, the admission window, trajectory affinity, release of
memory held by idle slots, error isolation and the latency summary.
"""
import threading
import time
from dataclasses import dataclass

import numpy as np
import pytest

from paper_2407_06409_gb300 import serve


@dataclass
class _S:
    n_atoms: int


@dataclass
class _Item:
    rid: int
    arrival: float
    structure: _S
    trajectory: int
    frame: int = 0


class FakeEngine:
    """Sleeps in proportion to the size; holds min(budget, full footprint) afterwards."""

    log_lock = threading.Lock()
    running_bytes = [0.0]
    peak_bytes = [0.0]

    def __init__(self, fp, fail_on=None):
        self.fp = fp
        self._held = 0.0
        self.fail_on = fail_on
        self.calls = []

    def run(self, structure, budget):
        n = structure.n_atoms
        with FakeEngine.log_lock:
            FakeEngine.running_bytes[0] += budget
            FakeEngine.peak_bytes[0] = max(FakeEngine.peak_bytes[0], FakeEngine.running_bytes[0])
        self.calls.append((n, budget))
        try:
            time.sleep(0.002 + n * 2e-5)
            if self.fail_on is not None and n == self.fail_on:
                raise RuntimeError("injected failure")
            self._held = min(budget, self.fp.full(n))
            waves = 1 if budget >= self.fp.full(n) else 2
            st = {"bytes_workspace": self._held, "bytes_arena": self._held - n * 1e3, "waves_scs": 1,
                  "waves_mbd": waves}
            return np.full(n, float(n)), np.zeros((n, 3)), st
        finally:
            with FakeEngine.log_lock:
                FakeEngine.running_bytes[0] -= budget

    def held(self):
        return self._held

    def release(self):
        self._held = 0.0


def _server(n_slots, hbm, fail_on=None, window=16, **kw):
    fp = serve.Footprint(per_centre=1e6, per_atom_whole=1e3, fixed=1e6, min_wave=64)
    FakeEngine.running_bytes[0] = 0.0
    FakeEngine.peak_bytes[0] = 0.0
    return serve.Server([FakeEngine(fp, fail_on) for _ in range(n_slots)], hbm_bytes=hbm, footprint=fp,
                        window=window, **kw)


def test_all_served_and_memory_never_exceeds_cap():
    rng = np.random.default_rng(0)
    sizes = np.exp(rng.uniform(np.log(10), np.log(2000), 60)).astype(int)
    items = [_Item(i, 0.0, _S(int(n)), i) for i, n in enumerate(sizes)]
    hbm = 800e6
    srv = _server(4, hbm)
    res = srv.serve(items, realtime=False)
    assert [r.rid for r in res] == list(range(60))
    assert all(r.error is None for r in res)
    assert srv.peak_accounted <= hbm
    assert FakeEngine.peak_bytes[0] <= hbm
    # requests larger than the cap ran with a reduced budget (waves) above their minimum
    # (the footprint model only grows from its initial values as runs are observed)
    fp0 = serve.Footprint(per_centre=1e6, per_atom_whole=1e3, fixed=1e6, min_wave=64)
    for r in res:
        assert fp0.minimum(r.n_atoms) <= r.budget <= srv.fp.full(r.n_atoms)
    assert any(r.waves != (1, 1) for r in res)
    for r in res:
        assert np.all(r.energies == r.n_atoms)


def test_small_requests_pass_a_request_waiting_for_memory():
    # slot 0 runs a large request; a second large one cannot get its minimum at first, and
    # the small ones behind it are admitted on the free slots meanwhile
    items = [_Item(0, 0.0, _S(700), 0), _Item(1, 0.0, _S(700), 1)] + \
            [_Item(i, 0.0, _S(20), i) for i in range(2, 8)]
    srv = _server(3, hbm=600e6)
    res = {r.rid: r for r in srv.serve(items, realtime=False)}
    assert all(r.error is None for r in res.values())
    assert sorted(res[i].admitted for i in range(2, 8))[1] < res[1].admitted
    assert res[0].budget < srv.fp.full(700) and res[1].budget < srv.fp.full(700)


def test_md_frames_follow_their_trajectory_slot():
    items = [_Item(0, 0.0, _S(300), 0, 0), _Item(1, 0.0, _S(200), 1, 0)]
    items += [_Item(2 + k, 0.05 * (k + 1), _S(300), 0, k + 1) for k in range(4)]
    srv = _server(2, hbm=10e9)
    res = {r.rid: r for r in srv.serve(items, realtime=True)}
    base_slot = res[0].slot
    for k in range(4):
        assert res[2 + k].slot == base_slot and res[2 + k].affinity


def test_idle_slots_give_back_memory():
    # two idle slots hold memory from earlier requests; a later request needs it
    items = [_Item(0, 0.0, _S(250), 0), _Item(1, 0.0, _S(250), 1), _Item(2, 0.2, _S(450), 2)]
    srv = _server(3, hbm=600e6)
    res = srv.serve(items, realtime=True)
    assert all(r.error is None for r in res)
    assert srv.releases >= 1
    assert srv.peak_accounted <= 600e6


def test_a_failing_request_does_not_stop_the_others():
    items = [_Item(i, 0.0, _S(n), i) for i, n in enumerate([10, 13, 20, 30])]
    srv = _server(2, hbm=1e9, fail_on=13)
    res = {r.rid: r for r in srv.serve(items, realtime=False)}
    assert res[1].error is not None and "injected" in res[1].error
    assert all(res[i].error is None for i in (0, 2, 3))


def test_summary():
    items = [_Item(i, 0.01 * i, _S(50), i) for i in range(20)]
    srv = _server(2, hbm=1e9)
    res = srv.serve(items, realtime=True)
    s = serve.summarize(res)
    assert s["requests"] == 20 and s["errors"] == 0 and s["atoms"] == 1000
    assert 0 < s["p50_s"] <= s["p99_s"] and s["atoms_per_s"] > 0
    for r in res:
        assert r.done >= r.admitted >= r.arrival - 1e-3


def test_serving_workload_shape():
    from paper_2407_06409_gb300 import inputs
    table, items = inputs.serving_workload(40, rate=50.0, lo=50, hi=400, seed=3)
    assert table.shape == (4, 3)
    arr = np.array([it.arrival for it in items])
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    for it in items:
        assert 50 <= it.structure.n_atoms <= 400
        if it.frame > 0:
            base = items[it.trajectory]
            assert base.frame == 0 and base.rid < it.rid
            d = it.structure.positions - base.structure.positions
            assert 0 < np.abs(d).max() < 0.2
            assert np.array_equal(it.structure.species, base.structure.species)
    assert any(it.frame > 0 for it in items)


def test_size_lanes():
    # large requests (>= 500 atoms) use slot 0 only and never overlap; small ones run beside them
    rng = np.random.default_rng(1)
    sizes = [800, 20, 900, 30, 40, 700, 25, 35, 600, 15, 45, 50]
    items = [_Item(i, 0.0, _S(n), i) for i, n in enumerate(sizes)]
    srv = _server(3, hbm=5e9, large_atoms=500, large_slots=1)
    res = srv.serve(items, realtime=False)
    assert all(r.error is None for r in res)
    large = sorted((r for r in res if r.n_atoms >= 500), key=lambda r: r.admitted)
    assert all(r.slot == 0 for r in large)
    for a, b in zip(large, large[1:]):
        assert b.admitted >= a.done - 1e-6
    small = [r for r in res if r.n_atoms < 500]
    assert any(r.admitted < large[0].done for r in small)
    s = serve.summarize(res, large_atoms=500)
    assert s["below_500_atoms"]["requests"] == 8 and s["from_500_atoms"]["requests"] == 4


def test_lanes_keep_small_requests_out_of_a_large_backlog():
    # a backlog of large requests longer than the admission window; small requests arriving
    # later are served from their own queue while the backlog drains
    items = [_Item(i, 0.0, _S(600), i) for i in range(24)]
    items += [_Item(24 + k, 0.02, _S(30), 24 + k) for k in range(5)]
    srv = _server(3, hbm=5e9, window=4, large_atoms=500, large_slots=1)
    res = {r.rid: r for r in srv.serve(items, realtime=True)}
    assert all(r.error is None for r in res.values())
    last_large = max(res[i].done for i in range(24))
    assert max(res[24 + k].done for k in range(5)) < 0.5 * last_large
