"""Continuous-batching lMBD server over the C ABI.

Structures of any size arrive over time (new structures, and MD frames of earlier ones).
The server keeps a few slots; a slot is one library context with its own CUDA stream and
host thread, so several requests are on the device at once and their kernels overlap.  A
request is admitted as soon as a slot is free and its device-memory reservation fits under
the HBM cap: its full footprint when that fits, otherwise what is left above its minimum,
in which case the library processes its central atoms in memory-bounded waves
(lmbd_set_memory_budget).  Every other idle slot keeps room for a small request, idle
slots give back the memory they hold (least recently used first) before a request is cut
to waves, and admission looks past a request that does not fit to the next ones in
arrival order (a bounded window).  An MD frame goes to the slot that last
served its trajectory when that slot is free: the workspaces there are sized for the
structure and stay resident, so the frame runs without device allocation, and the slot's site
lists (built with a Verlet skin) are refreshed in place instead of searched again while no atom
has moved by half the skin.

Timing is host wall-clock: latency = completion - arrival.
"""
from __future__ import annotations

import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Footprint:
    """Device bytes of a request of n atoms: whole-structure arrays plus the per-centre arena.

    Defaults are for forces at 0.1 atoms/A^3 with r_SCS = 5 A, a 7 A sphere, 12 frequencies
    and n_max = 6 (about 12 MB per central atom); `observe` raises them when a run shows more.
    """
    per_centre: float = 13.0e6
    per_atom_whole: float = 64.0e3
    fixed: float = 256.0e6
    min_wave: int = 512

    def full(self, n: int) -> float:
        return self.fixed + n * (self.per_atom_whole + self.per_centre)

    def minimum(self, n: int) -> float:
        return self.fixed + n * self.per_atom_whole + min(n, self.min_wave) * self.per_centre

    def observe(self, n: int, stats: dict) -> None:
        if n <= 0:
            return
        whole = (stats["bytes_workspace"] - stats["bytes_arena"]) / n
        self.per_atom_whole = max(self.per_atom_whole, whole * 1.05)
        if stats["waves_scs"] == 1 and stats["waves_mbd"] == 1:
            self.per_centre = max(self.per_centre, stats["bytes_arena"] / n)


@dataclass
class Result:
    rid: int
    n_atoms: int
    energies: np.ndarray | None
    forces: np.ndarray | None
    arrival: float
    admitted: float
    done: float
    slot: int
    budget: float
    affinity: bool
    waves: tuple[int, int] = (1, 1)
    error: str | None = None
    sites_refreshed: bool = False   # the slot's resident site lists were refreshed, not rebuilt

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class LmbdEngine:
    """One library context on its own CUDA stream (lower number = higher priority)."""

    def __init__(self, table, params=None, n_freq: int = 12, series_order: int = 6, forces: bool = True,
                 priority: int = 0, skin: float = 0.5):
        import torch
        from . import lmbd
        self.model = lmbd.LMBD(table, params, n_freq, series_order)
        # site lists stay resident across frames of the trajectory this slot serves
        self.model.set_verlet_skin(skin)
        self.stream = torch.cuda.Stream(priority=priority)
        self.forces = forces

    def run(self, structure, budget: float):
        if self.model.held_bytes() > budget:
            self.model.release_workspace()
        self.model.set_memory_budget(int(budget))
        s = structure
        e, f = self.model.energy_forces(s.positions, s.cell, s.species, s.hirshfeld, forces=self.forces,
                                        stream=self.stream)
        return e.numpy(), None if f is None else f.numpy(), self.model.stats()

    def held(self) -> int:
        return self.model.held_bytes()

    def release(self) -> None:
        self.model.release_workspace()

    def close(self) -> None:
        self.model.close()


def make_engines(table, n_slots: int, large_slots: int = 1, **kw) -> list:
    """Engines for a Server: the first `large_slots` on normal-priority streams (the large-request
    lane), the others on the highest-priority streams, so that the blocks of small requests are
    scheduled ahead of those of a large request running beside them."""
    return [LmbdEngine(table, priority=0 if i < large_slots else -8, **kw) for i in range(n_slots)]


@dataclass
class _Slot:
    index: int
    engine: object
    jobs: queue.Queue = field(default_factory=queue.Queue)
    busy: bool = False
    reserved: float = 0.0
    held: float = 0.0
    trajectory: int | None = None
    last_used: float = 0.0
    releasing: bool = False
    thread: threading.Thread | None = None


_RELEASE = object()   # job: free the slot's device memory


class Server:
    def __init__(self, engines: list, hbm_bytes: float = 150e9, footprint: Footprint | None = None,
                 window: int = 16, clock=time.perf_counter, large_atoms: int = 2048, large_slots: int = 1):
        """engines[:large_slots] form the lane for requests of at least `large_atoms` atoms (they
        fill the GPU on their own, so running two at once only splits memory); the other slots
        serve smaller requests, which may borrow an idle large-lane slot while no large request
        waits.  large_slots = 0 (or >= the number of engines) disables lanes."""
        if not engines:
            raise ValueError("at least one engine")
        self.slots = [_Slot(i, e) for i, e in enumerate(engines)]
        self.large_atoms = int(large_atoms)
        self.lanes = 0 < large_slots < len(engines)
        self.large_slots = int(large_slots) if self.lanes else 0
        self._large_waiting = False
        self.hbm = float(hbm_bytes)
        self.fp = footprint if footprint is not None else Footprint()
        self.window = int(window)
        self.clock = clock
        self._cv = threading.Condition()
        self.peak_accounted = 0.0
        self.releases = 0

    # -- memory accounting (caller holds the lock) --------------------------------------------
    def _accounted(self, exclude=None) -> float:
        return sum((s.reserved if s.busy else s.held) for s in self.slots if s is not exclude)

    def _pick_slot(self, item) -> _Slot | None:
        idle = [s for s in self.slots if not s.busy]
        large = item.structure.n_atoms >= self.large_atoms
        if self.lanes:
            lane = [s for s in idle if (s.index < self.large_slots) == large]
            if not lane and not large and not self._large_waiting:
                lane = [s for s in idle if s.index < self.large_slots]
            idle = lane
        if not idle:
            return None
        for s in idle:
            if s.trajectory == item.trajectory:
                return s
        if large:   # reuse the largest resident workspace
            return max(idle, key=lambda s: s.held)
        fresh = [s for s in idle if s.trajectory is None]
        if fresh:
            return fresh[0]
        return min(idle, key=lambda s: s.last_used)

    def _avail(self, slot: _Slot) -> tuple[float, float]:
        """(memory this slot may take, memory not accounted to any other slot).  Every other
        idle slot keeps room for a small request (the full footprint of min_wave atoms), so
        that a large request leaves the other slots usable."""
        free = self.hbm - self._accounted(exclude=slot)
        room = self.fp.full(self.fp.min_wave)
        need = sum(max(0.0, room - s.held) for s in self.slots if not s.busy and s is not slot)
        return free - need, free

    def _admit(self, pending: list, t0: float) -> None:
        # with lanes each lane has its own arrival-order queue and window, so that a backlog of
        # large requests does not hold back small ones (and the other way round)
        self._large_waiting = self.lanes and any(it.structure.n_atoms >= self.large_atoms for it in pending)
        seen = {False: 0, True: 0}
        i = 0
        while i < len(pending):
            item = pending[i]
            cls = self.lanes and item.structure.n_atoms >= self.large_atoms
            if seen[cls] >= self.window:
                if not self.lanes or seen[not cls] >= self.window:
                    return
                i += 1
                continue
            seen[cls] += 1
            slot = self._pick_slot(item)
            if slot is None:
                if not self.lanes:
                    return
                i += 1   # the other lane may still have a free slot
                continue
            n = item.structure.n_atoms
            lo, hi = self.fp.minimum(n), self.fp.full(n)
            avail, free = self._avail(slot)
            if avail < hi:
                # memory held by idle slots is a cache of allocations: have them give it back,
                # least recently used first, before the request is cut to smaller waves.  The
                # slot's own thread frees it; until then it stays accounted.
                coming = sum(s.reserved for s in self.slots if s.releasing)
                for s in sorted((s for s in self.slots if not s.busy and s is not slot and s.held > 0),
                                key=lambda s: s.last_used):
                    if avail + coming >= hi:
                        break
                    s.busy = s.releasing = True
                    s.reserved = s.held
                    coming += s.held
                    self.releases += 1
                    s.jobs.put(_RELEASE)
                if coming > 0:
                    i += 1   # sized once the memory is back; later requests may go first
                    continue
            if avail < lo:
                if any(s.busy for s in self.slots):
                    i += 1
                    continue
                avail = free   # alone on the device: take what there is, the library waves within it
            budget = float(int(min(hi, avail)))   # whole bytes
            pending.pop(i)
            affinity = slot.trajectory == item.trajectory and item.frame > 0
            slot.busy = True
            # what the slot holds stays accounted until its thread has cut it to the budget
            slot.reserved = max(budget, slot.held)
            self.peak_accounted = max(self.peak_accounted, self._accounted())
            slot.jobs.put((item, budget, self.clock() - t0, affinity, self._arrival[item.rid]))

    # -- worker ---------------------------------------------------------------------------------
    def _work(self, slot: _Slot, t0: float, results: dict) -> None:
        while True:
            job = slot.jobs.get()
            if job is None:
                return
            if job is _RELEASE:
                slot.engine.release()
                with self._cv:
                    slot.held = slot.reserved = 0.0
                    slot.trajectory = None
                    slot.busy = slot.releasing = False
                    self._cv.notify_all()
                continue
            item, budget, admitted, affinity, arrival = job
            err, e, f, st = None, None, None, {}
            try:
                if slot.engine.held() > budget:
                    slot.engine.release()
                with self._cv:
                    slot.reserved = budget
                    self._cv.notify_all()
                e, f, st = slot.engine.run(item.structure, budget)
            except Exception as ex:   # reported per request; the slot stays usable
                err = f"{type(ex).__name__}: {ex}"
            done = self.clock() - t0
            with self._cv:
                slot.busy = False
                slot.reserved = 0.0
                slot.held = float(slot.engine.held())
                slot.trajectory = item.trajectory
                slot.last_used = done
                if st:
                    self.fp.observe(item.structure.n_atoms, st)
                results[item.rid] = Result(item.rid, item.structure.n_atoms, e, f, arrival, admitted, done,
                                           slot.index, budget, affinity,
                                           (st.get("waves_scs", 1), st.get("waves_mbd", 1)), err,
                                           bool(st.get("sites_refreshed", 0)))
                self._cv.notify_all()

    def serve(self, items: list, realtime: bool = True) -> list[Result]:
        """Serve every item (with .rid, .arrival, .structure, .trajectory, .frame); arrivals are
        honoured in real time, or all at time 0 when realtime is False."""
        order = sorted(items, key=lambda it: it.arrival)
        self._arrival = {it.rid: (it.arrival if realtime else 0.0) for it in order}
        results: dict = {}
        t0 = self.clock()
        for s in self.slots:
            s.thread = threading.Thread(target=self._work, args=(s, t0, results), daemon=True)
            s.thread.start()
        pending: list = []
        nxt = 0
        try:
            with self._cv:
                while len(results) < len(order):
                    now = self.clock() - t0
                    while nxt < len(order) and (not realtime or order[nxt].arrival <= now):
                        pending.append(order[nxt])
                        nxt += 1
                    self._admit(pending, t0)
                    if len(results) == len(order):
                        break
                    timeout = None
                    if realtime and nxt < len(order):
                        timeout = max(0.0, order[nxt].arrival - (self.clock() - t0))
                    self._cv.wait(timeout if timeout is None else min(timeout, 0.5))
        finally:
            for s in self.slots:
                s.jobs.put(None)
            for s in self.slots:
                s.thread.join()
        return [results[it.rid] for it in items]


def _percentiles(results: list[Result]) -> dict:
    if not results:
        return {"requests": 0}
    lat = np.array([r.latency for r in results])
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean())}


def summarize(results: list[Result], large_atoms: int | None = None) -> dict:
    lat = np.array([r.latency for r in results])
    atoms = sum(r.n_atoms for r in results)
    span = max(r.done for r in results) - min(r.arrival for r in results)
    frames = [r for r in results if r.affinity]
    extra = {}
    if large_atoms is not None:
        extra = {f"below_{large_atoms}_atoms": _percentiles([r for r in results if r.n_atoms < large_atoms]),
                 f"from_{large_atoms}_atoms": _percentiles([r for r in results if r.n_atoms >= large_atoms])}
    return {**extra, 
        "requests": len(results),
        "errors": sum(r.error is not None for r in results),
        "sites_refreshed": sum(r.sites_refreshed for r in results),
        "atoms": int(atoms),
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()),
        "makespan_s": float(span),
        "atoms_per_s": float(atoms / span) if span > 0 else None,
        "waved_requests": sum(1 for r in results if r.waves != (1, 1)),
        "affinity_frames": len(frames),
    }
