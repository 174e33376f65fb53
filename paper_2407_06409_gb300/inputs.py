"""Seeded synthetic inputs for the lMBD hot path.

This module only draws random structures; it holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

Workloads (all numbers from the benchmark configurations of this project):

* ``cluster``: non-periodic cluster, positions uniform in a sphere of radius
  6 Angstrom, minimum separation 1.0 Angstrom, 3 species.
* ``box``: periodic cubic box at 0.1 atoms/Angstrom^3, minimum separation
  1.1 Angstrom (minimum image), 4 species, optional Gaussian jitter.

Species parameters are drawn uniformly: alpha0 in [4, 12] bohr^3,
C6 in [5, 50] Ha bohr^6, R_vdW in [3, 4] bohr; Hirshfeld ratios nu ~ U[0.6, 1].
The random generator is numpy's PCG64 seeded with ``seed``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Structure:
    positions: np.ndarray          # (N, 3) float64, Angstrom
    cell: np.ndarray | None        # (3, 3) float64 rows = lattice vectors, Angstrom; None = cluster
    species: np.ndarray            # (N,) int32
    hirshfeld: np.ndarray          # (N,) float64
    table: np.ndarray              # (S, 3) float64: alpha0 [bohr^3], C6 [Ha bohr^6], R_vdW [bohr]

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])


def species_table(n_species: int, rng: np.random.Generator) -> np.ndarray:
    a0 = rng.uniform(4.0, 12.0, n_species)
    c6 = rng.uniform(5.0, 50.0, n_species)
    r0 = rng.uniform(3.0, 4.0, n_species)
    return np.stack([a0, c6, r0], axis=1).astype(np.float64)


def _rsa_sphere(n: int, radius: float, min_sep: float, rng: np.random.Generator) -> np.ndarray:
    pts: list[np.ndarray] = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > 1000000:
            raise RuntimeError("random sequential addition did not converge")
        p = rng.uniform(-radius, radius, 3)
        if p @ p >= radius * radius:
            continue
        if pts:
            d = np.asarray(pts) - p
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep * min_sep:
                continue
        pts.append(p)
    return np.asarray(pts, dtype=np.float64)


def _rsa_box(n: int, box: float, min_sep: float, rng: np.random.Generator) -> np.ndarray:
    """Random sequential addition in a periodic cube with a cell grid."""
    ncell = max(1, int(box // min_sep))
    h = box / ncell
    grid: dict[tuple[int, int, int], list[int]] = {}
    pts = np.empty((n, 3), dtype=np.float64)
    count = 0
    tries = 0
    ms2 = min_sep * min_sep
    while count < n:
        tries += 1
        if tries > 200 * n + 100000:
            raise RuntimeError("random sequential addition did not converge")
        p = rng.uniform(0.0, box, 3)
        c = tuple(int(v // h) % ncell for v in p)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    cc = ((c[0] + dx) % ncell, (c[1] + dy) % ncell, (c[2] + dz) % ncell)
                    for j in grid.get(cc, ()):
                        d = pts[j] - p
                        d -= box * np.round(d / box)
                        if d @ d < ms2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        pts[count] = p
        grid.setdefault(c, []).append(count)
        count += 1
    return pts


def _resample_box(n: int, box: float, min_sep: float, rng: np.random.Generator) -> np.ndarray:
    """Uniform points in a periodic cube; every point closer than min_sep (minimum image) to a
    point of lower index is drawn again until no such pair is left.  Vectorised with a k-d
    tree, for the large structures of the serving workload."""
    from scipy.spatial import cKDTree
    pts = rng.uniform(0.0, box, (n, 3))
    pairs = cKDTree(pts, boxsize=box).query_pairs(min_sep, output_type="ndarray")
    bad = np.unique(np.max(pairs, axis=1)) if len(pairs) else np.zeros(0, dtype=np.int64)
    # the points outside `bad` have no close pair among themselves; redraw the others until
    # each of them is clear of every point
    for _ in range(1000):
        if len(bad) == 0:
            return pts
        pts[bad] = rng.uniform(0.0, box, (len(bad), 3))
        cnt = cKDTree(pts, boxsize=box).query_ball_point(pts[bad], min_sep, return_length=True)
        bad = bad[cnt > 1]
    raise RuntimeError("resampling did not remove every close pair")


def cluster(n_atoms: int = 24, radius: float = 6.0, min_sep: float = 1.0,
            n_species: int = 3, seed: int = 0) -> Structure:
    rng = np.random.default_rng(seed)
    table = species_table(n_species, rng)
    pos = _rsa_sphere(n_atoms, radius, min_sep, rng)
    species = rng.integers(0, n_species, n_atoms).astype(np.int32)
    nu = rng.uniform(0.6, 1.0, n_atoms)
    return Structure(pos, None, species, nu, table)


def box(n_atoms: int, density: float = 0.1, min_sep: float = 1.1, n_species: int = 4,
        seed: int = 0, jitter: float = 0.0, table: np.ndarray | None = None,
        method: str = "rsa") -> Structure:
    """Periodic cube at the given density.  method "rsa": random sequential addition;
    "resample": draw all points, then redraw those in close pairs (same minimum separation,
    much faster for large N).  table: species parameters to use instead of drawn ones."""
    rng = np.random.default_rng(seed)
    drawn = species_table(n_species, rng)
    if table is None:
        table = drawn
    side = (n_atoms / density) ** (1.0 / 3.0)
    if method == "rsa":
        pos = _rsa_box(n_atoms, side, min_sep, rng)
    elif method == "resample":
        pos = _resample_box(n_atoms, side, min_sep, rng)
    else:
        raise ValueError(method)
    species = rng.integers(0, n_species, n_atoms).astype(np.int32)
    nu = rng.uniform(0.6, 1.0, n_atoms)
    if jitter > 0.0:
        pos = pos + rng.normal(0.0, jitter, pos.shape)
    cell = np.eye(3) * side
    return Structure(pos, cell, species, nu, table)


def md_frame(s: Structure, jitter: float, seed: int) -> Structure:
    """A molecular-dynamics-like snapshot: the same structure with Gaussian noise."""
    rng = np.random.default_rng(seed)
    pos = s.positions + rng.normal(0.0, jitter, s.positions.shape)
    return Structure(pos, None if s.cell is None else s.cell.copy(), s.species.copy(),
                     s.hirshfeld.copy(), s.table.copy())


def serving_sizes(n_requests: int, lo: int = 50, hi: int = 20000, seed: int = 0) -> np.ndarray:
    """Log-uniform structure sizes for the serving workload."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n_requests)).astype(np.int64)


@dataclass
class ServeItem:
    """One request of the serving workload."""
    rid: int
    arrival: float                 # seconds after the start
    structure: Structure
    trajectory: int                # id of the base structure; MD frames share their base's id
    frame: int                     # 0 for a base structure, 1, 2, ... for its MD frames


def serving_workload(n_requests: int = 2000, rate: float = 50.0, lo: int = 50, hi: int = 20000,
                     md_fraction: float = 0.3, jitter: float = 0.02, seed: int = 0,
                     density: float = 0.1) -> tuple[np.ndarray, list[ServeItem]]:
    """Poisson arrivals at `rate` per second; a fraction `md_fraction` of the requests (never
    the first) are MD frames (Gaussian jitter) of an earlier base structure chosen uniformly;
    base structures are periodic boxes with log-uniform sizes in [lo, hi].  One species table
    (4 species) is shared by every request, as one model serves them all."""
    rng = np.random.default_rng(seed)
    table = species_table(4, rng)
    gaps = rng.exponential(1.0 / rate, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = serving_sizes(n_requests, lo, hi, seed=seed + 1)
    is_md = rng.uniform(size=n_requests) < md_fraction
    is_md[0] = False
    items: list[ServeItem] = []
    bases: list[int] = []
    frames: dict[int, int] = {}
    for r in range(n_requests):
        if is_md[r]:
            b = bases[int(rng.integers(len(bases)))]
            frames[b] += 1
            s = md_frame(items[b].structure, jitter, seed=int(rng.integers(1 << 31)))
            items.append(ServeItem(r, float(arrivals[r]), s, items[b].trajectory, frames[b]))
        else:
            s = box(int(sizes[r]), density=density, seed=int(rng.integers(1 << 31)), table=table,
                    method="resample")
            bases.append(r)
            frames[r] = 0
            items.append(ServeItem(r, float(arrivals[r]), s, r, 0))
    return table, items
