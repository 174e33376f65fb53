"""Process pool over central atoms for oracle evaluations of the full-size parity tests.

Test infrastructure only.  The oracle's local problems are independent per central atom, so the
gradients of several single local energies run in worker processes (started with ``spawn``:
never forked from a process that has used the GPU), each running the unchanged oracle with its
share of the host's threads.
"""
from __future__ import annotations

import multiprocessing as mp
import os



def _gradient(args):
    import torch
    pos, cell, species, nu, table, params, k, threads = args
    torch.set_num_threads(threads)
    import oracle
    so = oracle.System(pos, cell, species, nu, table, params)
    return so.energies_forces(centres=[k], weights=[1.0])[1]


def _workers(n):
    return max(1, min(n, os.cpu_count() or 1))


def gradients(s, params, centres):
    """Forces -dE_k/dR of single local energies (one-hot weights), one centre per worker."""
    nw = _workers(len(centres))
    threads = max(1, (os.cpu_count() or 1) // nw)
    jobs = [(s.positions, s.cell, s.species, s.hirshfeld, s.table, params, int(k), threads) for k in centres]
    with mp.get_context("spawn").Pool(nw) as pool:
        return pool.map(_gradient, jobs)
