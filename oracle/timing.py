"""Wall-clock timing of the scalar oracle on the host cores.

TEST INFRASTRUCTURE ONLY: used by bench.py's CPU-baseline and reference legs.  The
oracle runs unchanged; several copies of it run side by side in separate processes
(multiprocessing, "spawn" start method, so that no process is forked from one that
holds a CUDA context), each compressing and decompressing its own independent slabs
of one field.  This module imports numpy and the oracle binding only.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _round_trip(args):
    """One slab: oracle compression and decompression.  Returns (seconds, archive bytes)."""
    path, lo, hi, mode, eb, select = args
    from oracle import oracle as O
    x = np.load(path, mmap_mode="r")
    xs = np.ascontiguousarray(x[lo:hi])
    t0 = time.perf_counter()
    st, ar = O.compress(xs, mode, eb, select=select)
    O.decompress(ar, xs.size)
    return time.perf_counter() - t0, int(ar.size)


def _warm(_):
    from oracle import oracle as O
    O.lib()
    return os.getpid()


def slab_bounds(nrows: int, slabs: int):
    """Split nrows rows (slowest axis) into `slabs` contiguous ranges."""
    edges = np.linspace(0, nrows, slabs + 1).round().astype(int)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def time_slabs(path: str, bounds, mode: int, eb: float, select: int, workers: int):
    """Round trips of every slab (rows [lo, hi) of the .npy field at `path`), spread
    over `workers` processes.  Returns (wall seconds, summed per-slab seconds)."""
    if workers <= 1:
        t0 = time.perf_counter()
        per = [_round_trip((path, lo, hi, mode, eb, select)) for lo, hi in bounds]
        return time.perf_counter() - t0, sum(t for t, _ in per)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_warm, range(workers))  # process start-up and library load, untimed
        t0 = time.perf_counter()
        per = pool.map(_round_trip, [(path, lo, hi, mode, eb, select) for lo, hi in bounds], chunksize=1)
        wall = time.perf_counter() - t0
    return wall, sum(t for t, _ in per)
