"""Chunked map over forest pairs, optionally on a spawn-context process pool.

Pair sums are associative, so the oracle may split the pair list into chunks
and add the partial results; the per-pair arithmetic is unchanged.  Pools use
the ``spawn`` start method so that no worker is forked from a process that has
already touched a GPU.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_STATE = {}


def _init(fn, cat, bins, extra):
    _STATE["fn"] = fn
    _STATE["cat"] = cat
    _STATE["bins"] = bins
    _STATE["extra"] = extra


def _run(chunk):
    a, b = chunk
    return _STATE["fn"](_STATE["cat"], _STATE["bins"], a, b, _STATE["extra"])


def map_pairs(fn, cat, bins, a, b, extra=None, processes: int = 1, chunk: int = 2000):
    """Evaluate ``fn(cat, bins, a_chunk, b_chunk, extra)`` over chunks and sum the
    returned dicts of arrays (or scalars)."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    chunks = [(a[i:i + chunk], b[i:i + chunk]) for i in range(0, len(a), chunk)]
    if processes is None or processes <= 0:
        processes = os.cpu_count() or 1
    if processes == 1 or len(chunks) <= 1:
        parts = [fn(cat, bins, ca, cb, extra) for ca, cb in chunks]
    else:
        ctx = mp.get_context("spawn")
        with ctx.Pool(processes, initializer=_init, initargs=(fn, cat, bins, extra)) as pool:
            parts = pool.map(_run, chunks)
    if not parts:
        return fn(cat, bins, a[:0], b[:0], extra)
    total = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in parts[0].items()}
    for p in parts[1:]:
        for k, v in p.items():
            total[k] = total[k] + v
    return total
