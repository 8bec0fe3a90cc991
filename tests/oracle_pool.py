"""Oracle work spread over host processes for the large parity cases (test infrastructure).

The pool is started with the 'spawn' method, so no worker is forked from a process that already
holds a CUDA context.  Workers import only numpy and the oracle.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _initial_tour(job):
    import oracle

    xy, cand, params, ant = job
    ref = oracle.Oracle(xy, cand=cand, **params)
    ref.construct(0, ants=np.array([ant], np.int32))
    return ant, ref.newtours[ant].copy(), float(ref.newlen[ant])


def initial_tours(xy, cand, params, ants, workers=None):
    """Initial tours (Algorithm 1, before its iterations) of the listed ants, each built by the
    oracle from scratch in its own process: {ant: (tour, length)}."""
    workers = workers or max(1, min(len(ants), os.cpu_count() or 1))
    jobs = [(xy, cand, dict(params), int(a)) for a in ants]
    with mp.get_context("spawn").Pool(workers) as pool:
        out = pool.map(_initial_tour, jobs)
    return {a: (t, L) for a, t, L in out}
