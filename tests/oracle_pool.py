"""Per-sample oracle records of large sample sets, evaluated in chunks by a
pool of host processes (started with spawn, so it is safe after CUDA use).
Each chunk is one call of the oracle's per-sample evaluation; nothing is
computed here beyond splitting and concatenating."""
import multiprocessing as mp
import os

import numpy as np


def _eval_chunk(task):
    laser, beam, bins, xi = task
    import oracle
    return oracle.evaluate(laser, beam, bins, xi)


def host_procs() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def records(laser, beam, bins, xi, chunk=1 << 15, procs=None):
    """oracle.evaluate over all samples of ``xi`` (list of FP64 arrays or None)."""
    n = next(len(a) for a in xi if a is not None)
    tasks = [(laser, beam, bins, [None if a is None else a[o:o + chunk] for a in xi])
             for o in range(0, n, chunk)]
    procs = procs or host_procs()
    with mp.get_context("spawn").Pool(min(procs, len(tasks))) as pool:
        parts = pool.map(_eval_chunk, tasks)
    return np.concatenate(parts)
