"""Autotuner for the launch schedule (block size, tile size) of the kernels.

Candidates are timed on the caller's own problem with CUDA events after a
warm-up; the fastest is kept in a JSON cache keyed by the GPU name and a
workload class string, so later runs of the same class skip the search.
Results never depend on the schedule (fixed-order reductions, integer
histograms), only the time does.
"""
from __future__ import annotations

import json
import os
import threading

import torch

_lock = threading.Lock()

BATCH_CANDIDATES = ((128, 1024), (128, 2048), (256, 1024), (256, 2048), (256, 4096),
                    (256, 8192))


def cache_path() -> str:
    base = os.environ.get("QSCATTER_CACHE_DIR") or os.path.join(
        os.path.expanduser("~"), ".cache", "libqscatter")
    return os.path.join(base, "autotune.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def gpu_key() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def time_call(fn, reps: int = 3, warmup: int = 1) -> float:
    """Mean milliseconds of fn() on the current stream."""
    for _ in range(warmup):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune(workload_class: str, candidates, make_runner, reps: int = 3, force: bool = False):
    """Return (best_candidate, {candidate: ms}).  make_runner(candidate) must
    return a zero-argument callable that performs one launch."""
    key = f"{gpu_key()}|{workload_class}"
    with _lock:
        db = _load()
        if not force and key in db:
            return tuple(db[key]["best"]), {tuple(json.loads(k)): v
                                            for k, v in db[key]["ms"].items()}
    times = {}
    for c in candidates:
        fn = make_runner(c)
        times[tuple(c)] = time_call(fn, reps=reps)
    best = min(times, key=times.get)
    with _lock:
        db = _load()
        db[key] = {"best": list(best), "ms": {json.dumps(list(k)): v for k, v in times.items()}}
        _store(db)
    return best, times


def batch_class(batch, n_total: int) -> str:
    return (f"batch|shots={batch.n_shots}|mean={n_total // max(batch.n_shots, 1)}|"
            f"phase={batch.max_phase}|prec={batch.precision}|bins={batch.bins.n_bins}")
