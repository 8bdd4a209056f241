"""Sharding a beam over processes (one GPU each) and merging the results.

Samples are independent, so each rank integrates its own shard with
qs_scatter and the small outputs are merged: histograms add exactly (they are
sums of weights), and the moments combine exactly in exact arithmetic --
weighted means for the means, the law of total variance for the spread
(sum over shards of W_r (spread_r^2 + (mean_r - mean)^2) / W) and weighted
second moments for the divergences.  The merge runs in rank order on every
rank, so all ranks hold identical results.  The only collective is one
all-gather of the per-rank outputs (a few KB); there is no data-path
exchange.
"""
from __future__ import annotations

import math

import torch

from .binding import MOMENT_FIELDS

IDX = {k: i for i, k in enumerate(MOMENT_FIELDS)}


def merge_moments(rows) -> list[float]:
    """Merge per-shard qs_moments rows (sequences of 13 floats) in order."""
    W = sum(r[IDX["W"]] for r in rows)
    out = [0.0] * len(MOMENT_FIELDS)
    out[IDX["W"]] = W
    for k in ("under", "over", "map_out", "nonfinite"):
        out[IDX[k]] = sum(r[IDX[k]] for r in rows)
    if W > 0:
        mean = sum(r[IDX["W"]] * r[IDX["mean"]] for r in rows) / W
        var = sum(r[IDX["W"]] * (r[IDX["spread"]] ** 2 + (r[IDX["mean"]] - mean) ** 2)
                  for r in rows) / W
        dx2 = sum(r[IDX["W"]] * r[IDX["div_x"]] ** 2 for r in rows) / W
        dy2 = sum(r[IDX["W"]] * r[IDX["div_y"]] ** 2 for r in rows) / W
        out[IDX["mean"]] = mean
        out[IDX["spread"]] = math.sqrt(max(var, 0.0))
        out[IDX["rel_spread"]] = out[IDX["spread"]] / mean
        out[IDX["div_x"]] = math.sqrt(dx2)
        out[IDX["div_y"]] = math.sqrt(dy2)
        out[IDX["div"]] = math.sqrt(dx2 + dy2)
        out[IDX["mean_aeff"]] = sum(r[IDX["W"]] * r[IDX["mean_aeff"]] for r in rows) / W
        out[IDX["mean_gamma0"]] = sum(r[IDX["W"]] * r[IDX["mean_gamma0"]] for r in rows) / W
    return out


def merge(results: list[dict]) -> dict:
    """Merge per-shard result dicts {moments: list, spectrum, divmap, aeff_hist,
    spec_smooth: tensors} in the given order."""
    out = {"moments": merge_moments([r["moments"] for r in results])}
    for k in ("spectrum", "divmap", "aeff_hist", "spec_smooth"):
        vals = [r[k] for r in results if k in r and r[k] is not None]
        if vals:
            acc = vals[0].detach().double().cpu().clone()
            for v in vals[1:]:
                acc += v.detach().double().cpu()
            out[k] = acc
    return out


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, even (pair-aligned) shard [lo, hi) of n samples for a rank."""
    per = (n + world - 1) // world
    per += per % 2
    lo = min(n, rank * per)
    return lo, min(n, lo + per)


def allgather_merge(local: dict, group=None) -> dict:
    """All-gather each rank's outputs (as one float64 tensor) and merge them
    in rank order; every rank returns the same merged result."""
    import torch.distributed as dist
    keys = [k for k in ("spectrum", "divmap", "aeff_hist", "spec_smooth")
            if local.get(k) is not None]
    parts = [torch.as_tensor(local["moments"], dtype=torch.float64).reshape(-1)]
    parts += [local[k].detach().double().reshape(-1).cpu() for k in keys]
    flat = torch.cat(parts)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    flat = flat.to(dev)
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(flat) for _ in range(world)]
    dist.all_gather(bufs, flat, group=group)
    sizes = [len(MOMENT_FIELDS)] + [local[k].numel() for k in keys]
    results = []
    for b in bufs:
        b = b.cpu()
        chunks = torch.split(b, sizes)
        r = {"moments": chunks[0].tolist()}
        for k, c in zip(keys, chunks[1:]):
            r[k] = c.reshape(local[k].shape)
        results.append(r)
    return merge(results)
