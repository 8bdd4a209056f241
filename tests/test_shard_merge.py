"""Host-side merge of per-shard results (CPU; world-size-2 gloo run).

Each rank integrates its shard with the FP64 oracle (standing in for its
GPU), the small outputs are all-gathered over gloo and merged in rank order;
the merged moments and histograms must equal the oracle over all samples.
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2308_09348_gb300 import inputs as I
from paper_2308_09348_gb300 import shard

KEYS = ("W", "mean", "spread", "rel_spread", "div_x", "div_y", "div", "mean_aeff",
        "under", "over", "map_out", "mean_gamma0")


def _oracle_result(wl, xi, w, lo, hi):
    sub = [a[lo:hi].astype(np.float64) for a in xi]
    r = oracle.scatter(wl.laser, wl.beam, wl.bins, sub, None if w is None else w[lo:hi])
    mom = [r["moments"][k] for k in KEYS] + [0.0]
    return {"moments": mom, "spectrum": torch.from_numpy(r["spectrum"]),
            "divmap": torch.from_numpy(r["divmap"].reshape(-1)),
            "aeff_hist": torch.from_numpy(r["aeff_hist"])}


def _workload(n=3000):
    wl = I.full_qfp(n)
    wl = I.Workload(wl.name, I.Laser(**{**wl.laser.__dict__, "n_phase": 32}), wl.beam, wl.bins,
                    n, wl.seed)
    xi, _ = I.workload_inputs(wl, n)
    w = I.rng(3).uniform(0.5, 1.5, n)
    return wl, xi, w


def _check(merged, ref):
    for i, k in enumerate(KEYS):
        r = ref["moments"][i]
        assert abs(merged["moments"][i] - r) <= 1e-12 * max(abs(r), 1e-300), k
    for k in ("spectrum", "divmap", "aeff_hist"):
        np.testing.assert_allclose(merged[k].numpy(), ref[k].numpy(), rtol=1e-12, atol=1e-12)


def test_merge_of_shards_equals_whole_beam():
    wl, xi, w = _workload()
    n = len(xi[0])
    ref = _oracle_result(wl, xi, w, 0, n)
    for world in (2, 3, 5):
        parts = [_oracle_result(wl, xi, w, *shard.shard_range(n, r, world)) for r in range(world)]
        _check(shard.merge(parts), ref)


def test_merge_with_an_empty_shard():
    wl, xi, w = _workload(500)
    ref = _oracle_result(wl, xi, w, 0, 500)
    parts = [_oracle_result(wl, xi, w, 0, 500)]
    empty = {"moments": [0.0] * 13, "spectrum": torch.zeros_like(parts[0]["spectrum"]),
             "divmap": torch.zeros_like(parts[0]["divmap"]),
             "aeff_hist": torch.zeros_like(parts[0]["aeff_hist"])}
    _check(shard.merge([empty, parts[0], empty]), ref)


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, xi, w = _workload()
        lo, hi = shard.shard_range(len(xi[0]), rank, world)
        merged = shard.allgather_merge(_oracle_result(wl, xi, w, lo, hi))
        q.put((rank, merged["moments"], merged["spectrum"].numpy().tolist()))
    finally:
        dist.destroy_process_group()


def test_gloo_world_size_2_allgather_merge():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl, xi, w = _workload()
    ref = _oracle_result(wl, xi, w, 0, len(xi[0]))
    out.sort()
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]     # identical on both ranks
    merged = {"moments": out[0][1], "spectrum": torch.tensor(out[0][2], dtype=torch.float64),
              "divmap": ref["divmap"], "aeff_hist": ref["aeff_hist"]}
    _check(merged, ref)
