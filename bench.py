"""Benchmark of the beam phase-space integration (one JSON line on rank 0).

Workload: 2^26 Monte Carlo beam samples (gamma0 = 4000, 10% spread, 3 um x 3 um
x 10 um, 1 mrad), laser a0 = 30, W0 = 2.5 um, 30 fs, 2 um transverse offset,
40 fs delay; quantum-corrected Fokker-Planck model over 512 phase cells;
512-bin spectrum, 128x128 divergence map, 256-bin a_eff histogram; FP32 bulk
arithmetic with FP64 moments.  One step = one qs_scatter call over all
samples.  Inputs (2.1 GB) are larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank integrates its own 2^26 samples (weak scaling, no
data-path collective); rank 0 prints the line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "beam-sample evals/s"
UNIT = "samples/s"

# Arithmetic per phase cell of the QFP integration (FP32 path), counted from
# the model's expression: 2 base-2 logarithms (ln(1+1.7 chi) and that of the
# Gaunt polynomial B), 2 reciprocals (the mean energy, and 1/((1+1.7 chi) D)
# which gives both 1/(1+1.7 chi) and the second-moment fit's 1/D) and 1 base-2
# exponential (B^(-1/3)) on the MUFU pipe, where an ex2 issues at twice the
# rate of lg2/rcp on this GPU (half a slot); and 40 FMA-pipe operations (add,
# mul, fma).
QFP_FMA_OPS_PER_STEP = 40
QFP_MUFU_SLOTS_PER_STEP = 2 + 2 + 1 * 0.5
# The same cell counted from the oracle's expression of the model, evaluated
# as written with loop invariants hoisted and products fused into adds
# (oracle/op_count.py, checked by tests/test_op_count.py): 50 FMA-pipe
# operations and 6.5 MUFU slots.  The kernel reaches the same quantities
# with fewer (one reciprocal of (1 + 1.7 chi) D for both quotients, B' from
# the logarithm already taken, g' from g and B^(-1/3), the 1/gamma state),
# so the roofline against its own 40 is the lower, conservative fraction.
ORACLE_CELL_FMA_OPS = 50
ORACLE_CELL_MUFU_SLOTS = 6.5
QFP_MUFU_MIX = {"lg2": 2, "rcp": 2, "ex2": 1}
FMA_LANES_PER_SM = 128

# Adjoint (packed tangent recursion, FP32): per sample-step 103 FMA-pipe
# operations (the forward step with two tangents carried through mu, chi, the
# Gaunt factor with g' and g'', the second-moment fit with h', and the mean
# and variance updates) and 5 MUFU slots (2 lg2, 2 rcp, 2 ex2).
GRAD_FMA_OPS_PER_STEP = 103
# Photon spectrum (FP32): per (sample, cell, bin) evaluation 20 FMA-pipe
# operations (13 in the packed part of F and the accumulation, 1 saturating
# table coordinate, 6 in the two Horner sums) and 2.5 MUFU slots (rcp, lg2,
# one ex2 at half a slot); the two table gathers (16 bytes each from shared
# memory) took 0.223 shared-memory wavefronts per evaluation in an ncu
# capture of this workload (consecutive log-spaced bins share intervals), at
# one wavefront per SM and clock the pipe that binds.
PHOTON_FMA_OPS_PER_EVAL = 20
PHOTON_MUFU_SLOTS_PER_EVAL = 2.5
PHOTON_SMEM_WAVEFRONTS_PER_EVAL = 0.223
# The bound of the photon kernel: its two 16-byte table reads per evaluation
# against the shared-memory data pipe (fewer wavefronts than bytes / 128 are
# served, 0.223 instead of 0.25 per evaluation, because neighbouring lanes'
# reads of the same entry merge).
PHOTON_TABLE_BYTES_PER_EVAL = 32
SMEM_BYTES_PER_SM_CLOCK = 128
MUFU_SLOTS_PER_SM = 16      # lg2/rcp per SM per clock (measured)

# DRAM traffic of one k_scatter launch on the bench workload from an ncu
# capture, keyed by the hash of the kernel sources it was taken with; any
# other source version reports null.  The capture ran 2^23 samples (read
# and write both grow with the sample count), scaled by 8 to the 2^26 launch.
TRAFFIC_BY_SOURCE = {"12260eabdff95ccd": 8 * (269.31e6 + 2.95e6)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1 << 26, help="samples per rank")
    ap.add_argument("--precision", choices=["f32", "f64"], default="f32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--f64-steps", type=int, default=1, help="timed steps of the FP64 path")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-shots measurement")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient measurement")
    ap.add_argument("--no-broadband", action="store_true",
                    help="skip the broadband single-shot and delay-sweep measurements")
    ap.add_argument("--no-ll", action="store_true", help="skip the classical-model measurement")
    ap.add_argument("--batch-shots", type=int, default=4096)
    ap.add_argument("--grad-n", type=int, default=1 << 24)
    ap.add_argument("--broadband-n", type=int, default=1 << 27)
    ap.add_argument("--ll-n", type=int, default=1 << 26)
    ap.add_argument("--no-cell", action="store_true",
                    help="skip the model-variant measurements (per-cell focus, cycle-resolved chi)")
    ap.add_argument("--cell-n", type=int, default=1 << 24)
    ap.add_argument("--no-photon", action="store_true", help="skip the photon-spectrum measurement")
    ap.add_argument("--photon-n", type=int, default=1 << 19)
    ap.add_argument("--no-pw", action="store_true", help="skip the plane-wave reconstruction")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash() -> str:
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2308_09348_gb300", "csrc", "*.cu*"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    p = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
    except OSError:
        pass
    return p


def cpu_oracle_rate(wl, xi_host, seconds=12.0, chunk=2048):
    """Oracle samples/s on one host core over a bounded prefix of the workload."""
    import numpy as np
    import oracle
    oracle.build()
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and done + chunk <= len(xi_host[0]):
        sub = [a[done:done + chunk].astype(np.float64) for a in xi_host]
        oracle.scatter(wl.laser, wl.beam, wl.bins, sub)
        done += chunk
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def cpu_oracle_gh32():
    """The oracle's full run of the 32^3 Gauss-Hermite grid (classical LL,
    32768 weighted FP64 nodes, 256-bin spectrum) on one host thread."""
    from paper_2308_09348_gb300 import inputs as I
    import oracle
    oracle.build()
    wl = I.tiny_gauss_hermite()
    xi, w = I.workload_inputs(wl)
    oracle.scatter(wl.laser, wl.beam, wl.bins, xi, w)          # warm (page-in, libm)
    t0 = time.perf_counter()
    oracle.scatter(wl.laser, wl.beam, wl.bins, xi, w)
    dt = time.perf_counter() - t0
    return {"value": wl.n / dt, "unit": "samples/s", "cores": 1, "seconds": dt,
            "sample": f"all {wl.n} nodes of the {wl.name} workload (one thread, FP64 C oracle)"}


def cpu_oracle_discretization(wl, xi_host, n=256):
    """Discretisation error of the workload's phase grid: the oracle's
    continuum-accurate mode (n_phase, 2 n_phase, 4 n_phase cells and
    Richardson) on the first n samples, relative to the extrapolated
    continuum (median, 99th percentile and largest over the samples)."""
    import numpy as np
    import oracle
    oracle.build()
    sub = [a[:n].astype(np.float64) for a in xi_host]
    r = oracle.continuum(wl.laser, wl.beam, sub, levels=3)
    out = {"n_phase": r["n_phase"], "grids": r["grids"], "samples": n}
    for f in ("mu", "V"):
        e = r["err_" + f][np.isfinite(r["err_" + f])]
        out["rel_err_" + f] = {"median": float(np.median(e)), "p99": float(np.quantile(e, 0.99)),
                               "max": float(e.max())}
    return out


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_scatter_task(task):
    """One oracle call in a pool worker (the oracle as it stands, FP64 C)."""
    laser, beam, bins, sub = task
    import oracle
    oracle.scatter(laser, beam, bins, sub)
    return len(sub[0])


def oracle_pool(procs):
    """Process pool for the oracle, started with spawn (safe after CUDA use);
    each worker loads the oracle library once before any timing."""
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(procs)
    pool.map(_oracle_warm, range(procs))
    return pool


def _oracle_warm(_):
    import oracle
    oracle.lib()
    return 0


def cpu_oracle_rate_all_cores(wl, xi_host, procs, per_task=2048, seconds=10.0):
    """Oracle samples/s with one process per host core over a bounded prefix
    of the workload (tasks of per_task samples, as many rounds as fit in
    about `seconds`)."""
    import numpy as np
    pool = oracle_pool(procs)
    try:
        n = len(xi_host[0])
        tasks, done = [], 0
        t0 = time.perf_counter()
        while done + per_task * procs <= n and time.perf_counter() - t0 < seconds:
            tasks = [(wl.laser, wl.beam, wl.bins,
                      [a[o:o + per_task].astype(np.float64) for a in xi_host])
                     for o in range(done, done + per_task * procs, per_task)]
            done += sum(pool.map(_oracle_scatter_task, tasks))
        dt = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    return done / dt, done, dt


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, one process per host
    core, each step a bounded sample of the workload."""
    import numpy as np
    from paper_2308_09348_gb300 import inputs as I
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = I.full_qfp(args.n)
    procs = host_cores()
    per_proc = 1024
    per_step = per_proc * procs
    total = per_step * (args.steps + args.warmup)
    xi = I.sample_streams(total, wl.seed, dtype=np.float32)
    import oracle
    oracle.build()
    pool = oracle_pool(procs)
    times = []
    try:
        for s in range(args.warmup + args.steps):
            o0 = s * per_step
            tasks = [(wl.laser, wl.beam, wl.bins,
                      [a[o:o + per_proc].astype(np.float64) for a in xi])
                     for o in range(o0, o0 + per_step, per_proc)]
            t0 = time.perf_counter()
            pool.map(_oracle_scatter_task, tasks)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                times.append(dt)
    finally:
        pool.close()
        pool.join()
    t = sum(times) / len(times)
    v = per_step / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "n_samples_per_step": per_step,
                                             "n_phase": wl.laser.n_phase, "model": "qfp"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"{per_step} samples of the {wl.name} workload per step "
                                       f"({per_proc} per process, {procs} processes)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _fma_peak(dev):
    """FP32 FMA-pipe lane-operations per second at the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * FMA_LANES_PER_SM * float(peaks().get("sm_max_mhz", 2070.0)) * 1e6


def _events(n=2):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def bench_broadband(dev, rank, n, sweep_n=1 << 20, n_delays=512, steps=2):
    """Broadband beam: flat gamma0 on [1e3, 2e4], 2 mrad, 5 um offset, a0 = 100,
    W0 = 2 um, quantum model with 1024 phase cells, 1024 log-spaced bins; and
    the same laser swept over 512 delays on [-100, 100] fs in one batched
    launch over 2^20 shared samples."""
    import numpy as np
    import torch
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import inputs as I
    wl = I.broadband_qfp(n)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl.seed + 7919 * rank)
    xi = [torch.randn(n, generator=gen, device=dev, dtype=torch.float32) for _ in range(8)]
    xi[3] = torch.rand(n, generator=gen, device=dev, dtype=torch.float32)   # flat energy
    out = B.Outputs(wl.bins, n, dev, "f32")
    B.qs_scatter(wl.laser, wl.beam, xi, wl.bins, out=out)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for _ in range(steps):
        B.qs_scatter(wl.laser, wl.beam, xi, wl.bins, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    res = {"metric": "beam-sample evals/s", "value": n / (ms * 1e-3), "unit": "samples/s",
           "ms_per_step": ms, "n_samples": n, "n_phase": wl.laser.n_phase,
           "bins": f"{wl.bins.n_bins} log-spaced", "workload": wl.name}
    # delay sweep over shared samples
    delays = np.linspace(-100.0, 100.0, n_delays)
    lasers = [I.Laser(**{**wl.laser.__dict__, "delay_fs": float(d)}) for d in delays]
    sub = [x[:sweep_n] for x in xi]
    bt = B.Batch(lasers, [wl.beam] * n_delays, None, wl.bins, sweep_n, dev, precision="f32")
    bt.run(sub)
    torch.cuda.synchronize()
    a.record()
    bt.run(sub)
    b.record()
    torch.cuda.synchronize()
    ms2 = a.elapsed_time(b)
    res["delay_sweep"] = {"metric": "shots/s", "value": n_delays / (ms2 * 1e-3), "unit": "shots/s",
                          "sample_evals_per_s": n_delays * sweep_n / (ms2 * 1e-3),
                          "ms_per_launch": ms2, "n_delays": n_delays,
                          "shared_samples": sweep_n, "delay_range_fs": [-100.0, 100.0]}
    return res


def bench_gh32(dev, rank, steps=20):
    """The 32^3 Gauss-Hermite grid (classical LL, 32768 weighted nodes,
    256-bin spectrum, mean and rms energy): one qs_scatter call per step on
    inputs resident in HBM, FP64 and FP32 (launch-bound at this size)."""
    import torch
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import inputs as I
    wl = I.tiny_gauss_hermite()
    xi, w = I.workload_inputs(wl)
    res = {"workload": wl.name, "n_samples": wl.n, "unit": "samples/s"}
    for prec, dt in (("f64", torch.float64), ("f32", torch.float32)):
        xt = [torch.from_numpy(a).to(dev, dt) for a in xi]
        wt = torch.from_numpy(w).to(dev, dt)
        out = B.Outputs(wl.bins, wl.n, dev, prec)
        for _ in range(3):
            B.qs_scatter(wl.laser, wl.beam, xt, wl.bins, w=wt, precision=prec, out=out)
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        for _ in range(steps):
            B.qs_scatter(wl.laser, wl.beam, xt, wl.bins, w=wt, precision=prec, out=out)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        res[prec] = {"value": wl.n / (ms * 1e-3), "ms_per_call": ms}
    return res


def bench_ll(dev, rank, n=1 << 26, steps=5):
    """Classical LL model on the bench beam (HBM-bound: 24 B/sample read)."""
    import torch
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import inputs as I
    wl = I.full_ll(n)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl.seed + 7919 * rank)
    xi = [torch.randn(n, generator=gen, device=dev, dtype=torch.float32) for _ in range(6)]
    out = B.Outputs(wl.bins, n, dev, "f32")
    B.qs_scatter(wl.laser, wl.beam, xi, wl.bins, out=out)
    torch.cuda.synchronize()
    kev = [tuple(_events()) for _ in range(steps)]
    for k in range(steps):
        B.qs_scatter(wl.laser, wl.beam, xi, wl.bins, out=out, kernel_events=kev[k])
    torch.cuda.synchronize()
    kms = sum(x.elapsed_time(y) for x, y in kev) / steps
    gbs = n * 24 / (kms * 1e-3) / 1e9
    pk = peaks().get("hbm_gbs", 6784.5)
    return {"metric": "beam-sample evals/s", "value": n / (kms * 1e-3), "unit": "samples/s",
            "kernel_ms": kms, "n_samples": n, "bytes_per_sample": 24,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk, "unit": "GB/s",
                         "frac": gbs / pk}, "workload": wl.name}


# Per-cell focus adds, per sample-step, the local amplitude of Eq. 2 along
# the path: one rsqrt (a full MUFU slot) and one ex2 (half a slot), and a net
# 14 FMA-pipe operations.
CELL_MUFU_SLOTS_PER_STEP = QFP_MUFU_SLOTS_PER_STEP + 1 + 0.5
# Cycle-resolved chi (FP32): the packed update without the Gaunt and
# second-moment fits (17 packed FMA-pipe instructions per pair of samples: 17
# lane-operations per sample) plus the per-sample table lookup (19 FMA-pipe
# operations: the table coordinate 6, the factor of S 3, G and its
# t-derivative by synthetic division 5, H by Horner 3, S 2) = 36; MUFU: the
# mean-energy reciprocal, the lookup's lg2 and its reciprocal = 3 slots;
# shared memory: two 16-byte reads per sample, 2 x 16 / 128 = 0.25
# wavefronts per sample-step at one 128-byte wavefront per SM and clock.
CYC_FMA_OPS_PER_STEP = 17 + 19
CYC_MUFU_SLOTS_PER_STEP = 3
CYC_SMEM_WAVEFRONTS_PER_STEP = 0.25
CELL_FMA_OPS_PER_STEP = QFP_FMA_OPS_PER_STEP + 14


def bench_variant(dev, rank, variant, n=1 << 24, steps=3):
    """The bench beam and laser with a model variant: Eq. 2 evaluated in
    every phase cell along the electron's path, or the Gaunt and diffusion
    factors averaged over the laser cycle (quantum model, 512 cells, FP32)."""
    import torch
    from dataclasses import replace
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import inputs as I
    wl = I.full_qfp(n)
    L = replace(wl.laser, variant=variant)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl.seed + 7919 * rank)
    xi = [torch.randn(n, generator=gen, device=dev, dtype=torch.float32) for _ in range(8)]
    out = B.Outputs(wl.bins, n, dev, "f32")
    B.qs_scatter(L, wl.beam, xi, wl.bins, out=out)
    torch.cuda.synchronize()
    kev = [tuple(_events()) for _ in range(steps)]
    for k in range(steps):
        B.qs_scatter(L, wl.beam, xi, wl.bins, out=out, kernel_events=kev[k])
    torch.cuda.synchronize()
    kms = sum(x.elapsed_time(y) for x, y in kev) / steps
    props = torch.cuda.get_device_properties(dev)
    fmax = float(peaks().get("sm_max_mhz", 2070.0)) * 1e6
    steps_total = n * L.n_phase
    peak_mufu = props.multi_processor_count * MUFU_SLOTS_PER_SM * fmax
    peak_fma = props.multi_processor_count * FMA_LANES_PER_SM * fmax
    t_mufu = CELL_MUFU_SLOTS_PER_STEP * steps_total / peak_mufu
    t_fma = CELL_FMA_OPS_PER_STEP * steps_total / peak_fma
    t = kms * 1e-3
    line = {"metric": "beam-sample evals/s", "value": n / t, "unit": "samples/s",
            "kernel_ms": kms, "n_samples": n, "n_phase": L.n_phase,
            "workload": wl.name + ("_cellfocus" if variant == I.VAR_CELL_FOCUS else "_cyclechi")}
    if variant == I.VAR_CELL_FOCUS:
        mufu = t_mufu >= t_fma
        ops = (CELL_MUFU_SLOTS_PER_STEP if mufu else CELL_FMA_OPS_PER_STEP) * steps_total
        line["roofline"] = {"bound": "alu", "pipe": "mufu" if mufu else "fma",
                            "achieved": ops / t / 1e12,
                            "peak": (peak_mufu if mufu else peak_fma) / 1e12, "unit": "Top/s",
                            "frac": max(t_mufu, t_fma) / t,
                            "mufu_frac": t_mufu / t, "fma_frac": t_fma / t}
    else:
        # cycle-resolved chi: per sample-step the packed state update and, per
        # sample, the Hermite lookup of (G, H) with S from G's derivative;
        # two 16-byte shared-memory gathers (the node-pair tables), i.e.
        # 0.25 wavefronts of 128 B per sample-step without bank conflicts
        sms = props.multi_processor_count
        t_fma = CYC_FMA_OPS_PER_STEP * steps_total / peak_fma
        t_mufu = CYC_MUFU_SLOTS_PER_STEP * steps_total / peak_mufu
        t_smem = CYC_SMEM_WAVEFRONTS_PER_STEP * steps_total / (sms * fmax)
        pipe = max((t_fma, "fma"), (t_mufu, "mufu"), (t_smem, "smem"))[1]
        line["roofline"] = {"bound": "alu", "pipe": pipe,
                            "achieved": CYC_FMA_OPS_PER_STEP * steps_total / t / 1e12,
                            "peak": peak_fma / 1e12, "unit": "Top/s",
                            "frac": max(t_fma, t_mufu, t_smem) / t,
                            "fma_frac": t_fma / t, "mufu_frac": t_mufu / t,
                            "smem_wavefront_frac": t_smem / t}
    return line


def bench_photon(dev, rank, n=1 << 19, steps=2):
    """Photon spectrum of the bench beam (quantum model, 512 cells): LCFA
    emission of every cell into 256 log-spaced photon-energy bins on
    [1e-3, 6720] m c^2, FP32."""
    import torch
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import inputs as I
    wl = I.full_qfp(n)
    pb = I.Bins(n_bins=256, lo=1e-3, hi=6720.0, log_spaced=1)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl.seed + 7919 * rank)
    xi = [torch.randn(n, generator=gen, device=dev, dtype=torch.float32) for _ in range(8)]
    out = B.qs_photon_spectrum(wl.laser, wl.beam, xi, pb)
    torch.cuda.synchronize()
    kev = [tuple(_events()) for _ in range(steps)]
    for k in range(steps):
        B.qs_photon_spectrum(wl.laser, wl.beam, xi, pb, out=out, kernel_events=kev[k])
    torch.cuda.synchronize()
    kms = sum(x.elapsed_time(y) for x, y in kev) / steps
    evals = n * wl.laser.n_phase * pb.n_bins
    peak = _fma_peak(dev)
    rate = evals / (kms * 1e-3)
    clk = peak / FMA_LANES_PER_SM                    # SM x clock per second
    # shared-memory data pipe: one 128-byte wavefront per SM and clock
    smem_peak = clk * SMEM_BYTES_PER_SM_CLOCK
    return {"metric": "beam-sample evals/s", "value": n / (kms * 1e-3), "unit": "samples/s",
            "kernel_ms": kms, "n_samples": n, "n_phase": wl.laser.n_phase,
            "photon_bins": "256 log-spaced on [1e-3, 6720] m c^2",
            "evaluations_per_s": rate,
            "roofline": {"bound": "smem", "pipe": "shared-memory data pipe (table reads)",
                         "achieved": PHOTON_TABLE_BYTES_PER_EVAL * rate / 1e12,
                         "peak": smem_peak / 1e12, "unit": "TB/s",
                         "frac": PHOTON_TABLE_BYTES_PER_EVAL * rate / smem_peak,
                         "peak_source": "152 SMs x 128 B per clock x 2070 MHz (derived)",
                         "evaluations": evals, "bytes_per_eval": PHOTON_TABLE_BYTES_PER_EVAL,
                         "pipe_fracs": {
                             "shared_memory_bytes": PHOTON_TABLE_BYTES_PER_EVAL * rate / smem_peak,
                             "shared_memory_wavefronts":
                                 PHOTON_SMEM_WAVEFRONTS_PER_EVAL * rate / clk,
                             "fma": PHOTON_FMA_OPS_PER_EVAL * rate / peak,
                             "mufu": PHOTON_MUFU_SLOTS_PER_EVAL * rate / (MUFU_SLOTS_PER_SM * clk)},
                         "fma_ops_per_eval": PHOTON_FMA_OPS_PER_EVAL},
            "workload": "mc2p19_photon_qfp512"}


def bench_pw(dev, rank, n_pw=1 << 20, n_hist=4096, steps=3):
    """Plane-wave reconstruction (Eq. 5): a 61-point plane-wave table (a0
    from 0 to 12 in steps of 0.2, as in Sec. 3.2; quantum model, 512 cells,
    2^20 samples per amplitude, 512 energy bins) from one batched sweep, then
    4096 a_eff histograms contracted with it."""
    import torch
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import inputs as I
    wl = I.full_qfp(n_pw)
    bins = wl.bins
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl.seed + 7919 * rank)
    xi = [torch.randn(n_pw, generator=gen, device=dev, dtype=torch.float32) for _ in range(8)]
    n_a, a_max = 61, 12.2
    hist = torch.rand(n_hist, n_a, generator=gen, device=dev, dtype=torch.float64)
    pw = B.pw_table(wl.laser, wl.beam, bins, n_a, a_max, xi)
    out = B.qs_pw_reconstruct(hist, pw)
    torch.cuda.synchronize()
    a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t_t = t_r = 0.0
    for _ in range(steps):
        a.record()
        pw = B.pw_table(wl.laser, wl.beam, bins, n_a, a_max, xi)
        m.record()
        B.qs_pw_reconstruct(hist, pw, out=out)
        b.record()
        torch.cuda.synchronize()
        t_t += a.elapsed_time(m)
        t_r += m.elapsed_time(b)
    t_t /= steps
    t_r /= steps
    return {"metric": "plane-wave table + reconstruction ms", "value": t_t + t_r, "unit": "ms",
            "table_ms": t_t, "reconstruct_ms": t_r, "n_amplitudes": n_a,
            "samples_per_amplitude": n_pw, "n_histograms": n_hist, "energy_bins": bins.n_bins,
            "table_sample_evals_per_s": n_a * n_pw / (t_t * 1e-3),
            "workload": "pw61_2p20_qfp512_x4096"}


def bench_batch(dev, rank, steps=3, n_shots=4096):
    """4096 shots, sample counts log-uniform in [1e3, 1e6], per-shot laser and
    beam drawn from seed, quantum model with 512 phase cells, FP32 with FP64
    moments, one persistent launch per step; schedule from the autotuner.
    Beside it the same shots with the classical and quantum models
    alternating (``mixed_models``)."""
    import torch
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import inputs as I
    from paper_2308_09348_gb300 import tune
    bw = I.batch_shots(n_shots)
    n = int(bw.offsets[-1])
    gen = torch.Generator(device=dev)
    gen.manual_seed(bw.seed + 7919 * rank)
    xi = [torch.randn(n, generator=gen, device=dev, dtype=torch.float32) for _ in range(8)]

    def runner(c):
        bt = B.Batch(bw.lasers, bw.beams, bw.offsets, bw.bins, n, dev, ranges=bw.ranges,
                     precision="f32", block=c[0], tile=c[1])
        return lambda: bt.run(xi)

    probe = B.Batch(bw.lasers, bw.beams, bw.offsets, bw.bins, n, dev, ranges=bw.ranges,
                    precision="f32")
    best, times = tune.tune(tune.batch_class(probe, n), tune.BATCH_CANDIDATES, runner, reps=1)
    del probe
    bt = B.Batch(bw.lasers, bw.beams, bw.offsets, bw.bins, n, dev, ranges=bw.ranges,
                 precision="f32", block=best[0], tile=best[1])
    bt.run(xi)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        bt.run(xi)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    bad = int((bt.moments[:, B.MOMENT_FIELDS.index("nonfinite")] != 0).sum())
    del bt
    # the same shots and samples with the models alternating (even shots
    # quantum, odd shots classical) in one launch, same schedule
    bm = I.batch_shots(n_shots, model_mix=True)
    btm = B.Batch(bm.lasers, bm.beams, bm.offsets, bm.bins, n, dev, ranges=bm.ranges,
                  precision="f32", block=best[0], tile=best[1])
    btm.run(xi)
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        btm.run(xi)
    b.record()
    torch.cuda.synchronize()
    ms_mix = a.elapsed_time(b) / steps
    bad_mix = int((btm.moments[:, B.MOMENT_FIELDS.index("nonfinite")] != 0).sum())
    del btm
    return {"metric": "shots/s", "value": n_shots / (ms * 1e-3), "unit": "shots/s",
            "samples_per_s": n / (ms * 1e-3), "ms_per_step": ms, "steps": steps,
            "n_shots": n_shots, "n_samples": n, "n_phase": 512, "schedule": {"block": best[0],
                                                                             "tile": best[1]},
            "tuned_ms": {f"{k[0]}x{k[1]}": v for k, v in times.items()},
            "shots_flagged": bad, "workload": bw.name,
            "mixed_models": {"value": n_shots / (ms_mix * 1e-3), "unit": "shots/s",
                             "samples_per_s": n / (ms_mix * 1e-3), "ms_per_step": ms_mix,
                             "shots_flagged": bad_mix,
                             "models": "even shots quantum (512 cells), odd shots classical"}}


def bench_grad(dev, rank, steps=3, n=1 << 24):
    """Forward + adjoint of 2^24 FP32 samples (quantum model, 512 cells) with a
    loss on the moments and the 2-bin-smoothed 256-bin spectrum."""
    import torch
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import inputs as I
    wl = I.fit_qfp(n)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl.seed + 7919 * rank)
    xi = [torch.randn(n, generator=gen, device=dev, dtype=torch.float32) for _ in range(8)]
    out = B.Outputs(wl.bins, n, dev, "f32")
    dm = torch.zeros(13, dtype=torch.float64, device=dev)
    dm[1] = 1e-3
    dm[2] = 1e-3
    dm[4] = 1e3
    dS = torch.full((wl.bins.n_bins,), 1e-3, dtype=torch.float64, device=dev)

    def fwd_bwd():
        B.qs_scatter(wl.laser, wl.beam, xi, wl.bins, precision="f32", out=out)
        return B.qs_scatter_grad(wl.laser, wl.beam, xi, wl.bins, out.moments, dm, dS,
                                 precision="f32", out=out)

    fwd_bwd()
    torch.cuda.synchronize()
    a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t_f = t_b = 0.0
    for _ in range(steps):
        a.record()
        B.qs_scatter(wl.laser, wl.beam, xi, wl.bins, precision="f32", out=out)
        m.record()
        B.qs_scatter_grad(wl.laser, wl.beam, xi, wl.bins, out.moments, dm, dS, precision="f32",
                          out=out)
        b.record()
        torch.cuda.synchronize()
        t_f += a.elapsed_time(m)
        t_b += m.elapsed_time(b)
    t_f /= steps
    t_b /= steps
    steps_total = n * wl.laser.n_phase
    peak = _fma_peak(dev)
    return {"metric": "grad evals/s", "value": n / ((t_f + t_b) * 1e-3), "unit": "samples/s",
            "forward_ms": t_f, "adjoint_ms": t_b, "n_samples": n, "n_phase": wl.laser.n_phase,
            "roofline": {"kernel": "k_grad<float>", "bound": "alu", "pipe": "fma",
                         "achieved": GRAD_FMA_OPS_PER_STEP * steps_total / (t_b * 1e-3) / 1e12,
                         "peak": peak / 1e12, "unit": "Top/s",
                         "frac": GRAD_FMA_OPS_PER_STEP * steps_total / peak / (t_b * 1e-3)},
            "workload": wl.name}


def bench_fit256(dev, rank, steps=10, n_shots=256, per=1 << 16):
    """The batched gradient fit of the reconstruction use: 256 shots of 2^16
    FP32 samples each (2^24 in all), hidden parameters drawn from the batched
    configuration's ranges (a0 U[5,50], W0 U[2,10] um, offsets N(0,2) um,
    delay N(0,30) fs, gamma_mean U[1e3,2e4], spread U[0.01,0.2], 1 mrad),
    quantum model over 512 cells, loss on the moments and the 2-bin-smoothed
    256-bin spectrum of every shot; perturbed starts; Adam.  Timed: whole
    Adam steps (batched forward, batched adjoint, loss, update), and the two
    batched kernels alone."""
    import numpy as np
    import torch
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import fit as F
    from paper_2308_09348_gb300 import inputs as I
    g = I.rng(0x23080904 + rank)
    a0, w0 = g.uniform(5, 50, n_shots), g.uniform(2, 10, n_shots)
    dx, dy, delay = g.normal(0, 2, n_shots), g.normal(0, 2, n_shots), g.normal(0, 30, n_shots)
    gm, sp = g.uniform(1e3, 2e4, n_shots), g.uniform(0.01, 0.2, n_shots)
    lasers = [I.Laser(lambda_um=0.8, a0=a0[k], w0_um=w0[k], tau_fs=30.0, model=I.MODEL_QFP,
                      dx_um=dx[k], dy_um=dy[k], delay_fs=delay[k], n_phase=512)
              for k in range(n_shots)]
    beams = [I.Beam(gamma_mean=gm[k], rel_spread=sp[k], sigma_x_um=3.0, sigma_y_um=3.0,
                    sigma_z_um=10.0, div_rad=1e-3) for k in range(n_shots)]
    ranges = np.array([[0.0, 1.2 * gm[k] * (1 + 4 * sp[k])] for k in range(n_shots)])
    bins = I.Bins(n_bins=256, lo=0.0, hi=1.0, smooth_sigma_bins=2.0)
    n = n_shots * per
    gen = torch.Generator(device=dev)
    gen.manual_seed(0x23080904 + 7919 * rank)
    xi = [torch.randn(n, generator=gen, device=dev, dtype=torch.float32) for _ in range(8)]
    offsets = np.arange(n_shots + 1, dtype=np.int64) * per
    bt = B.Batch(lasers, beams, offsets, bins, n, dev, ranges=ranges, precision="f32")
    prob = F.BatchProblem(bt, xi)
    hidden = bt.params().clone()
    with torch.no_grad():
        tm, tS = F.BatchScatterFn.apply(hidden, prob)
        tm, tS = tm.clone(), tS.clone()
    pert = torch.from_numpy(I.rng(77).normal(size=(n_shots, 8))).to(dev).clamp(-2, 2)
    rel = torch.tensor([0.1, 0.1, 0, 0, 0, 0.05, 0.2, 0.2], dtype=torch.float64, device=dev)
    absd = torch.tensor([0, 0, 0.3, 0.3, 5.0, 0, 0, 0], dtype=torch.float64, device=dev)
    start = hidden * (1 + rel * pert) + absd * pert
    scale = torch.tensor([20.0, 4.0, 2.0, 2.0, 30.0, 6000.0, 0.05, 1e-3], dtype=torch.float64,
                         device=dev)
    F.fit_batch(prob, start, tm, tS, steps=2, lr=0.03, scale=scale)        # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    th, hist, last = F.fit_batch(prob, start, tm, tS, steps=steps, lr=0.03, scale=scale)
    b.record()
    torch.cuda.synchronize()
    ms_step = a.elapsed_time(b) / steps
    # the batched kernels alone (forward at the start, adjoint of a loss)
    bt.set_params(start)
    dm = torch.zeros(n_shots, 13, dtype=torch.float64, device=dev)
    dm[:, 1] = 1e-3
    dS = torch.full((n_shots, 256), 1e-3, dtype=torch.float64, device=dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_f = t_b = 0.0
    for _ in range(3):
        e[0].record()
        bt.run(xi)
        e[1].record()
        bt.grad(xi, dm, dS)
        e[2].record()
        torch.cuda.synchronize()
        t_f += e[0].elapsed_time(e[1]) / 3
        t_b += e[1].elapsed_time(e[2]) / 3
    steps_total = n * 512
    peak = _fma_peak(dev)
    return {"metric": "fit shots/s", "value": n_shots / (ms_step * 1e-3), "unit": "shot-steps/s",
            "ms_per_adam_step": ms_step, "n_shots": n_shots, "samples_per_shot": per,
            "n_phase": 512, "steps": steps, "loss_first_last": [hist[0], hist[-1]],
            "batched_forward_ms": t_f, "batched_adjoint_ms": t_b,
            "grad_samples_per_s": n / ((t_f + t_b) * 1e-3),
            "adjoint_roofline": {"kernel": "k_bgrad<float>", "bound": "alu", "pipe": "fma",
                                 "frac": GRAD_FMA_OPS_PER_STEP * steps_total / peak / (t_b * 1e-3)},
            "workload": "fit256_2p16_qfp512"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2308_09348_gb300 import inputs as I
    from paper_2308_09348_gb300 import binding as B
    from paper_2308_09348_gb300 import build as _build

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    if rank == 0 or ws == 1:
        _build.build()
    if ws > 1:
        dist.barrier()

    wl = I.full_qfp(args.n)
    n = args.n
    dev = torch.device("cuda", local)
    # seeded synthetic variates, generated on the device (rank-dependent seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(wl.seed + 7919 * rank)
    xi = [torch.randn(n, generator=gen, device=dev, dtype=torch.float32) for _ in range(8)]
    stream = torch.cuda.current_stream()
    out = B.Outputs(wl.bins, n, dev, args.precision)

    def step(events=None, precision=args.precision, o=out, streams=xi):
        B.qs_scatter(wl.laser, wl.beam, streams, wl.bins, precision=precision, out=o,
                     kernel_events=events)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- device-resident timed region ------------------------------------
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local)
    clk.start()
    time.sleep(1.0)            # nvidia-smi starts before the timed steps
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(args.steps):
        step(kev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = t0.elapsed_time(t1) / args.steps
    kern_ms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = n * ws / (ms * 1e-3)

    # ---- end to end through the public API with host buffers --------------
    # qs_scatter_host: pinned host samples streamed in double-buffered chunks
    # (copy of chunk c+1 overlaps the kernel on chunk c), results read back to
    # pinned host memory; timed on the device with events, synchronised,
    # right after the device-resident steps and with its own clock record.
    e2e = None
    if not args.no_e2e:
        host = [x.cpu().pin_memory() for x in xi]
        hout = B.HostOutputs(wl.bins, host, None, 0, args.precision, dev)
        h2d = sum(h.numel() * h.element_size() for h in host)
        d2h = 8 * (hout.spectrum.numel() + hout.divmap.numel() + hout.aeff_hist.numel()
                   + hout.moments.numel())

        def e2e_step():
            B.qs_scatter_host(wl.laser, wl.beam, host, wl.bins, precision=args.precision,
                              out=hout)

        # this box's pinned host-to-device copy rate (one stream, 512 MB):
        # the end-to-end step is copy-bound when it falls below ~50 GB/s
        hb = host[0][:1 << 27] if host[0].numel() >= 1 << 27 else host[0]
        db = torch.empty_like(hb, device=dev)
        db.copy_(hb, non_blocking=True)
        torch.cuda.synchronize()
        ca, cb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ca.record(stream)
        for _ in range(3):
            db.copy_(hb, non_blocking=True)
        cb.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = 3 * hb.numel() * hb.element_size() / (ca.elapsed_time(cb) * 1e-3) / 1e9

        k2 = max(4, args.steps)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k2 + 1)]
        clk2 = ClockSampler(local)
        clk2.start()
        time.sleep(1.0)            # nvidia-smi starts before the timed steps
        # warm-up steps after the pause (the first step after an idle second
        # ran up to 4x slower), as many as the device-resident line's
        for _ in range(max(3, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        evs[0].record(stream)
        for k in range(k2):
            e2e_step()
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        e2e_clocks = clk2.stop()
        step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(k2)]
        ms_e2e = evs[0].elapsed_time(evs[k2]) / k2
        if ws > 1:
            t = torch.tensor([ms_e2e], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t.item())
        ca.record(stream)
        for _ in range(3):
            db.copy_(hb, non_blocking=True)
        cb.record(stream)
        torch.cuda.synchronize()
        h2d_gbs_after = 3 * hb.numel() * hb.element_size() / (ca.elapsed_time(cb) * 1e-3) / 1e9
        del db
        same = bool(torch.equal(hout.spectrum, out.spectrum.cpu()))
        e2e = {"value": n * ws / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
               "api": "qs_scatter_host (pinned host samples, automatic chunks: whole waves, "
                      "growing x3 to 2^23; copy/compute overlap)",
               "spectrum_equals_device_path": same, "clocks": e2e_clocks,
               "steps": k2, "step_ms": [round(x, 3) for x in step_ms],
               "h2d_copy_gbs": [h2d_gbs, h2d_gbs_after]}
        del host, hout

    # ---- plain FP64 GPU path, same samples --------------------------------
    f64 = None
    if args.precision == "f32" and args.f64_steps > 0:
        o64 = B.Outputs(wl.bins, n, dev, "f64")
        # warm-up on a short prefix (module load, first launch); one full
        # FP64 step takes seconds
        B.qs_scatter(wl.laser, wl.beam, [x[:1 << 16] for x in xi], wl.bins, precision="f64")
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.f64_steps):
            step(precision="f64", o=o64)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b) / args.f64_steps
        m32, m64 = out.moments_dict(), o64.moments_dict()
        f64 = {"value": n / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
               "steps": args.f64_steps,
               "f32_vs_f64_rel_err": {k: abs(m32[k] / m64[k] - 1) if m64[k] else 0.0
                                      for k in ("mean", "spread", "div_x", "div_y")},
               "f32_vs_f64_spectrum_l1": float((out.spectrum - o64.spectrum).abs().sum()) / n}
        del o64

    # ---- roofline of the evaluation kernel --------------------------------
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    pk = peaks()
    fmax_mhz = float(pk.get("sm_max_mhz", 2070.0))
    steps_total = n * wl.laser.n_phase
    fma_ops = QFP_FMA_OPS_PER_STEP * steps_total
    mufu_ops = QFP_MUFU_SLOTS_PER_STEP * steps_total
    peak_fma = sms * FMA_LANES_PER_SM * fmax_mhz * 1e6
    peak_mufu = sms * MUFU_SLOTS_PER_SM * fmax_mhz * 1e6
    t_k = kern_ms * 1e-3
    t_bound = max(fma_ops / peak_fma, mufu_ops / peak_mufu)
    bound_pipe = "mufu" if mufu_ops / peak_mufu >= fma_ops / peak_fma else "fma"
    if bound_pipe == "mufu":
        achieved, peak_v = mufu_ops / t_k / 1e12, peak_mufu / 1e12
    else:
        achieved, peak_v = fma_ops / t_k / 1e12, peak_fma / 1e12
    # the same bound with the unit rates measured on this GPU now (per SM per
    # clock at the maximum clock)
    ur = B.unit_rates()
    sm_clk = ur["sms"] * ur["sm_max_mhz"] * 1e6
    t_meas_mufu = steps_total * sum(c / ur[k] for k, c in QFP_MUFU_MIX.items()) / sm_clk
    # the FMA pipe's measured rate for the instruction the loop issues (the
    # packed f32x2 FMA), in lane-operations
    t_meas_fma = steps_total * QFP_FMA_OPS_PER_STEP / ur.get("fma2", ur["fma"]) / sm_clk
    tr = TRAFFIC_BY_SOURCE.get(kernel_source_hash())
    roof = {"bound": "alu", "pipe": bound_pipe, "achieved": achieved, "peak": peak_v,
            "unit": "Top/s", "frac": t_bound / t_k,
            "traffic": None if tr is None else tr * n / (1 << 26),
            "kernel": "k_scatter<float>", "kernel_ms": kern_ms,
            "peak_source": f"{sms} SMs x {MUFU_SLOTS_PER_SM if bound_pipe == 'mufu' else FMA_LANES_PER_SM}"
                           f" per clock x {fmax_mhz:.0f} MHz (max SM clock)",
            "fma_frac": (fma_ops / peak_fma) / t_k, "mufu_frac": (mufu_ops / peak_mufu) / t_k,
            "measured_unit_rates": {k: round(v, 3) for k, v in ur.items()},
            "frac_of_measured_rates": max(t_meas_mufu, t_meas_fma) / t_k,
            "ops_per_sample_step": {"fma_pipe": QFP_FMA_OPS_PER_STEP,
                                    "mufu_slots": QFP_MUFU_SLOTS_PER_STEP,
                                    "source": "the FP32 kernel's packed instructions"},
            "oracle_expression_ops_per_sample_step": {"fma_pipe": ORACLE_CELL_FMA_OPS,
                                                      "mufu_slots": ORACLE_CELL_MUFU_SLOTS},
            # time the oracle expression's operation count needs at the pipes'
            # peaks over the kernel's time: above 1 when the kernel computes
            # the cell with fewer operations than the expression as written
            "oracle_expression_bound_over_kernel_time":
                max(ORACLE_CELL_FMA_OPS * steps_total / peak_fma,
                    ORACLE_CELL_MUFU_SLOTS * steps_total / peak_mufu) / t_k,
            "mufu_frac_of_measured": t_meas_mufu / t_k,
            "fma_frac_of_measured": t_meas_fma / t_k}

    batch = None if args.no_batch else bench_batch(dev, rank, n_shots=args.batch_shots)
    grad = None if args.no_grad else bench_grad(dev, rank, n=args.grad_n)
    if grad is not None:
        grad["fit256"] = bench_fit256(dev, rank)
    broad = None if args.no_broadband else bench_broadband(dev, rank, args.broadband_n)
    ll = None if args.no_ll else bench_ll(dev, rank, n=args.ll_n)
    cell = None if args.no_cell else bench_variant(dev, rank, 1, n=args.cell_n)
    cyc = None if args.no_cell else bench_variant(dev, rank, 2, n=args.cell_n)
    phot = None if args.no_photon else bench_photon(dev, rank, n=args.photon_n)
    pwr = None if args.no_pw else bench_pw(dev, rank)
    gh = bench_gh32(dev, rank)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        procs = host_cores()
        nh = 1 << 16
        xi_host = [x[:nh].cpu().numpy() for x in xi]
        rate1, done1, dt1 = cpu_oracle_rate(wl, xi_host, seconds=6.0)
        xi_host = [x[:max(nh, 2048 * procs * 64)].cpu().numpy() for x in xi]
        rate, done, dt = cpu_oracle_rate_all_cores(wl, xi_host, procs)
        cpu = {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"first {done} samples of the workload ({dt:.1f} s, FP64 C oracle, "
                         f"{procs} processes)",
               "single_core": {"value": rate1, "cores": 1,
                               "sample": f"first {done1} samples ({dt1:.1f} s, one thread)"},
               "gh32_full": cpu_oracle_gh32(),
               "discretization": cpu_oracle_discretization(wl, xi_host)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
                "data": "synthetic",
                "config": {"workload": wl.name, "n_samples_per_gpu": n, "model": "qfp",
                           "n_phase": wl.laser.n_phase, "spectrum_bins": wl.bins.n_bins,
                           "divmap": f"{wl.bins.n_tx}x{wl.bins.n_ty}",
                           "aeff_bins": wl.bins.n_aeff,
                           "moments": "f64", "parallelism": f"dp{ws} (independent samples)",
                           "l2": "inputs (2.1 GB per GPU) larger than L2; no flush"},
                "gpu_launches": 2 * args.steps, "clocks": clocks, "roofline": roof,
                "cpu_baseline": cpu, "e2e": e2e, "fp64_path": f64,
                "paper_context": "the paper's own Python tool gives one prediction in a few "
                                 "minutes on an unspecified personal computer (no per-sample "
                                 "rate or hardware stated): context, not a baseline",
                "batch_shots": batch, "grad": grad, "broadband": broad, "classical_ll": ll,
                "cell_focus": cell, "cycle_chi": cyc, "photon": phot,
                "pw_reconstruction": pwr, "gauss_hermite_32": gh,
                "gpu": props.name}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
