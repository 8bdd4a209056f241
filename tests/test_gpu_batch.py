"""qs_scatter_batch: many shots in one persistent launch, checked shot by
shot against single-shot qs_scatter calls and against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_09348_gb300 import binding as B
from paper_2308_09348_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# agreement of moments between different sample partitions of one problem
# GPU path against GPU path: the FP32 classical single-shot path sums each
# group of four samples before its compensated step, the batch path adds
# sample by sample, so the FP32 moments differ by the rounding of those
# groupings (a couple of FP32 ulps, 2^-24 = 6e-8)
MOM_RTOL = {"f64": 1e-12, "f32": 1e-7}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_09348_gb300 import build
    build.build()


def _small_batch(n_shots=37, seed=5, n_phase=64, log10_range=(0.0, 3.7)):
    bw = I.batch_shots(n_shots, seed=seed, log10_range=log10_range, n_phase=n_phase,
                       n_bins=96, model_mix=True)
    counts = bw.counts.copy()
    # ragged edge cases: empty, single, around the pair and tile boundaries
    special = [0, 1, 2, 63, 64, 65, 2047, 2048, 2049]
    counts[:len(special)] = special
    offsets = np.zeros(n_shots + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    n = int(offsets[-1])
    xi = I.sample_streams(n, seed + 100, dtype=np.float32)
    return bw, counts, offsets, xi


def _run_batch(bw, offsets, xi, prec, w=None, tile=0, block=0):
    xt = [torch.from_numpy(a).cuda() for a in xi]
    wt = None if w is None else torch.from_numpy(w).cuda()
    bt = B.Batch(bw.lasers, bw.beams, offsets, bw.bins, len(xi[0]), ranges=bw.ranges,
                 precision=prec, tile=tile, block=block)
    bt.run(xt, wt)
    torch.cuda.synchronize()
    return bt, xt, wt


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("weighted", [False, True])
def test_batch_equals_single_shot_calls(prec, weighted):
    bw, counts, offsets, xi = _small_batch()
    w = I.rng(77).uniform(0.5, 1.5, len(xi[0])).astype(np.float32) if weighted else None
    bt, xt, wt = _run_batch(bw, offsets, xi, prec, w)
    spectra = bt.spectra.cpu().numpy()
    mom = bt.moments.cpu().numpy()
    for s in range(len(counts)):
        o0, o1 = int(offsets[s]), int(offsets[s + 1])
        bins = I.Bins(n_bins=bw.bins.n_bins, lo=float(bw.ranges[s, 0]), hi=float(bw.ranges[s, 1]))
        if o1 == o0:
            assert mom[s, 0] == 0 and spectra[s].sum() == 0
            continue
        sub = [x[o0:o1] for x in xt]
        ws = None if wt is None else wt[o0:o1]
        ref = B.qs_scatter(bw.lasers[s], bw.beams[s], sub, bins, w=ws, precision=prec)
        torch.cuda.synchronize()
        # identical per-sample code: integer histograms agree exactly
        assert np.array_equal(spectra[s], ref.spectrum.cpu().numpy()), s
        r = ref.moments.cpu().numpy()
        # FP32 path: per-thread compensated FP32 sums over different sample
        # partitions (batch tiles vs single-shot grid) differ in rounding
        np.testing.assert_allclose(mom[s], r, rtol=MOM_RTOL[prec], atol=1e-300)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("weighted", [False, True])
def test_batch_divergence_maps_and_aeff_histograms_equal_single_shot_calls(prec, weighted):
    """Per-shot divergence maps (64 x 48 over +-10 mrad) and a_eff
    histograms (40 bins on [0, 50]) beside the spectra: every shot's map,
    a_eff histogram and weight outside its map equal its single-shot call
    exactly (integer accumulation of the same per-sample bins), quantum and
    classical shots, ragged and empty shots; the batched adjoint accepts the
    same bins."""
    bw, counts, offsets, xi = _small_batch(n_shots=21, seed=8)
    bins = I.Bins(n_bins=bw.bins.n_bins, lo=0.0, hi=1.0, n_tx=64, n_ty=48, theta_max=10e-3,
                  n_aeff=40, aeff_max=50.0)
    xt = [torch.from_numpy(a).cuda() for a in xi]
    w = I.rng(78).uniform(0.5, 1.5, len(xi[0])).astype(np.float32) if weighted else None
    wt = None if w is None else torch.from_numpy(w).cuda()
    bt = B.Batch(bw.lasers, bw.beams, offsets, bins, len(xi[0]), ranges=bw.ranges,
                 precision=prec)
    bt.run(xt, wt)
    torch.cuda.synchronize()
    assert bt.divmaps.shape == (21, 48, 64) and bt.aeff_hists.shape == (21, 40)
    mom = bt.moments.cpu().numpy()
    i_out = B.MOMENT_FIELDS.index("map_out")
    nonzero = 0
    for s in range(21):
        o0, o1 = int(offsets[s]), int(offsets[s + 1])
        if o1 == o0:
            assert torch.count_nonzero(bt.divmaps[s]) == 0 and mom[s, 0] == 0
            continue
        b_s = I.Bins(**{**bins.__dict__, "lo": float(bw.ranges[s, 0]),
                        "hi": float(bw.ranges[s, 1])})
        ref = B.qs_scatter(bw.lasers[s], bw.beams[s], [x[o0:o1] for x in xt], b_s,
                           w=None if wt is None else wt[o0:o1], precision=prec)
        r = ref.result()
        torch.cuda.synchronize()
        assert torch.equal(bt.divmaps[s], r["divmap"]), s
        assert torch.equal(bt.aeff_hists[s], r["aeff_hist"]), s
        assert torch.equal(bt.spectra[s], r["spectrum"]), s
        assert mom[s, i_out] == r["moments"]["map_out"], s
        nonzero += int(torch.count_nonzero(bt.divmaps[s]) > 0)
    assert nonzero >= 10
    # the batched adjoint takes the same bins (maps and a_eff histograms do
    # not enter the gradient)
    dm = torch.zeros(21, 13, dtype=torch.float64)
    dm[:, 1] = 1e-3
    g = bt.grad(xt, dm, w=wt)
    torch.cuda.synchronize()
    assert torch.isfinite(g).all()


def test_batch_matches_oracle_f64():
    bw, counts, offsets, xi = _small_batch(n_shots=12, seed=6, log10_range=(1.0, 3.0))
    bt, _, _ = _run_batch(bw, offsets, xi, "f64")
    mom = bt.moments_dicts()
    spectra = bt.spectra.cpu().numpy()
    for s in range(12):
        o0, o1 = int(offsets[s]), int(offsets[s + 1])
        if o1 == o0:
            continue
        bins = I.Bins(n_bins=bw.bins.n_bins, lo=float(bw.ranges[s, 0]), hi=float(bw.ranges[s, 1]))
        ref = oracle.scatter(bw.lasers[s], bw.beams[s], bins,
                             [a[o0:o1].astype(np.float64) for a in xi])
        for k in ("W", "mean", "spread", "div_x", "div_y", "mean_aeff", "mean_gamma0"):
            assert abs(mom[s][k] - ref["moments"][k]) <= 1e-12 * abs(ref["moments"][k]), (s, k)
        assert np.abs(spectra[s] - ref["spectrum"]).sum() <= 1e-4 * (o1 - o0)


def test_batch_matches_oracle_f32_512_cells():
    """FP32 batch at the benchmarked 512 phase cells against the oracle
    directly: moments within 1e-5; spectrum bins exact for every sample
    farther than the FP32 path's error bound from an edge (L1 at most twice
    the weight of the others)."""
    from test_gpu_parity import away_from_edges, gout_bound
    bw, counts, offsets, xi = _small_batch(n_shots=12, seed=16, n_phase=512,
                                           log10_range=(1.0, 3.0))
    bt, _, _ = _run_batch(bw, offsets, xi, "f32")
    mom = bt.moments_dicts()
    spectra = bt.spectra.cpu().numpy()
    for s in range(12):
        o0, o1 = int(offsets[s]), int(offsets[s + 1])
        if o1 == o0:
            continue
        bins = I.Bins(n_bins=bw.bins.n_bins, lo=float(bw.ranges[s, 0]), hi=float(bw.ranges[s, 1]))
        sub = [a[o0:o1].astype(np.float64) for a in xi]
        ref = oracle.scatter(bw.lasers[s], bw.beams[s], bins, sub)
        for k in ("W", "mean", "spread", "div_x", "div_y", "mean_aeff", "mean_gamma0"):
            assert abs(mom[s][k] - ref["moments"][k]) <= 1e-5 * abs(ref["moments"][k]), (s, k)
        rec = oracle.evaluate(bw.lasers[s], bw.beams[s], bins, sub)
        near = ~away_from_edges(rec["gamma_out"], gout_bound(rec, "f32"), bins)
        l1 = np.abs(spectra[s] - ref["spectrum"]).sum()
        assert l1 <= 2.0 * near.sum(), (s, l1, int(near.sum()))


def test_invalid_shot_is_flagged_and_others_unaffected():
    bw, counts, offsets, xi = _small_batch(n_shots=10, seed=7, log10_range=(2.0, 3.0))
    lasers = list(bw.lasers)
    lasers[4] = I.Laser(**{**lasers[4].__dict__, "w0_um": -1.0})
    bad = I.BatchWorkload(bw.name, tuple(lasers), bw.beams, bw.counts, bw.offsets, bw.ranges,
                          bw.bins, bw.seed)
    bt, _, _ = _run_batch(bad, offsets, xi, "f32")
    good, _, _ = _run_batch(bw, offsets, xi, "f32")
    m, mg = bt.moments.cpu().numpy(), good.moments.cpu().numpy()
    assert m[4, 0] == 0 and m[4, B.MOMENT_FIELDS.index("nonfinite")] == -1
    for s in range(10):
        if s != 4:
            assert np.array_equal(m[s], mg[s])


@pytest.mark.parametrize("tile,block", [(64, 64), (512, 128), (4096, 256)])
def test_schedule_does_not_change_results(tile, block):
    bw, counts, offsets, xi = _small_batch(seed=8)
    ref, _, _ = _run_batch(bw, offsets, xi, "f32")
    bt, _, _ = _run_batch(bw, offsets, xi, "f32", tile=tile, block=block)
    assert torch.equal(bt.spectra, ref.spectra)
    np.testing.assert_allclose(bt.moments.cpu().numpy(), ref.moments.cpu().numpy(),
                               rtol=MOM_RTOL["f32"])


def test_batch_repeated_and_graph_replay_identical():
    bw, counts, offsets, xi = _small_batch(seed=9)
    bt, xt, _ = _run_batch(bw, offsets, xi, "f32")
    m1, s1 = bt.moments.clone(), bt.spectra.clone()
    bt.run(xt)
    torch.cuda.synchronize()
    assert torch.equal(bt.moments, m1) and torch.equal(bt.spectra, s1)
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        bt.run(xt, stream=st)
    bt.moments.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(bt.moments, m1) and torch.equal(bt.spectra, s1)


def test_all_empty_shots():
    bw = I.batch_shots(5, seed=10, log10_range=(1, 2), n_bins=16)
    offsets = np.zeros(6, dtype=np.int64)
    xi = [np.zeros(4, dtype=np.float32) for _ in range(8)]
    bt, _, _ = _run_batch(bw, offsets, xi, "f32")
    assert float(bt.moments.abs().sum()) == 0 and float(bt.spectra.abs().sum()) == 0


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_delay_sweep_over_shared_samples(prec):
    """A sweep (no offsets): every shot integrates the same samples with its
    own delay; each equals a single-shot call with that delay."""
    wl = I.broadband_qfp(3001)
    L0 = I.Laser(**{**wl.laser.__dict__, "n_phase": 128})
    delays = np.linspace(-100.0, 100.0, 9)
    lasers = [I.Laser(**{**L0.__dict__, "delay_fs": float(d)}) for d in delays]
    beams = [wl.beam] * len(delays)
    xi, _ = I.workload_inputs(wl, 3001)
    xt = [torch.from_numpy(a).cuda() for a in xi]
    bt = B.Batch(lasers, beams, None, wl.bins, 3001, precision=prec)
    bt.run(xt)
    torch.cuda.synchronize()
    for k, L in enumerate(lasers):
        ref = B.qs_scatter(L, wl.beam, xt, wl.bins, precision=prec)
        torch.cuda.synchronize()
        assert torch.equal(bt.spectra[k], ref.spectrum), k
        np.testing.assert_allclose(bt.moments[k].cpu().numpy(), ref.moments.cpu().numpy(),
                                   rtol=MOM_RTOL[prec])
    # the sweep is symmetric in nothing in particular, but the spectra differ
    assert not torch.equal(bt.spectra[0], bt.spectra[4])


def test_decreasing_offsets_invalidate_every_shot():
    """Offsets that decrease anywhere ([0, N, 0, N, ...]: shot ranges that
    overlap) make every shot invalid and no shot does any work, whatever the
    per-shot checks alone would pass; a valid batch on the same workspace
    afterwards is unaffected."""
    n_shots = 8
    bw = I.batch_shots(n_shots, seed=9, log10_range=(3.0, 3.5), n_phase=64, n_bins=64)
    n = int(bw.offsets[-1])
    xi = I.sample_streams(n, 909, dtype=np.float32)
    xt = [torch.from_numpy(a).cuda() for a in xi]
    bad = np.array([0, n] * (n_shots // 2) + [n], dtype=np.int64)
    bt = B.Batch(bw.lasers, bw.beams, bad, bw.bins, n, ranges=bw.ranges, precision="f32")
    bt.spectra.fill_(7.0)
    bt.run(xt)
    torch.cuda.synchronize()
    m = bt.moments.cpu().numpy()
    assert np.all(m[:, B.MOMENT_FIELDS.index("W")] == 0)
    assert np.all(m[:, B.MOMENT_FIELDS.index("nonfinite")] == -1)
    assert np.all(bt.spectra.cpu().numpy() == 0)
    # the same descriptors with valid offsets, on the same workspace
    bt.d_offsets = torch.as_tensor(bw.offsets, dtype=torch.int64).cuda()
    bt.run(xt)
    torch.cuda.synchronize()
    m = bt.moments.cpu().numpy()
    assert np.all(m[:, B.MOMENT_FIELDS.index("nonfinite")] == 0)
    np.testing.assert_array_equal(m[:, 0], np.diff(bw.offsets).astype(float))
