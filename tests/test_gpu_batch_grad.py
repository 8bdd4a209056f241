"""qs_scatter_grad_batch and the batched smoothed spectrum: every shot's
gradient against a single-shot qs_scatter_grad call and against the oracle,
through the C ABI; the batched autograd function; a batched gradient fit that
brings every parameter of every shot back to its hidden value."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_09348_gb300 import binding as B
from paper_2308_09348_gb300 import fit as F
from paper_2308_09348_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SCALE = np.array([20.0, 4.0, 1.0, 1.0, 10.0, 6000.0, 0.08, 1e-3])


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_09348_gb300 import build
    build.build()


def _shots(n_shots=9, seed=31, n_phase=64, log10_range=(2.0, 3.6), model_mix=True, n_bins=128):
    bw = I.batch_shots(n_shots, seed=seed, log10_range=log10_range, n_phase=n_phase,
                       n_bins=n_bins, model_mix=model_mix)
    bins = I.Bins(n_bins=n_bins, lo=0.0, hi=1.0, smooth_sigma_bins=2.0)
    counts = bw.counts.copy()
    counts[:4] = [0, 1, 63, 2049][:min(4, n_shots)]
    offsets = np.zeros(n_shots + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    xi = I.sample_streams(int(offsets[-1]), seed + 1, dtype=np.float32)
    return bw, bins, offsets, xi


def _upstream(n_shots, nb, seed):
    rg = I.rng(seed)
    dm = np.zeros((n_shots, 13))
    for k, sc in (("mean", 1e-3), ("spread", 1e-3), ("rel_spread", 1.0), ("div_x", 1e3),
                  ("div_y", 1e3), ("div", 1e3), ("mean_aeff", 1.0), ("mean_gamma0", 1e-3)):
        dm[:, B.MOMENT_FIELDS.index(k)] = rg.normal(size=n_shots) * sc
    dS = rg.normal(size=(n_shots, nb)) * 1e-3
    return dm, dS


def _batch(bw, bins, offsets, xi, prec, w=None):
    xt = [torch.from_numpy(a).cuda() for a in xi]
    wt = None if w is None else torch.from_numpy(w).cuda()
    bt = B.Batch(bw.lasers, bw.beams, offsets, bins, len(xi[0]), ranges=bw.ranges, precision=prec)
    bt.run(xt, wt)
    return bt, xt, wt


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_gradient_equals_single_shot_calls(prec):
    """Row s of the batched gradient equals qs_scatter_grad of shot s alone
    (quantum and classical shots, weights, ragged and empty shots); the
    batched smoothed spectra equal the single-shot ones exactly (integer
    accumulation of the same per-sample deposits)."""
    bw, bins, offsets, xi = _shots()
    w = I.rng(5).uniform(0.5, 1.5, len(xi[0])).astype(np.float32)
    bt, xt, wt = _batch(bw, bins, offsets, xi, prec, w)
    n_shots = len(bw.lasers)
    dm, dS = _upstream(n_shots, bins.n_bins, 7)
    g = bt.grad(xt, torch.from_numpy(dm), torch.from_numpy(dS), w=wt).cpu().numpy()
    torch.cuda.synchronize()
    mom = bt.moments.cpu().numpy()
    for s in range(n_shots):
        o0, o1 = int(offsets[s]), int(offsets[s + 1])
        if o1 == o0:
            assert np.all(g[s] == 0) and mom[s, 0] == 0
            continue
        b_s = I.Bins(**{**bins.__dict__, "lo": float(bw.ranges[s, 0]), "hi": float(bw.ranges[s, 1])})
        sub, ws = [x[o0:o1] for x in xt], wt[o0:o1]
        ref = B.qs_scatter(bw.lasers[s], bw.beams[s], sub, b_s, w=ws, precision=prec)
        gr = B.qs_scatter_grad(bw.lasers[s], bw.beams[s], sub, b_s, ref.moments,
                               torch.from_numpy(dm[s]), torch.from_numpy(dS[s]), w=ws,
                               precision=prec, out=ref).cpu().numpy()
        torch.cuda.synchronize()
        assert torch.equal(bt.spec_smooth[s], ref.spec_smooth), s
        assert torch.equal(bt.spectra[s], ref.spectrum), s
        err = np.abs((g[s] - gr) * SCALE) / max(np.max(np.abs(gr * SCALE)), 1e-300)
        print(f"[{prec}] shot {s} model {bw.lasers[s].model}: n={o1 - o0} max scaled err {err.max():.2e}")
        assert np.all(err <= (1e-12 if prec == "f64" else 1e-6)), (s, err)


def test_batched_gradient_matches_oracle_f64():
    bw, bins, offsets, xi = _shots(n_shots=6, seed=33, log10_range=(2.0, 3.0))
    bt, xt, _ = _batch(bw, bins, offsets, xi, "f64")
    dm, dS = _upstream(6, bins.n_bins, 8)
    g = bt.grad(xt, torch.from_numpy(dm), torch.from_numpy(dS)).cpu().numpy()
    for s in range(6):
        o0, o1 = int(offsets[s]), int(offsets[s + 1])
        if o1 - o0 < 2:
            continue
        b_s = I.Bins(**{**bins.__dict__, "lo": float(bw.ranges[s, 0]), "hi": float(bw.ranges[s, 1])})
        ref = oracle.grad(bw.lasers[s], bw.beams[s], b_s, b_s.smooth_sigma_bins,
                          [a[o0:o1].astype(np.float64) for a in xi], None, dL_dm=dm[s],
                          dL_dS=dS[s])
        rs = ref["grad"] * SCALE
        err = np.abs(g[s] * SCALE - rs) / np.max(np.abs(rs))
        assert np.all(err <= 1e-10), (s, err)
        np.testing.assert_allclose(bt.spec_smooth[s].cpu().numpy(), ref["smooth"], rtol=0,
                                   atol=1e-12 * (o1 - o0) + 25 * (o1 - o0) * 2.0 ** -32)


def test_batched_gradient_repeatable_and_autograd():
    bw, bins, offsets, xi = _shots(n_shots=7, seed=35)
    bt, xt, _ = _batch(bw, bins, offsets, xi, "f32")
    dm, dS = _upstream(7, bins.n_bins, 9)
    g1 = bt.grad(xt, torch.from_numpy(dm), torch.from_numpy(dS)).clone()
    g2 = bt.grad(xt, torch.from_numpy(dm), torch.from_numpy(dS)).clone()
    assert torch.equal(g1, g2)
    prob = F.BatchProblem(bt, xt)
    theta = bt.params().clone().requires_grad_(True)
    mom, S = F.BatchScatterFn.apply(theta, prob)
    L = (mom * torch.from_numpy(dm).cuda()).sum() + (S * torch.from_numpy(dS).cuda()).sum()
    L.backward()
    assert torch.equal(theta.grad, g1)


def test_set_params_round_trip():
    bw, bins, offsets, xi = _shots(n_shots=5, seed=37)
    bt, _, _ = _batch(bw, bins, offsets, xi, "f32")
    th = bt.params().clone()
    ref = torch.tensor([[getattr(l, k) for k in F.LASER_FIELDS] + [getattr(b, k) for k in F.BEAM_FIELDS]
                        for l, b in zip(bw.lasers, bw.beams)], dtype=torch.float64)
    assert torch.equal(th.cpu(), ref)
    bt.set_params(th * 1.5)
    assert torch.equal(bt.params(), th * 1.5)
