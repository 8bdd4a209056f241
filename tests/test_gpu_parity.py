"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bars (floating point): per-sample FP64 results to rel 1e-12; moments to rel
1e-12 (FP64 path) and 1e-5 (FP32 path); spectra to 1e-4 of the total weight
in L1.  Bin indices are bit-exact for every sample whose oracle value lies
farther from a bin edge than the path's per-sample error bound.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2308_09348_gb300 import inputs as I
from paper_2308_09348_gb300 import MOMENT_FIELDS, QsError, qs_eval_samples, qs_scatter
from paper_2308_09348_gb300 import binding as B

pytestmark = pytest.mark.gpu

# per-sample error bounds of the two paths (relative, on mu; V; gamma_out)
TOL = {"f64": dict(mu=1e-12, V=1e-10, aeff=1e-13),
       "f32": dict(mu=4e-6, V=2e-5, aeff=None)}
MOM_TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_09348_gb300 import build
    build.build()


def dev(xi, w=None):
    xt = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in xi]
    wt = None if w is None else torch.from_numpy(np.ascontiguousarray(w)).cuda()
    return xt, wt


def f64(xi):
    return [None if a is None else a.astype(np.float64) for a in xi]


def cfg2(n, **laser_kw):
    wl = I.full_qfp(n)
    L = I.Laser(**{**wl.laser.__dict__, **laser_kw})
    xi, _ = I.workload_inputs(wl, n)
    return wl, L, xi


def away_from_edges(g_ref, tol_abs, bins):
    """Mask of samples whose oracle energy is farther than tol_abs from any
    energy-bin edge (or the under/over boundaries)."""
    if bins.log_spaced:
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.log(np.maximum(g_ref, 1e-300) / bins.lo) * (bins.n_bins / math.log(bins.hi / bins.lo))
            dt = tol_abs / np.maximum(g_ref, 1e-300) * (bins.n_bins / math.log(bins.hi / bins.lo))
    else:
        t = (g_ref - bins.lo) * (bins.n_bins / (bins.hi - bins.lo))
        dt = tol_abs * (bins.n_bins / (bins.hi - bins.lo))
    frac = np.abs(t - np.round(t))
    return frac > dt


def _relerr(a, b, floor=0.0):
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def compare_samples(rec, ref, prec, bins, check_bins=True):
    """Element-wise comparison; prints the error profile before asserting."""
    tol = TOL[prec]
    g = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in rec.items()}
    vmax = max(float(np.max(ref["V"])), 1e-300)
    # a_eff = a0 q^-1/2 exp(-X): in FP32 the argument X carries ~6 ulp of
    # relative rounding (rho^2, 1/W0^2, 1/q, log2 e) that the exponential turns
    # into an absolute error of X 6 2^-24; ex2, rsqrt and the products add a few
    # ulp more: bound (3 X + 16) 2^-23
    X = np.log(np.maximum(np.max(ref["aeff"]), 1e-300) / np.maximum(ref["aeff"], 1e-300))
    a_tol = tol["aeff"] if prec == "f64" else (3.0 * X + 16.0) * 2.0 ** -23
    # gamma_out = mu + sqrt(V) xi7: its error is bounded by that of mu plus half
    # the relative error of V times |gamma_out - mu|
    gabs = gout_bound(ref, prec)
    prof = {"gamma0": float(np.max(_relerr(g["gamma0"], ref["gamma0"]))),
            "aeff": float(np.max(_relerr(g["aeff"], ref["aeff"], 1e-300) / a_tol)),
            "mu": float(np.max(_relerr(g["mu"], ref["mu"]))),
            "V": float(np.max(np.abs(g["V"] - ref["V"]) / (np.abs(ref["V"]) + 1e-6 * vmax))),
            "gout_abs/tol": float(np.max(np.abs(g["gamma_out"] - ref["gamma_out"]) / gabs))}
    print(f"[{prec}] error profile:", prof)
    # FP32 path: gamma0 = gamma_mean (1 + s xi3) is formed in FP32 (then
    # promoted exactly for the FP64 recombination)
    assert prof["gamma0"] <= (1e-15 if prec == "f64" else 2.0 ** -22)
    assert prof["aeff"] <= 1.0
    assert prof["mu"] <= tol["mu"]
    assert prof["V"] <= tol["V"]
    assert prof["gout_abs/tol"] <= 1.0
    if check_bins and bins is not None and bins.n_bins > 0:
        ok = away_from_edges(ref["gamma_out"], gabs, bins)
        print(f"[{prec}] samples near an energy-bin edge: {int((~ok).sum())} of {ok.size}")
        assert ok.mean() > 0.99
        np.testing.assert_array_equal(g["bin"][ok], ref["bin"][ok])
    if bins is not None and bins.n_aeff > 0:
        fa = ref["aeff"] * bins.n_aeff / bins.aeff_max
        a_ok = np.abs(fa - np.round(fa)) > 2 * a_tol * fa + 1e-12
        np.testing.assert_array_equal(g["abin"][a_ok], ref["abin"][a_ok])
    return g


# ---------------------------------------------------------------------------
# per-sample records
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("model,env", [(I.MODEL_LL, I.ENV_GAUSS), (I.MODEL_QFP, I.ENV_GAUSS),
                                       (I.MODEL_QFP, I.ENV_SIN2)])
def test_eval_matches_oracle_elementwise(prec, model, env):
    n = 2500          # ~10 tiles of 256 and a ragged tail
    wl, L, xi = cfg2(n, model=model, envelope=env)
    xt, _ = dev(xi)
    rec = qs_eval_samples(L, wl.beam, xt, wl.bins, precision=prec)
    torch.cuda.synchronize()
    ref = oracle.evaluate(L, wl.beam, wl.bins, f64(xi))
    compare_samples(rec, ref, prec, wl.bins)


def test_eval_float64_streams_and_missing_optional_streams():
    n = 777
    wl, L, xi = cfg2(n)
    xi64 = f64(xi)
    xi64[5] = None      # theta_y stream absent: reads as zeros
    xi64[6] = None
    xt, _ = dev(xi64)
    rec = qs_eval_samples(L, wl.beam, xt, wl.bins, precision="f64")
    ref = oracle.evaluate(L, wl.beam, wl.bins, xi64)
    compare_samples(rec, ref, "f64", wl.bins)


# ---------------------------------------------------------------------------
# per-cell focus (Eq. 2 along the electron's path)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("model,env", [(I.MODEL_LL, I.ENV_GAUSS), (I.MODEL_QFP, I.ENV_GAUSS),
                                       (I.MODEL_QFP, I.ENV_SIN2), (I.MODEL_LL, I.ENV_SIN2)])
def test_per_cell_focus_eval_matches_oracle(prec, model, env):
    n = 1500
    wl, L, xi = cfg2(n, model=model, envelope=env, n_phase=256, variant=I.VAR_CELL_FOCUS)
    xt, _ = dev(xi)
    rec = qs_eval_samples(L, wl.beam, xt, wl.bins, precision=prec)
    torch.cuda.synchronize()
    ref = oracle.evaluate(L, wl.beam, wl.bins, f64(xi))
    compare_samples(rec, ref, prec, wl.bins)
    # the variant changes the result at this focus (z_R = 24.5 um, 40 fs delay)
    Lx = I.Laser(**{**L.__dict__, "variant": 0})
    refx = oracle.evaluate(Lx, wl.beam, wl.bins, f64(xi))
    assert np.max(np.abs(refx["mu"] / ref["mu"] - 1)) > 1e-3


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("model", [I.MODEL_LL, I.MODEL_QFP])
def test_per_cell_focus_scatter_matches_oracle_and_records(prec, model):
    n = 3001
    wl, L, xi = cfg2(n, model=model, n_phase=128, variant=I.VAR_CELL_FOCUS)
    w = I.rng(17).uniform(0.25, 2.0, n).astype(np.float32)
    xt, wt = dev(xi, w)
    out = qs_scatter(L, wl.beam, xt, wl.bins, w=wt, precision=prec)
    torch.cuda.synchronize()
    ref = oracle.scatter(L, wl.beam, wl.bins, f64(xi), w.astype(np.float64))
    compare_scatter(out, ref, prec, float(w.astype(np.float64).sum()),
                    inputs=(L, wl.beam, wl.bins, xi, w))
    # unit weights: the fused spectrum is the histogram of the per-sample records
    out1 = qs_scatter(L, wl.beam, xt, wl.bins, precision=prec)
    rec = qs_eval_samples(L, wl.beam, xt, wl.bins, precision=prec)
    torch.cuda.synchronize()
    b = rec["bin"].cpu().numpy()
    hist = np.bincount(b[(b >= 0) & (b < wl.bins.n_bins)], minlength=wl.bins.n_bins)
    np.testing.assert_array_equal(out1.spectrum.cpu().numpy(), hist.astype(np.float64))


@pytest.mark.parametrize("prec,n,n_phase", [("f64", 300, 64), ("f32", 2500, 256)])
@pytest.mark.parametrize("variant", [I.VAR_CYCLE_CHI, I.VAR_CYCLE_CHI | I.VAR_CELL_FOCUS])
def test_cycle_resolved_chi_eval_matches_oracle(prec, n, n_phase, variant):
    """Cycle-resolved Gaunt and diffusion factors: FP64 by the same
    128-point cycle quadrature as the oracle, FP32 by the Hermite tables."""
    wl, L, xi = cfg2(n, model=I.MODEL_QFP, n_phase=n_phase, variant=variant)
    xt, _ = dev(xi)
    rec = qs_eval_samples(L, wl.beam, xt, wl.bins, precision=prec)
    torch.cuda.synchronize()
    ref = oracle.evaluate(L, wl.beam, wl.bins, f64(xi))
    compare_samples(rec, ref, prec, wl.bins)
    # the variant matters for this beam (chi ~ 1 at the peak)
    L0 = I.Laser(**{**L.__dict__, "variant": variant & I.VAR_CELL_FOCUS})
    ref0 = oracle.evaluate(L0, wl.beam, wl.bins, f64(xi))
    assert np.max(np.abs(ref0["mu"] / ref["mu"] - 1)) > 1e-3


def test_cycle_resolved_chi_scatter_matches_oracle():
    n = 2001
    wl, L, xi = cfg2(n, model=I.MODEL_QFP, n_phase=64, variant=I.VAR_CYCLE_CHI)
    xt, _ = dev(xi)
    out = qs_scatter(L, wl.beam, xt, wl.bins, precision="f32")
    torch.cuda.synchronize()
    ref = oracle.scatter(L, wl.beam, wl.bins, f64(xi))
    compare_scatter(out, ref, "f32", float(n), inputs=(L, wl.beam, wl.bins, xi, None))


VARIANT_CASES = [(I.MODEL_LL, I.VAR_CELL_FOCUS), (I.MODEL_QFP, I.VAR_CELL_FOCUS),
                 (I.MODEL_QFP, I.VAR_CYCLE_CHI), (I.MODEL_QFP, I.VAR_CELL_FOCUS | I.VAR_CYCLE_CHI)]


def _variant_case(n, model, variant, n_phase=48):
    """The bench laser with a tighter focus and a wider divergence, so that
    the path through the focus matters (the per-cell focus), and a strong
    field (chi ~ 1: the cycle-resolved factors differ from the rms ones)."""
    wl, L, xi = cfg2(n, n_phase=n_phase, model=model, variant=variant, w0_um=2.0)
    beam = I.Beam(**{**wl.beam.__dict__, "div_rad": 5e-3})
    bins = I.Bins(n_bins=128, lo=0.0, hi=6720.0, smooth_sigma_bins=2.0)
    return wl, L, beam, bins, xi


GRAD_SCALE = np.array([30.0, 2.0, 1.0, 1.0, 10.0, 4000.0, 0.1, 5e-3])


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("model,variant", VARIANT_CASES)
def test_variant_gradient_matches_oracle(prec, model, variant):
    """qs_scatter_grad for the model variants (seven tangents through the
    per-cell amplitudes; the cycle-resolved factors and their chi-derivatives)
    against the oracle's dual-number gradient, parameter-scaled relative to
    the largest component: FP64 1e-10, FP32 5e-7 (measured 2.4e-8 to 5.7e-8:
    the FP32 cycle factors come from the Hermite tables, 3e-7 in S, and the
    seven FP32 tangents sum over the cells without compensation)."""
    n = 1001 if not variant & I.VAR_CYCLE_CHI else 401
    wl, L, beam, bins, xi = _variant_case(n, model, variant)
    w = I.rng(41).uniform(0.5, 1.5, n).astype(np.float32)
    xt, wt = dev(xi, w)
    rg = I.rng(42)
    dm = np.zeros(13)
    for k, sc in (("mean", 1e-3), ("spread", 1e-3), ("div_x", 1e3), ("div_y", 1e3), ("div", 1e3),
                  ("mean_aeff", 1.0), ("mean_gamma0", 1e-3), ("rel_spread", 1.0)):
        dm[B.MOMENT_FIELDS.index(k)] = rg.normal() * sc
    dS = rg.normal(size=bins.n_bins) * 1e-3
    out = qs_scatter(L, beam, xt, bins, w=wt, precision=prec)
    g = B.qs_scatter_grad(L, beam, xt, bins, out.moments, torch.from_numpy(dm),
                          torch.from_numpy(dS), w=wt, precision=prec, out=out).cpu().numpy()
    ref = oracle.grad(L, beam, bins, bins.smooth_sigma_bins, f64(xi), w.astype(np.float64),
                      dL_dm=dm, dL_dS=dS)
    rs = ref["grad"] * GRAD_SCALE
    err = np.abs(g * GRAD_SCALE - rs) / np.max(np.abs(rs))
    print(f"[{prec}, model {model}, variant {variant}] scaled grad rel err: max {err.max():.3e}")
    assert np.all(err <= (1e-10 if prec == "f64" else 5e-7)), err


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_with_model_variants_equals_single_shot_calls(prec):
    """A batch mixing the paper's model with both variants (and the classical
    model with the per-cell focus): every shot equals its single-shot call
    (histograms exactly, moments to the batch's partition rounding), and the
    batched adjoint equals the single-shot adjoint shot by shot."""
    bw = I.batch_shots(8, seed=21, log10_range=(2.3, 3.0), n_phase=48, n_bins=64, model_mix=True)
    variants = [0, I.VAR_CELL_FOCUS, I.VAR_CYCLE_CHI, I.VAR_CELL_FOCUS | I.VAR_CYCLE_CHI,
                0, I.VAR_CELL_FOCUS, I.VAR_CYCLE_CHI, I.VAR_CELL_FOCUS]
    lasers = []
    for k, L0 in enumerate(bw.lasers):
        v = variants[k]
        model = I.MODEL_QFP if (v & I.VAR_CYCLE_CHI or k % 2 == 0) else L0.model
        lasers.append(I.Laser(**{**L0.__dict__, "variant": v, "model": model, "w0_um": 2.5}))
    beams = [I.Beam(**{**b.__dict__, "div_rad": 5e-3}) for b in bw.beams]
    bins = I.Bins(n_bins=64, lo=0.0, hi=1.0, smooth_sigma_bins=2.0)
    offsets = np.zeros(9, dtype=np.int64)
    offsets[1:] = np.cumsum(bw.counts)
    n = int(offsets[-1])
    xs = [torch.from_numpy(a).cuda() for a in I.sample_streams(n, 22, dtype=np.float32)]
    bt = B.Batch(lasers, beams, offsets, bins, n, ranges=bw.ranges, precision=prec)
    bt.run(xs)
    rg = I.rng(23)
    dm = np.zeros((8, 13))
    dm[:, 1] = rg.normal(size=8) * 1e-3
    dm[:, 2] = rg.normal(size=8) * 1e-3
    dm[:, 4] = rg.normal(size=8) * 1e3
    dS = rg.normal(size=(8, 64)) * 1e-3
    gb = bt.grad(xs, torch.from_numpy(dm), torch.from_numpy(dS)).cpu().numpy()
    torch.cuda.synchronize()
    mom = bt.moments.cpu().numpy()
    assert np.all(mom[:, B.MOMENT_FIELDS.index("nonfinite")] == 0), mom[:, -1]
    for s_ in range(8):
        o0, o1 = int(offsets[s_]), int(offsets[s_ + 1])
        b_s = I.Bins(**{**bins.__dict__, "lo": float(bw.ranges[s_, 0]),
                        "hi": float(bw.ranges[s_, 1])})
        sub = [x[o0:o1] for x in xs]
        ref = qs_scatter(lasers[s_], beams[s_], sub, b_s, precision=prec)
        gr = B.qs_scatter_grad(lasers[s_], beams[s_], sub, b_s, ref.moments,
                               torch.from_numpy(dm[s_]), torch.from_numpy(dS[s_]),
                               precision=prec, out=ref).cpu().numpy()
        torch.cuda.synchronize()
        assert torch.equal(bt.spectra[s_], ref.spectrum), s_
        assert torch.equal(bt.spec_smooth[s_], ref.spec_smooth), s_
        np.testing.assert_allclose(mom[s_], ref.moments.cpu().numpy(),
                                   rtol=1e-12 if prec == "f64" else 1e-7, atol=1e-300)
        err = np.abs((gb[s_] - gr) * GRAD_SCALE) / max(np.max(np.abs(gr * GRAD_SCALE)), 1e-300)
        assert np.all(err <= (1e-12 if prec == "f64" else 1e-6)), (s_, lasers[s_].variant, err)


# ---------------------------------------------------------------------------
# whole-beam integration
# ---------------------------------------------------------------------------

def gout_bound(ref, prec):
    """Per-sample absolute error bound of gamma_out = mu + sqrt(V) xi7: that
    of mu plus half the relative error of V times |gamma_out - mu|."""
    tol = TOL[prec]
    sv = math.sqrt(max(float(np.max(ref["V"])), 1e-300)) if len(ref) else 0.0
    return tol["mu"] * np.abs(ref["mu"]) + 0.5 * tol["V"] * np.abs(ref["gamma_out"] - ref["mu"]) \
        + 1e-3 * tol["V"] * sv + 1e-300


def edge_weights(inputs, prec):
    """Weight of the samples whose oracle energy, or divergence-map angle,
    lies within the path's per-sample error bound of a bin edge.  Such a
    sample may land in the neighbouring bin, which moves 2 w of L1 mass; all
    other samples must land in the oracle's bin."""
    L, beam, bins, xi, w = inputs
    rec = oracle.evaluate(L, beam, bins, f64(xi))
    ww = np.ones(len(rec)) if w is None else np.asarray(w, dtype=np.float64)
    near_e = np.zeros(len(rec), dtype=bool)
    near_m = np.zeros(len(rec), dtype=bool)
    if bins.n_bins > 0:
        near_e = ~away_from_edges(rec["gamma_out"], gout_bound(rec, prec), bins)
    if bins.n_tx > 0 and bins.n_ty > 0:
        rel = 2.0 ** -19 if prec == "f32" else 1e-13
        tm = bins.theta_max
        for t, nc in ((rec["theta_x"], bins.n_tx), (rec["theta_y"], bins.n_ty)):
            sc = nc / (2.0 * tm)
            f = (t + tm) * sc
            d = rel * (np.abs(t) + np.abs(rec["theta_e"]) + tm * 1e-9) * sc
            near_m |= np.abs(f - np.round(f)) <= d
    return float(ww[near_e].sum()), float(ww[near_m].sum())


def compare_scatter(out, ref, prec, W, inputs=None):
    """Moments within MOM_TOL; histograms within 1e-4 of the weight in L1,
    plus twice the weight of near-edge samples when ``inputs`` (laser, beam,
    bins, xi, w) are given."""
    e_w, m_w = edge_weights(inputs, prec) if inputs is not None else (0.0, 0.0)
    res = out.result()
    m = res["moments"]
    keys = ("W", "mean", "spread", "rel_spread", "div_x", "div_y", "div", "mean_aeff",
            "mean_gamma0")
    errs = {k: abs(m[k] - ref["moments"][k]) / max(abs(ref["moments"][k]), 1e-300) for k in keys}
    spec = res["spectrum"].cpu().numpy()
    l1 = np.abs(spec - ref["spectrum"]).sum() + abs(m["under"] - ref["moments"]["under"]) + \
        abs(m["over"] - ref["moments"]["over"])
    print(f"[{prec}] moment rel errors:", errs, "spectrum L1/W:", l1 / W,
          "near-edge weight (energy, map):", e_w, m_w)
    for k in keys:
        assert errs[k] <= MOM_TOL[prec], (k, m[k], ref["moments"][k])
    assert l1 <= 1e-4 * W + 2.0 * e_w, (l1 / W, e_w)
    assert e_w <= 1e-2 * W
    if ref["divmap"].size:
        dm = res["divmap"].cpu().numpy().reshape(ref["divmap"].shape)
        assert np.abs(dm - ref["divmap"]).sum() <= 1e-4 * W + 2.0 * m_w
        assert m_w <= 1e-2 * W
    if ref["aeff_hist"].size:
        assert np.abs(res["aeff_hist"].cpu().numpy() - ref["aeff_hist"]).sum() <= 1e-4 * W
    assert m["nonfinite"] == 0
    return res


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("model", [I.MODEL_LL, I.MODEL_QFP])
@pytest.mark.parametrize("weighted", [False, True])
def test_scatter_matches_oracle(prec, model, weighted):
    n = 5003
    wl, L, xi = cfg2(n, model=model)
    w = I.rng(7).uniform(0.25, 2.0, n).astype(np.float32) if weighted else None
    xt, wt = dev(xi, w)
    out = qs_scatter(L, wl.beam, xt, wl.bins, w=wt, precision=prec)
    torch.cuda.synchronize()
    ref = oracle.scatter(L, wl.beam, wl.bins, f64(xi), None if w is None else w.astype(np.float64))
    W = float(n if w is None else w.astype(np.float64).sum())
    res = compare_scatter(out, ref, prec, W, inputs=(L, wl.beam, wl.bins, xi, w))
    if not weighted:
        # unit weights: histogram entries are integer counts
        spec = res["spectrum"].cpu().numpy()
        assert np.array_equal(spec, np.round(spec))


@pytest.mark.parametrize("weighted", [False, True])
def test_ll_f32_aligned_and_unaligned_streams_agree(weighted):
    """The FP32 classical path reads 16-byte-aligned FP32 streams four
    samples at a time and other streams one at a time; both give the same
    integer histograms (moments within the FP32 path's partition bar)."""
    n = 4 * 3001 + 3
    wl, L, xi = cfg2(n, model=I.MODEL_LL)
    w = I.rng(9).uniform(0.25, 2.0, n).astype(np.float32) if weighted else None
    xa, wa = dev(xi, w)

    def shifted(a):                       # same values at a 4-byte offset
        t = torch.empty(a.numel() + 1, dtype=a.dtype, device=a.device)
        t[1:] = a
        return t[1:]

    xu = [None if a is None else shifted(a) for a in xa]
    wu = None if wa is None else shifted(wa)
    assert xu[0].data_ptr() % 16 == 4
    oa = qs_scatter(L, wl.beam, xa, wl.bins, w=wa, precision="f32")
    ou = qs_scatter(L, wl.beam, xu, wl.bins, w=wu, precision="f32")
    torch.cuda.synchronize()
    assert torch.equal(oa.spectrum, ou.spectrum)
    assert torch.equal(oa.divmap, ou.divmap)
    assert torch.equal(oa.aeff_hist, ou.aeff_hist)
    np.testing.assert_allclose(oa.moments.cpu().numpy(), ou.moments.cpu().numpy(), rtol=1e-8)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("model", [I.MODEL_LL, I.MODEL_QFP])
@pytest.mark.parametrize("sigma", [0.3, 5.5])
def test_smoothed_spectrum_windows_narrow_and_wider_than_a_warp(prec, model, sigma):
    """Kernel-smoothed spectrum against the oracle for a window of a few bins
    and one of 67 bins (more than one pass of 32 lanes), ragged n."""
    n = 777
    wl, L, xi = cfg2(n, model=model, n_phase=64)
    bins = I.Bins(**{**wl.bins.__dict__, "smooth_sigma_bins": sigma})
    xt, _ = dev(xi)
    out = qs_scatter(L, wl.beam, xt, bins, precision=prec)
    torch.cuda.synchronize()
    ref = oracle.smooth_spectrum(L, wl.beam, bins, sigma, f64(xi))
    S = out.spec_smooth.cpu().numpy()
    l1 = np.abs(S - ref).sum() / n
    print(f"[{prec}, model {model}, sigma {sigma}] smoothed L1/W:", l1)
    # fixed-point rounding: at most half a unit of 2^-32 per deposit; FP32:
    # a kernel moved by eps bins changes by at most 2 eps / (sigma sqrt(2 pi))
    # in L1, eps from the path's per-sample bound on gamma_out
    eps = TOL["f32"]["mu"] * bins.hi * bins.n_bins / (bins.hi - bins.lo)
    bound = 1e-12 if prec == "f64" else 2 * eps / (sigma * math.sqrt(2 * math.pi))
    assert l1 <= bound + 13 * sigma * 2.0 ** -32
    assert abs(S.sum() - ref.sum()) <= 1e-5 * n


def test_gauss_hermite_tiny_config_f64():
    """32^3 Gauss-Hermite nodes, LL model, 256-bin spectrum, weighted FP64."""
    wl = I.tiny_gauss_hermite()
    xi, w = I.workload_inputs(wl)
    xt, wt = dev(xi, w)
    out = qs_scatter(wl.laser, wl.beam, xt, wl.bins, w=wt, precision="f64", weight_frac_bits=48)
    torch.cuda.synchronize()
    ref = oracle.scatter(wl.laser, wl.beam, wl.bins, xi, w)
    compare_scatter(out, ref, "f64", float(w.sum()))
    # fixed-point weights: every bin within n * 2^-49 of the oracle's mass
    spec = out.spectrum.cpu().numpy()
    assert np.max(np.abs(spec - ref["spectrum"])) <= len(w) * 2.0 ** -49 + 1e-15


def test_broadband_log_bins_flat_energy():
    wl = I.broadband_qfp(4099)
    L = I.Laser(**{**wl.laser.__dict__, "n_phase": 256})
    xi, _ = I.workload_inputs(wl, 4099)
    xt, _ = dev(xi)
    for prec in ("f64", "f32"):
        out = qs_scatter(L, wl.beam, xt, wl.bins, precision=prec)
        rec = qs_eval_samples(L, wl.beam, xt, wl.bins, precision=prec)
        torch.cuda.synchronize()
        ref = oracle.scatter(L, wl.beam, wl.bins, f64(xi))
        compare_scatter(out, ref, prec, 4099.0, inputs=(L, wl.beam, wl.bins, xi, None))
        compare_samples(rec, oracle.evaluate(L, wl.beam, wl.bins, f64(xi)), prec, wl.bins)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_empty_input():
    wl, L, xi = cfg2(4)
    xt = [torch.empty(0, dtype=torch.float32, device="cuda") for _ in range(8)]
    out = qs_scatter(L, wl.beam, xt, wl.bins)
    torch.cuda.synchronize()
    assert all(v == 0 for v in out.moments.cpu().tolist())
    assert float(out.spectrum.abs().sum()) == 0 and float(out.divmap.abs().sum()) == 0


@pytest.mark.parametrize("n", [1, 31, 255, 256, 257])
def test_tiny_and_ragged_sizes(n):
    wl, L, xi = cfg2(n)
    xt, _ = dev(xi)
    out = qs_scatter(L, wl.beam, xt, wl.bins, precision="f64")
    torch.cuda.synchronize()
    compare_scatter(out, oracle.scatter(L, wl.beam, wl.bins, f64(xi)), "f64", float(n))


def test_zero_intensity_is_identity():
    wl, L, xi = cfg2(3000, a0=0.0)
    xt, _ = dev(xi)
    for prec in ("f64", "f32"):
        rec = qs_eval_samples(L, wl.beam, xt, wl.bins, precision=prec)
        assert torch.equal(rec["mu"], rec["gamma0"])
        assert float(rec["V"].abs().max()) == 0.0
    out = qs_scatter(L, wl.beam, xt, wl.bins, precision="f64")
    g0 = rec["gamma0"].cpu().numpy()
    h, _ = np.histogram(g0, bins=wl.bins.n_bins, range=(wl.bins.lo, wl.bins.hi))
    assert np.array_equal(out.spectrum.cpu().numpy(), h.astype(float))


@pytest.mark.parametrize("n_phase", [1, 4096])
def test_phase_count_limits(n_phase):
    wl, L, xi = cfg2(600, n_phase=n_phase)
    xt, _ = dev(xi)
    rec = qs_eval_samples(L, wl.beam, xt, wl.bins, precision="f64")
    compare_samples(rec, oracle.evaluate(L, wl.beam, wl.bins, f64(xi)), "f64", wl.bins)


def test_large_map_uses_global_accumulators():
    """A 700x700 divergence map does not fit in shared memory."""
    wl, L, xi = cfg2(3001)
    bins = I.Bins(**{**wl.bins.__dict__, "n_tx": 700, "n_ty": 700})
    xt, _ = dev(xi)
    for prec in ("f64", "f32"):
        out = qs_scatter(L, wl.beam, xt, bins, precision=prec)
        torch.cuda.synchronize()
        compare_scatter(out, oracle.scatter(L, wl.beam, bins, f64(xi)), prec, 3001.0,
                        inputs=(L, wl.beam, bins, xi, None))


def test_everything_outside_the_bins():
    wl, L, xi = cfg2(1000)
    bins = I.Bins(n_bins=16, lo=1e6, hi=2e6, n_tx=8, n_ty=8, theta_max=1e-9, n_aeff=4,
                  aeff_max=1e-12)
    xt, _ = dev(xi)
    out = qs_scatter(L, wl.beam, xt, bins, precision="f64")
    m = out.moments_dict()
    assert m["under"] == 1000 and m["over"] == 0 and m["map_out"] == 1000
    assert float(out.spectrum.sum()) == 0 and float(out.aeff_hist.sum()) == 0


def test_zero_and_tiny_weights():
    n = 2000
    wl, L, xi = cfg2(n)
    w = I.rng(8).uniform(0, 1, n)
    w[::3] = 0.0
    w = w.astype(np.float32)
    xt, wt = dev(xi, w)
    out = qs_scatter(L, wl.beam, xt, wl.bins, w=wt, precision="f64")
    torch.cuda.synchronize()
    ref = oracle.scatter(L, wl.beam, wl.bins, f64(xi), w.astype(np.float64))
    compare_scatter(out, ref, "f64", float(w.astype(np.float64).sum()))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_weight_fixed_point_rounds_to_nearest_even(prec):
    """Weights enter the integer histograms as round-to-nearest-even of
    w 2^bits.  With 4 fraction bits and weights k/64 every quarter (ties
    included) occurs; the histogram totals equal the host's rounding exactly,
    and a weight above 2^59 saturates at 2^63 - 1 units."""
    n = 4096
    wl, L, xi = cfg2(n, n_phase=16)
    k = I.rng(12).integers(0, 1 << 16, n)
    k[:8] = [0, 1, 2, 3, 4, 5, 6, 7]                      # 0, 1/4, 1/2, 3/4, ... of a unit
    w = (k / 64.0).astype(np.float32)
    xt, wt = dev(xi, w)
    out = qs_scatter(L, wl.beam, xt, wl.bins, w=wt, precision=prec, weight_frac_bits=4)
    torch.cuda.synchronize()
    m = out.moments_dict()
    expect = np.rint(k / 4.0).sum() / 16.0                 # numpy rint: ties to even
    total = float(out.spectrum.double().sum()) + m["under"] + m["over"]
    assert total == expect
    assert float(out.aeff_hist.double().sum()) <= expect
    # saturation: one sample carrying 2^60 at 4 fraction bits
    w1 = np.zeros(n, dtype=np.float32)
    w1[0] = 2.0 ** 60
    xt, wt = dev(xi, w1)
    out = qs_scatter(L, wl.beam, xt, wl.bins, w=wt, precision=prec, weight_frac_bits=4)
    torch.cuda.synchronize()
    m = out.moments_dict()
    total = float(out.spectrum.double().sum()) + m["under"] + m["over"]
    assert total == float((1 << 63) - 1) / 16.0


def test_nonfinite_samples_are_excluded_and_counted():
    n = 1000
    wl, L, xi = cfg2(n)
    xi = [a.copy() for a in xi]
    xi[0][[3, 500]] = np.nan
    xt, _ = dev(xi)
    out = qs_scatter(L, wl.beam, xt, wl.bins, precision="f64")
    m = out.moments_dict()
    assert m["nonfinite"] == 2 and m["W"] == n - 2


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("model", [I.MODEL_LL, I.MODEL_QFP])
def test_nonfinite_y_angle_alone_is_excluded(prec, model):
    """A sample whose only non-finite input is the y-angle variate is left
    out of every output and counted, as any other non-finite sample (it
    would otherwise make div_y and div NaN)."""
    n = 1000
    wl, L, xi = cfg2(n, model=model)
    xi = [a.copy() for a in xi]
    xi[5][[7, 600]] = np.nan
    xi[4][[11]] = np.inf
    xt, _ = dev(xi)
    out = qs_scatter(L, wl.beam, xt, wl.bins, precision=prec)
    m = out.moments_dict()
    assert m["nonfinite"] == 3 and m["W"] == n - 3
    assert all(math.isfinite(m[k]) for k in ("div_x", "div_y", "div", "mean", "spread"))
    keep = np.ones(n, dtype=bool)
    keep[[7, 600, 11]] = False
    ref = oracle.scatter(L, wl.beam, wl.bins, [a[keep] for a in f64(xi)])
    for k in ("mean", "spread", "div_x", "div_y"):
        assert abs(m[k] / ref["moments"][k] - 1) <= MOM_TOL[prec], k


def test_check_finite_flag_reports_excluded_samples():
    """QS_EXEC_CHECK_FINITE: the call waits, writes every output and returns
    QS_ERR_NONFINITE when samples were excluded; QS_OK otherwise; refused
    (before any launch) on a stream that is being captured."""
    n = 2000
    wl, L, xi = cfg2(n)
    xt, _ = dev(xi)
    out = B.Outputs(wl.bins, n)
    qs_scatter(L, wl.beam, xt, wl.bins, out=out, check_finite=True)      # clean: no error
    clean = out.moments.clone()
    bad = [a.copy() for a in xi]
    bad[3][[5]] = np.nan
    bt, _ = dev(bad)
    with pytest.raises(QsError) as e:
        qs_scatter(L, wl.beam, bt, wl.bins, out=out, check_finite=True)
    assert e.value.status == B.QS_ERR_NONFINITE
    m = out.moments_dict()                      # outputs written all the same
    assert m["nonfinite"] == 1 and m["W"] == n - 1 and m["mean"] != 0.0
    assert not torch.equal(out.moments, clean)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(QsError) as e2:
        with torch.cuda.graph(g, stream=s):
            qs_scatter(L, wl.beam, xt, wl.bins, out=out, check_finite=True, stream=s)
    assert e2.value.status == B.QS_ERR_UNSUPPORTED
    torch.cuda.synchronize()


def test_workspace_too_small_is_rejected():
    wl, L, xi = cfg2(100)
    xt, _ = dev(xi)
    out = B.Outputs(wl.bins, 100)
    out.ws_bytes = 64
    with pytest.raises(QsError) as e:
        qs_scatter(L, wl.beam, xt, wl.bins, out=out)
    assert e.value.status == B.QS_ERR_WORKSPACE


# ---------------------------------------------------------------------------
# determinism, launch shapes, graph capture
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_repeated_calls_are_bit_identical(prec):
    wl, L, xi = cfg2(20000)
    xt, _ = dev(xi)
    a = qs_scatter(L, wl.beam, xt, wl.bins, precision=prec)
    ma, sa = a.moments.clone(), a.spectrum.clone()
    b = qs_scatter(L, wl.beam, xt, wl.bins, precision=prec)
    assert torch.equal(ma, b.moments) and torch.equal(sa, b.spectrum)


@pytest.mark.parametrize("block,grid", [(64, 3), (128, 0), (512, 0), (256, 1000)])
def test_launch_shapes_agree(block, grid):
    wl, L, xi = cfg2(9000)
    xt, _ = dev(xi)
    ref = qs_scatter(L, wl.beam, xt, wl.bins, precision="f32")
    o = qs_scatter(L, wl.beam, xt, wl.bins, precision="f32", block=block, grid=grid)
    assert torch.equal(ref.spectrum, o.spectrum) and torch.equal(ref.divmap, o.divmap)
    rm, om = ref.moments.cpu().numpy(), o.moments.cpu().numpy()
    # per-thread compensated FP32 sums over a different partition of samples
    np.testing.assert_allclose(om, rm, rtol=1e-8)


@pytest.mark.parametrize("weighted", [False, True])
def test_classical_launch_shapes_agree(weighted):
    """The FP32 classical path's default launch (one 768-thread CTA per SM)
    against caller-chosen shapes (256 and 512 threads, a small grid): the
    same integer histograms, moments within the FP32 path's partition bar."""
    n = 4 * 50001 + 3
    wl, L, xi = cfg2(n, model=I.MODEL_LL)
    w = I.rng(19).uniform(0.25, 2.0, n).astype(np.float32) if weighted else None
    xt, wt = dev(xi, w)
    ref = qs_scatter(L, wl.beam, xt, wl.bins, w=wt, precision="f32")
    for block, grid in ((256, 0), (512, 0), (256, 7)):
        o = qs_scatter(L, wl.beam, xt, wl.bins, w=wt, precision="f32", block=block, grid=grid)
        torch.cuda.synchronize()
        assert torch.equal(ref.spectrum, o.spectrum), (block, grid)
        assert torch.equal(ref.divmap, o.divmap), (block, grid)
        assert torch.equal(ref.aeff_hist, o.aeff_hist), (block, grid)
        np.testing.assert_allclose(o.moments.cpu().numpy(), ref.moments.cpu().numpy(), rtol=1e-8)


def test_graph_capture_replay():
    wl, L, xi = cfg2(8000)
    xt, _ = dev(xi)
    out = B.Outputs(wl.bins, 8000)
    qs_scatter(L, wl.beam, xt, wl.bins, out=out)      # warm-up (first-use set-up)
    torch.cuda.synchronize()
    ref_m = out.moments.clone()
    out.moments.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        qs_scatter(L, wl.beam, xt, wl.bins, out=out, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.moments, ref_m)


# ---------------------------------------------------------------------------
# full-size workload (2^26 samples, QFP, 512 phase steps), as benchmarked
# ---------------------------------------------------------------------------

@pytest.mark.slow
def test_full_size_quantum_workload_sampled_parity():
    wl = I.full_qfp()
    n = wl.n
    xi, _ = I.workload_inputs(wl)
    xt, _ = dev(xi)
    out = qs_scatter(wl.laser, wl.beam, xt, wl.bins, precision="f32")
    rec = qs_eval_samples(wl.laser, wl.beam, xt, wl.bins, precision="f32")
    torch.cuda.synchronize()
    m = out.moments_dict()
    # weight conservation at full size
    assert m["W"] == n and m["nonfinite"] == 0
    assert float(out.spectrum.sum()) + m["under"] + m["over"] == n
    assert float(out.divmap.sum()) + m["map_out"] == n
    # the fused histogram equals the histogram of the per-sample records
    b = rec["bin"].long()
    cnt = torch.bincount(b.clamp(min=0, max=wl.bins.n_bins - 1)[(b >= 0) & (b < wl.bins.n_bins)],
                         minlength=wl.bins.n_bins)
    assert torch.equal(cnt.double(), out.spectrum)
    # fused moments equal moments of the per-sample records up to the FP32
    # path's compensated per-thread accumulation
    mu = rec["mu"]
    mean = float(mu.mean())
    var = float(((mu - mean) ** 2).mean() + rec["V"].mean())
    assert abs(m["mean"] / mean - 1) < 1e-8
    assert abs(m["spread"] / math.sqrt(var) - 1) < 1e-8
    # sampled per-sample parity with the oracle across the whole index range
    idx = np.unique(np.concatenate([np.arange(64), n - 1 - np.arange(64),
                                    I.rng(9).integers(0, n, 1024)]))
    sub = [a[idx].astype(np.float64) for a in xi]
    ref = oracle.evaluate(wl.laser, wl.beam, wl.bins, sub)
    got = {k: v[torch.from_numpy(idx).cuda()] for k, v in rec.items()}
    compare_samples(got, ref, "f32", wl.bins)


@pytest.mark.slow
def test_bench_workload_2p20_matches_oracle_at_the_stated_bars():
    """The benchmarked configuration (FP32, QFP, 512 cells, 512 energy
    bins, 128x128 map, 256 a_eff bins) on the first 2^20 samples of the bench
    workload, against the oracle's per-sample records reduced by their plain
    definitions: spectrum L1 <= 1e-4 of the total weight with no allowance
    for samples near a bin edge, moments within 1e-5, the energy bin of every
    sample farther than its error bound from an edge bit-exact (the fused
    histogram is compared as a whole, the per-sample records element by
    element)."""
    import oracle_pool
    n = 1 << 20
    wl = I.full_qfp(n)
    xi, _ = I.workload_inputs(wl, n)
    xt, _ = dev(xi)
    out = qs_scatter(wl.laser, wl.beam, xt, wl.bins, precision="f32")
    rec = qs_eval_samples(wl.laser, wl.beam, xt, wl.bins, precision="f32")
    torch.cuda.synchronize()
    ref = oracle_pool.records(wl.laser, wl.beam, wl.bins, f64(xi))
    bins = wl.bins
    # the oracle's histogram and moments from its records (half-open bins,
    # law of total variance, Eq. 8 term on x)
    b = ref["bin"]
    hist = np.bincount(b[(b >= 0) & (b < bins.n_bins)], minlength=bins.n_bins).astype(float)
    under, over = float((b < 0).sum()), float((b >= bins.n_bins).sum())
    mean = ref["mu"].mean()
    spread = math.sqrt(((ref["mu"] - mean) ** 2).mean() + ref["V"].mean())
    thx0 = wl.beam.div_rad * xi[4].astype(np.float64)
    thy0 = wl.beam.div_rad * xi[5].astype(np.float64)
    div_x = math.sqrt((thx0 ** 2 + ref["theta_e"] ** 2).mean())
    div_y = math.sqrt((thy0 ** 2).mean())
    expect = dict(W=float(n), mean=mean, spread=spread, rel_spread=spread / mean, div_x=div_x,
                  div_y=div_y, div=math.hypot(div_x, div_y), mean_aeff=ref["aeff"].mean(),
                  mean_gamma0=ref["gamma0"].mean())
    m = out.moments_dict()
    errs = {k: abs(m[k] / v - 1) for k, v in expect.items()}
    spec = out.spectrum.cpu().numpy()
    l1 = np.abs(spec - hist).sum() + abs(m["under"] - under) + abs(m["over"] - over)
    print("moment rel errors:", errs, "spectrum L1/W:", l1 / n)
    assert m["nonfinite"] == 0
    for k, e in errs.items():
        assert e <= MOM_TOL["f32"], (k, m[k], expect[k])
    assert l1 <= 1e-4 * n, l1 / n
    # divergence map and a_eff histogram at the same bar
    ix, iy = ref["ix"], ref["iy"]
    inmap = ix >= 0
    dm = np.bincount((iy * bins.n_tx + ix)[inmap], minlength=bins.n_tx * bins.n_ty)
    got_dm = out.divmap.cpu().numpy().reshape(-1)
    assert np.abs(got_dm - dm).sum() + abs(m["map_out"] - (~inmap).sum()) <= 1e-4 * n
    ah = np.bincount(ref["abin"][ref["abin"] < bins.n_aeff], minlength=bins.n_aeff)
    assert np.abs(out.aeff_hist.cpu().numpy() - ah).sum() <= 1e-4 * n
    # every sample farther than its error bound from an energy-bin edge lands
    # in the oracle's bin
    g = rec["bin"].cpu().numpy()
    ok = away_from_edges(ref["gamma_out"], gout_bound(ref, "f32"), bins)
    print("samples near an energy-bin edge:", int((~ok).sum()), "moved:", int((g != b).sum()))
    np.testing.assert_array_equal(g[ok], b[ok])


def test_unit_rates_probe():
    """The unit-rate probe reports plausible per-SM-per-clock rates."""
    r = B.unit_rates()
    print("unit rates:", r)
    assert r["sms"] > 0 and r["sm_max_mhz"] > 0
    assert r["fma"] > 64 and r["lg2"] > 8 and r["ex2"] >= 0.9 * r["lg2"] and r["rcp"] > 8
    assert 0 < r["dfma"] < r["fma"]
    # the packed f32x2 FMA, in lane-operations (two per instruction)
    print("packed / scalar FMA lane rate:", r["fma2"] / r["fma"])
    assert 0.5 * r["fma"] <= r["fma2"] <= 2.5 * r["fma"]
