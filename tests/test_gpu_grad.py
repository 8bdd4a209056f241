"""Adjoint (qs_scatter_grad) and smoothed spectrum vs the oracle and vs
central finite differences of the GPU forward, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2308_09348_gb300 import binding as B
from paper_2308_09348_gb300 import inputs as I
from paper_2308_09348_gb300 import fit as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_09348_gb300 import build
    build.build()


def _setup(n, model, n_phase=64, weighted=True):
    wl = I.fit_qfp(n)
    L = I.Laser(**{**wl.laser.__dict__, "model": model, "n_phase": n_phase})
    xi, _ = I.workload_inputs(wl, n)
    w = I.rng(41).uniform(0.5, 1.5, n).astype(np.float32) if weighted else None
    return wl, L, wl.beam, wl.bins, xi, w


def _upstream(nb, seed=42):
    rg = I.rng(seed)
    dm = np.zeros(13)
    for k, sc in (("mean", 1e-3), ("spread", 1e-3), ("rel_spread", 1.0), ("div_x", 1e3),
                  ("div_y", 1e3), ("div", 1e3), ("mean_aeff", 1.0), ("mean_gamma0", 1e-3)):
        dm[B.MOMENT_FIELDS.index(k)] = rg.normal() * sc
    dS = rg.normal(size=nb) * 1e-3
    return dm, dS


def _dev(xi, w):
    xt = [torch.from_numpy(a).cuda() for a in xi]
    wt = None if w is None else torch.from_numpy(w).cuda()
    return xt, wt


def _gpu_grad(L, Bm, bins, xt, wt, dm, dS, prec):
    out = B.qs_scatter(L, Bm, xt, bins, w=wt, precision=prec)
    g = B.qs_scatter_grad(L, Bm, xt, bins, out.moments, torch.from_numpy(dm),
                          torch.from_numpy(dS), w=wt, precision=prec, out=out)
    torch.cuda.synchronize()
    return g.cpu().numpy(), out


SCALE = np.array([20.0, 4.0, 1.0, 1.0, 10.0, 6000.0, 0.08, 1e-3])


# FP32 adjoint against the oracle's gradient, parameter-scaled, relative to
# the largest component: measured ~5e-7 (FP32 tangents over 512 cells)
GRAD_TOL = {"f64": 1e-10, "f32": 1e-5}


@pytest.mark.parametrize("model,n_phase", [(I.MODEL_LL, 64), (I.MODEL_QFP, 64),
                                           (I.MODEL_QFP, 512), (I.MODEL_QFP, 509)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gradient_matches_oracle(model, n_phase, prec):
    n = 3001
    wl, L, Bm, bins, xi, w = _setup(n, model, n_phase=n_phase)
    xt, wt = _dev(xi, w)
    dm, dS = _upstream(bins.n_bins)
    g, out = _gpu_grad(L, Bm, bins, xt, wt, dm, dS, prec)
    ref = oracle.grad(L, Bm, bins, bins.smooth_sigma_bins, [a.astype(np.float64) for a in xi],
                      w.astype(np.float64), dL_dm=dm, dL_dS=dS)
    # compare in parameter-scaled units (dL/d ln theta-like)
    gs, rs = g * SCALE, ref["grad"] * SCALE
    err = np.abs(gs - rs) / np.max(np.abs(rs))
    print(f"[{prec}, model {model}] scaled grad rel err per param:", err)
    assert np.all(err <= GRAD_TOL[prec]), err
    # forward smoothed spectrum against the oracle
    S = out.spec_smooth.cpu().numpy()
    l1 = np.abs(S - ref["smooth"]).sum() / w.astype(np.float64).sum()
    print(f"[{prec}] smoothed spectrum L1/W:", l1)
    assert l1 <= (1e-12 if prec == "f64" else 1e-5) + n * 2.0 ** -32 * 25 / w.sum()


def test_fp32_gradient_with_a_spectrum_too_large_to_stage():
    """FP32 adjoint over a 9000-bin smoothed spectrum (upstream gradient read
    from global memory instead of the shared-memory stage) vs the oracle."""
    n = 2001
    wl, L, Bm, bins, xi, w = _setup(n, I.MODEL_QFP)
    bins = I.Bins(**{**bins.__dict__, "n_bins": 9000})
    xt, wt = _dev(xi, w)
    dm, dS = _upstream(bins.n_bins, seed=44)
    g, _ = _gpu_grad(L, Bm, bins, xt, wt, dm, dS, "f32")
    ref = oracle.grad(L, Bm, bins, bins.smooth_sigma_bins, [a.astype(np.float64) for a in xi],
                      w.astype(np.float64), dL_dm=dm, dL_dS=dS)
    gs, rs = g * SCALE, ref["grad"] * SCALE
    err = np.abs(gs - rs) / np.max(np.abs(rs))
    print("[f32, 9000 bins] scaled grad rel err per param:", err)
    # the FP32 bin coordinate t < 9000 of a sample carries up to 2^-11 bins of
    # rounding (ulp at 2^13), which the smoothed spectrum's derivative turns
    # into a relative error of that order over sigma = 2 bins (measured 2.3e-4)
    assert np.all(err <= 5e-4), err


def test_fp64_adjoint_vs_central_differences_of_gpu_forward():
    """FP64 adjoint vs Richardson central differences of the FP64 GPU forward
    (h = 1e-4 of each parameter's scale, same samples): rel <= 1e-6."""
    n = 2000
    wl, L, Bm, bins, xi, w = _setup(n, I.MODEL_QFP)
    xt, wt = _dev(xi, w)
    dm, dS = _upstream(bins.n_bins, seed=43)
    g, _ = _gpu_grad(L, Bm, bins, xt, wt, dm, dS, "f64")
    prob = F.Problem(L, Bm, bins, xt, wt, "f64")
    theta = prob.theta_of()

    def loss(th):
        lz, bm = prob.descriptors(th)
        # fine fixed point for the smoothed deposits keeps rounding steps out of the FD
        o = B.qs_scatter(lz, bm, xt, bins, w=wt, precision="f64", weight_frac_bits=48)
        return float((o.moments.cpu().numpy() * dm).sum() + (o.spec_smooth.cpu().numpy() * dS).sum())

    for k in range(8):
        h = 1e-4 * SCALE[k]

        def D(hh):
            tp, tm = theta.clone(), theta.clone()
            tp[k] += hh
            tm[k] -= hh
            return (loss(tp) - loss(tm)) / (2 * hh)

        fd = (4 * D(h / 2) - D(h)) / 3
        assert abs(g[k] - fd) * SCALE[k] <= 1e-6 * np.max(np.abs(g * SCALE)), (k, g[k], fd)


def test_fp32_adjoint_vs_central_differences_h1e4():
    """FP32 adjoint vs plain central differences (h = 1e-4 relative) of the
    FP32 forward, common random numbers, with the upstream gradient on the
    moments and on the smoothed spectrum."""
    n = 1 << 16
    wl, L, Bm, bins, xi, w = _setup(n, I.MODEL_QFP, n_phase=128, weighted=False)
    xt, wt = _dev(xi, None)
    dm, dS = _upstream(bins.n_bins, seed=44)
    g, _ = _gpu_grad(L, Bm, bins, xt, wt, dm, dS, "f32")
    prob = F.Problem(L, Bm, bins, xt, None, "f32")
    theta = prob.theta_of()

    def loss(th):
        lz, bm = prob.descriptors(th)
        o = B.qs_scatter(lz, bm, xt, bins, precision="f32")
        return float((o.moments.cpu().numpy() * dm).sum() + (o.spec_smooth.cpu().numpy() * dS).sum())

    errs = []
    for k in range(8):
        h = 1e-4 * SCALE[k]
        tp, tm = theta.clone(), theta.clone()
        tp[k] += h
        tm[k] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        errs.append(abs(g[k] - fd) * SCALE[k] / np.max(np.abs(g * SCALE)))
    print("fp32 adjoint vs FD, scaled rel err:", errs)
    assert max(errs) <= 1e-3


def test_gradient_is_deterministic():
    n = 5000
    wl, L, Bm, bins, xi, w = _setup(n, I.MODEL_QFP)
    xt, wt = _dev(xi, w)
    dm, dS = _upstream(bins.n_bins)
    g1, _ = _gpu_grad(L, Bm, bins, xt, wt, dm, dS, "f32")
    g2, _ = _gpu_grad(L, Bm, bins, xt, wt, dm, dS, "f32")
    assert np.array_equal(g1, g2)


def test_autograd_function_backward_equals_c_abi():
    n = 4000
    wl, L, Bm, bins, xi, w = _setup(n, I.MODEL_QFP)
    xt, wt = _dev(xi, w)
    prob = F.Problem(L, Bm, bins, xt, wt, "f64")
    theta = prob.theta_of().requires_grad_(True)
    mom, S = F.ScatterFn.apply(theta, prob)
    dm, dS = _upstream(bins.n_bins, seed=45)
    L_ = (mom.cpu() * torch.from_numpy(dm)).sum() + (S.cpu() * torch.from_numpy(dS)).sum()
    L_.backward()
    g_ref, _ = _gpu_grad(L, Bm, bins, xt, wt, dm, dS, "f64")
    np.testing.assert_allclose(theta.grad.numpy(), g_ref, rtol=1e-12, atol=0)


def test_fit_recovers_hidden_parameters():
    """Adam on the smoothed spectrum and moments of a synthetic shot moves
    perturbed parameters back towards the hidden ones."""
    n = 1 << 15
    wl, L, Bm, bins, xi, w = _setup(n, I.MODEL_QFP, n_phase=128, weighted=False)
    xt, _ = _dev(xi, None)
    prob = F.Problem(L, Bm, bins, xt, None, "f32")
    hidden = prob.theta_of()
    tm, tS = F.ScatterFn.apply(hidden, prob)
    tm, tS = tm.detach().clone(), tS.detach().clone()
    start = hidden.clone()
    start[0] *= 1.15       # a0
    start[5] *= 0.95       # gamma_mean
    _, hist = F.fit(prob, start, tm, tS, steps=60, lr=0.01)
    print("fit loss history:", hist[0], hist[len(hist) // 2], hist[-1])
    assert hist[-1] < 0.2 * hist[0]
