"""Differentiable forward model and gradient fit (reconstruction of laser and
beam parameters from observables, the use the paper names in Sec. 6).

``ScatterFn`` is a ``torch.autograd.Function``: its forward runs qs_scatter
(moments + kernel-smoothed spectrum), its backward runs qs_scatter_grad, which
recomputes every sample with tangents instead of storing per-sample state.
The 8 parameters are (a0, w0_um, dx_um, dy_um, delay_fs, gamma_mean,
rel_spread, div_rad).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import torch

from . import binding as B
from . import inputs as I

PARAMS = B.GRAD_PARAMS
LASER_FIELDS = PARAMS[:5]
BEAM_FIELDS = PARAMS[5:]


@dataclass
class Problem:
    """Everything fixed during a fit: descriptor templates, samples, bins."""
    laser: I.Laser
    beam: I.Beam
    bins: I.Bins
    xi: list
    w: torch.Tensor | None = None
    precision: str = "f32"
    out: B.Outputs | None = None

    def descriptors(self, theta) -> tuple[I.Laser, I.Beam]:
        v = [float(x) for x in theta]
        lz = replace(self.laser, **dict(zip(LASER_FIELDS, v[:5])))
        bm = replace(self.beam, **dict(zip(BEAM_FIELDS, v[5:])))
        return lz, bm

    def theta_of(self, laser=None, beam=None) -> torch.Tensor:
        lz = laser or self.laser
        bm = beam or self.beam
        return torch.tensor([getattr(lz, k) for k in LASER_FIELDS] +
                            [getattr(bm, k) for k in BEAM_FIELDS], dtype=torch.float64)


class ScatterFn(torch.autograd.Function):
    """theta (8,) -> (moments (13,), smoothed spectrum (n_bins,))."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, prob: Problem):
        lz, bm = prob.descriptors(theta.detach().cpu())
        if prob.out is None:
            prob.out = B.Outputs(prob.bins, prob.xi[0].numel(), prob.xi[0].device, prob.precision)
        out = B.qs_scatter(lz, bm, prob.xi, prob.bins, w=prob.w, precision=prob.precision,
                           out=prob.out)
        mom = out.moments.clone()
        S = out.spec_smooth.clone()
        ctx.prob = prob
        ctx.desc = (lz, bm)
        ctx.save_for_backward(mom)
        ctx.theta_meta = (theta.dtype, theta.device)
        return mom, S

    @staticmethod
    def backward(ctx, g_mom, g_S):
        (mom,) = ctx.saved_tensors
        prob = ctx.prob
        lz, bm = ctx.desc
        if g_mom is None:
            g_mom = torch.zeros_like(mom)
        g = B.qs_scatter_grad(lz, bm, prob.xi, prob.bins, mom, g_mom, g_S, w=prob.w,
                              precision=prob.precision, out=prob.out)
        dt, dev = ctx.theta_meta
        return g.to(device=dev, dtype=dt), None


MOMENT_INDEX = {k: i for i, k in enumerate(B.MOMENT_FIELDS)}


def loss_fn(mom, S, target_mom, target_S, moment_weights: dict, spectrum_weight: float):
    """Weighted squared error of selected moments (relative) and of the
    smoothed spectrum (normalised by the target's total weight)."""
    L = torch.zeros((), dtype=torch.float64, device=mom.device)
    for k, c in moment_weights.items():
        i = MOMENT_INDEX[k]
        ref = target_mom[i]
        L = L + c * ((mom[i] - ref) / (ref.abs() + 1e-30)) ** 2
    if spectrum_weight and S.numel():
        norm = target_S.sum().clamp_min(1e-30)
        L = L + spectrum_weight * (((S - target_S) / norm) ** 2).sum() * S.numel()
    return L


DEFAULT_MOMENT_WEIGHTS = {"mean": 1.0, "spread": 1.0, "div_x": 1.0, "div_y": 1.0,
                          "mean_aeff": 1.0}


def fit(prob: Problem, theta0: torch.Tensor, target_mom, target_S, steps: int = 100,
        lr: float = 0.02, scale: torch.Tensor | None = None, moment_weights=None,
        spectrum_weight: float = 1.0, callback=None):
    """Adam on theta / scale (unit-free steps).  Returns (theta, history)."""
    mw = DEFAULT_MOMENT_WEIGHTS if moment_weights is None else moment_weights
    scale = theta0.abs().clamp_min(1e-12) if scale is None else scale
    z = (theta0 / scale).clone().requires_grad_(True)
    opt = torch.optim.Adam([z], lr=lr)
    hist = []
    for it in range(steps):
        opt.zero_grad()
        mom, S = ScatterFn.apply(z * scale, prob)
        L = loss_fn(mom, S, target_mom, target_S, mw, spectrum_weight)
        L.backward()
        opt.step()
        hist.append(float(L.detach()))
        if callback is not None:
            callback(it, z.detach() * scale, float(L.detach()))
    return (z.detach() * scale), hist


# ---- many shots at once ------------------------------------------------------

@dataclass
class BatchProblem:
    """Everything fixed during a batched fit: the device descriptors, outputs
    and workspace of one batch (``binding.Batch``, whose bins carry the
    smoothing width), the concatenated samples and their weights."""
    batch: B.Batch
    xi: list
    w: torch.Tensor | None = None


class BatchScatterFn(torch.autograd.Function):
    """theta (n_shots, 8) -> (moments (n_shots, 13), smoothed spectra
    (n_shots, n_bins)): forward qs_scatter_batch, backward
    qs_scatter_grad_batch (every sample recomputed with tangents)."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, prob: BatchProblem):
        bt = prob.batch
        th = theta.detach().to(bt.moments.device, torch.float64)
        bt.set_params(th)
        bt.run(prob.xi, prob.w)
        mom = bt.moments.clone()
        S = bt.spec_smooth.clone()
        ctx.prob = prob
        ctx.save_for_backward(th.clone(), mom)
        ctx.theta_meta = (theta.dtype, theta.device)
        return mom, S

    @staticmethod
    def backward(ctx, g_mom, g_S):
        th, mom = ctx.saved_tensors
        prob = ctx.prob
        bt = prob.batch
        bt.set_params(th)           # the descriptors of this forward
        if g_mom is None:
            g_mom = torch.zeros_like(mom)
        g = bt.grad(prob.xi, g_mom, g_S, w=prob.w, moments=mom).clone()
        dt, dev = ctx.theta_meta
        return g.to(device=dev, dtype=dt), None


def loss_batch(mom, S, target_mom, target_S, moment_weights: dict, spectrum_weight: float):
    """Per-shot loss (n_shots,): loss_fn of every shot, vectorised."""
    L = torch.zeros(mom.shape[0], dtype=torch.float64, device=mom.device)
    for k, c in moment_weights.items():
        i = MOMENT_INDEX[k]
        ref = target_mom[:, i]
        L = L + c * ((mom[:, i] - ref) / (ref.abs() + 1e-30)) ** 2
    if spectrum_weight and S.numel():
        norm = target_S.sum(dim=1, keepdim=True).clamp_min(1e-30)
        L = L + spectrum_weight * (((S - target_S) / norm) ** 2).sum(dim=1) * S.shape[1]
    return L


# The beam's mean energy without the laser (mean_gamma0) is part of the
# batched fit's default loss: a shot's reference measurement.
BATCH_MOMENT_WEIGHTS = {**DEFAULT_MOMENT_WEIGHTS, "mean_gamma0": 1.0}


def fit_batch(prob: BatchProblem, theta0: torch.Tensor, target_mom, target_S, steps: int = 200,
              lr: float = 0.01, scale: torch.Tensor | None = None, moment_weights=None,
              spectrum_weight: float = 1.0, lr_decay: float = 1.0, callback=None):
    """Adam on every shot's theta / scale at once (the shots' losses add, so
    each shot's parameters follow their own loss).  The learning rate is
    multiplied by ``lr_decay`` after every step.  Returns (theta, history of
    the summed loss, final per-shot losses)."""
    mw = BATCH_MOMENT_WEIGHTS if moment_weights is None else moment_weights
    scale = theta0.abs().clamp_min(1e-12) if scale is None else scale
    z = (theta0 / scale).clone().requires_grad_(True)
    opt = torch.optim.Adam([z], lr=lr)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=lr_decay)
    hist = []
    last = None
    for it in range(steps):
        opt.zero_grad()
        mom, S = BatchScatterFn.apply(z * scale, prob)
        per = loss_batch(mom, S, target_mom, target_S, mw, spectrum_weight)
        L = per.sum()
        L.backward()
        opt.step()
        sched.step()
        hist.append(float(L.detach()))
        last = per.detach()
        if callback is not None:
            callback(it, z.detach() * scale, per.detach())
    return (z.detach() * scale), hist, last


def fit_batch_multistart(lasers, beams, counts, xi, bins, starts: torch.Tensor, target_mom,
                         target_S, ranges=None, w=None, precision="f32", **kw):
    """Batched fit from several starting points per shot at once.

    ``starts`` is (K, n_shots, 8): K starting parameter sets for each of the
    n_shots shots (descriptor templates ``lasers``/``beams``, sample counts
    ``counts``, concatenated samples ``xi``).  The K x n_shots problems run as
    one batch over K copies of the samples (each copy sees its shot's own
    samples, so a shot's loss is exactly zero at its hidden parameters when
    the targets come from them), and for every shot the start whose fit ends
    with the lowest loss is kept: a local minimum (the reflections of the
    transverse offsets and of the delay leave the loss nearly unchanged)
    then costs nothing unless every start falls into one.  ``kw`` goes to
    fit_batch.  Returns (theta (n_shots, 8), final per-shot losses, index
    of the start kept per shot, history)."""
    K, n_shots = int(starts.shape[0]), int(starts.shape[1])
    dev = xi[0].device
    counts = [int(c) for c in counts]
    offs = [0]
    for _ in range(K):
        for c in counts:
            offs.append(offs[-1] + c)
    xk = [None if x is None else x.repeat(K) for x in xi]
    wk = None if w is None else w.repeat(K)
    rk = None if ranges is None else list(ranges) * K
    bt = B.Batch(list(lasers) * K, list(beams) * K, offs, bins, int(offs[-1]), dev, ranges=rk,
                 precision=precision)
    prob = BatchProblem(bt, xk, wk)
    tm = target_mom.repeat(K, 1)
    tS = target_S.repeat(K, 1)
    theta, hist, last = fit_batch(prob, starts.reshape(K * n_shots, 8).to(dev, torch.float64),
                                  tm, tS, **kw)
    per = last.reshape(K, n_shots)
    best = per.argmin(dim=0)
    th = theta.reshape(K, n_shots, 8)[best, torch.arange(n_shots, device=dev)]
    return th, per.min(dim=0).values, best, hist
