"""Seeded synthetic inputs and workload descriptions.

This module is the one piece shared by the CUDA path's tests/benchmark and the
oracle: it describes workloads (laser, beam and binning parameters) and draws
the standard variates that a beam sample is decoded from.  It holds none of
the method's arithmetic: no focus, no energy loss, no binning.

Sample streams (structure of arrays, one array per variate):
    xi[0], xi[1]  transverse position variates (x, y)      standard normal
    xi[2]         longitudinal position variate (z)        standard normal
    xi[3]         energy variate                           standard normal,
                                                           or uniform [0, 1)
                                                           for a flat spectrum
    xi[4], xi[5]  initial angle variates (theta_x, theta_y) standard normal
    xi[6]         angular-noise variate (quantum model)     standard normal
    xi[7]         energy-noise variate (quantum model)      standard normal

The paper measures on no public dataset; these draws stand in for the beams
of its PIC comparison setups (Sec. 3, Appendix A) with the shapes of the
workloads below.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

ENV_GAUSS, ENV_SIN2 = 0, 1
MODEL_LL, MODEL_QFP = 0, 1
VAR_CELL_FOCUS, VAR_CYCLE_CHI = 1, 2   # model variants (bit flags)

GAMMA_PER_GEV = 1.0e3 / 0.51099895  # 1 GeV in units of m_e c^2


@dataclass(frozen=True)
class Laser:
    lambda_um: float = 0.8
    a0: float = 10.0
    w0_um: float = 3.0
    tau_fs: float = 30.0          # intensity FWHM
    envelope: int = ENV_GAUSS
    model: int = MODEL_LL
    dx_um: float = 0.0            # laser-axis offset (misalignment)
    dy_um: float = 0.0
    delay_fs: float = 0.0         # pulse-peak arrival at the focal plane
    n_phase: int = 512
    div_prefactor: float = 1.0
    variant: int = 0               # VAR_* flags; 0 = the paper's model as read


@dataclass(frozen=True)
class Beam:
    gamma_mean: float = 1956.95
    rel_spread: float = 0.05
    gamma_lo: float = 0.0
    gamma_hi: float = 0.0
    flat_energy: int = 0
    sigma_x_um: float = 2.0
    sigma_y_um: float = 2.0
    sigma_z_um: float = 0.0
    div_rad: float = 0.0
    dx_um: float = 0.0
    dy_um: float = 0.0


@dataclass(frozen=True)
class Bins:
    n_bins: int = 256
    lo: float = 0.0
    hi: float = 2348.34
    log_spaced: int = 0
    n_tx: int = 0
    n_ty: int = 0
    theta_max: float = 0.0
    n_aeff: int = 0
    aeff_max: float = 0.0
    smooth_sigma_bins: float = 0.0   # kernel-smoothed spectrum (0 = off)


@dataclass(frozen=True)
class Workload:
    name: str
    laser: Laser
    beam: Beam
    bins: Bins
    n: int
    seed: int
    weighted: bool = False
    dtype: str = "f32"            # storage type of the sample streams
    notes: str = ""


# ---------------------------------------------------------------------------
# Workloads (sizes and parameters of the five benchmark configurations)
# ---------------------------------------------------------------------------

def tiny_gauss_hermite() -> Workload:
    """Head-on, aligned; 32^3 Gauss-Hermite nodes over (x, y, gamma0); LL."""
    g0 = GAMMA_PER_GEV
    return Workload(
        name="gh32_ll_1gev",
        laser=Laser(lambda_um=0.8, a0=10.0, w0_um=3.0, tau_fs=30.0, model=MODEL_LL),
        beam=Beam(gamma_mean=g0, rel_spread=0.05, sigma_x_um=2.0, sigma_y_um=2.0,
                  sigma_z_um=0.0, div_rad=0.0),
        bins=Bins(n_bins=256, lo=0.0, hi=1.2 * g0),
        n=32 ** 3, seed=0, weighted=True, dtype="f64",
        notes="32x32x32 probabilists' Gauss-Hermite tensor grid, weights sum to 1")


def full_qfp(n: int = 1 << 26) -> Workload:
    """2^26 Monte Carlo samples, quantum FP model, 512 phase steps."""
    gmax = 4000.0 * (1.0 + 4 * 0.1)
    return Workload(
        name="mc2p26_qfp512_4000",
        laser=Laser(lambda_um=0.8, a0=30.0, w0_um=2.5, tau_fs=30.0, model=MODEL_QFP,
                    dx_um=2.0, dy_um=0.0, delay_fs=40.0, n_phase=512),
        beam=Beam(gamma_mean=4000.0, rel_spread=0.1, sigma_x_um=3.0, sigma_y_um=3.0,
                  sigma_z_um=10.0, div_rad=1.0e-3),
        bins=Bins(n_bins=512, lo=0.0, hi=1.2 * gmax, n_tx=128, n_ty=128, theta_max=10.0e-3,
                  n_aeff=256, aeff_max=30.0),
        n=n, seed=0x23080902, dtype="f32")


def full_ll(n: int = 1 << 26) -> Workload:
    """The same beam and laser with the classical LL model (HBM-bound case)."""
    w = full_qfp(n)
    return replace(w, name="mc2p26_ll_4000", laser=replace(w.laser, model=MODEL_LL))


def fit_qfp(n: int = 1 << 24) -> Workload:
    """Differentiable fit: 2^24 FP32 samples, QFP, loss on the moments and a
    256-bin spectrum smoothed with a Gaussian kernel of 2 bins."""
    return Workload(
        name="mc2p24_fit_qfp512",
        laser=Laser(lambda_um=0.8, a0=20.0, w0_um=4.0, tau_fs=30.0, model=MODEL_QFP,
                    dx_um=1.0, dy_um=-0.5, delay_fs=10.0, n_phase=512),
        beam=Beam(gamma_mean=6000.0, rel_spread=0.08, sigma_x_um=3.0, sigma_y_um=3.0,
                  sigma_z_um=10.0, div_rad=1.0e-3),
        bins=Bins(n_bins=256, lo=0.0, hi=1.2 * 6000.0 * 1.32, smooth_sigma_bins=2.0),
        n=n, seed=0x23080904, dtype="f32")


def broadband_qfp(n: int = 1 << 27) -> Workload:
    """Flat gamma0 on [1e3, 2e4], 2 mrad, a0 = 100, w0 = 2, 1024 steps, log bins."""
    return Workload(
        name="mc2p27_broadband_qfp1024",
        laser=Laser(lambda_um=0.8, a0=100.0, w0_um=2.0, tau_fs=30.0, model=MODEL_QFP,
                    n_phase=1024),
        beam=Beam(gamma_mean=10500.0, rel_spread=0.0, gamma_lo=1000.0, gamma_hi=20000.0,
                  flat_energy=1, sigma_x_um=3.0, sigma_y_um=3.0, sigma_z_um=10.0,
                  div_rad=2.0e-3, dx_um=5.0),
        bins=Bins(n_bins=1024, lo=10.0, hi=24000.0, log_spaced=1),
        n=n, seed=0x23080905, dtype="f32")


# ---------------------------------------------------------------------------
# Variates
# ---------------------------------------------------------------------------

def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def sample_streams(n: int, seed: int, dtype=np.float32, flat_energy: bool = False,
                   antithetic: bool = False, chunk: int = 1 << 22) -> list[np.ndarray]:
    """Eight variate streams of length n (see module docstring).

    With ``antithetic`` the second half of every stream is the negation of the
    first (energy uniforms u -> 1-u), for the symmetry pins.
    """
    g = rng(seed)
    out = []
    m = (n + 1) // 2 if antithetic else n
    for k in range(8):
        a = np.empty(m, dtype=dtype)
        for s in range(0, m, chunk):
            e = min(m, s + chunk)
            if k == 3 and flat_energy:
                a[s:e] = g.random(e - s, dtype=np.float64).astype(dtype)
            else:
                a[s:e] = g.standard_normal(e - s, dtype=np.float64).astype(dtype)
        if antithetic:
            b = (np.asarray(1.0, dtype) - a) if (k == 3 and flat_energy) else -a
            a = np.concatenate([a, b])[:n]
        out.append(a)
    return out


def gauss_hermite(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Probabilists' Gauss-Hermite rule (weight exp(-x^2/2)/sqrt(2 pi)), sum w = 1.

    Golub-Welsch start: nodes are the eigenvalues of the symmetric Jacobi
    matrix of the He_k recurrence (off-diagonal sqrt(k)).  Each node is then
    polished by Newton steps on the orthonormal polynomial p_n, and the
    weights are the Christoffel numbers 1 / sum_k p_k(x_i)^2, which keeps the
    tiny outer weights accurate to full relative precision.
    """
    k = np.arange(1, n, dtype=np.float64)
    J = np.diag(np.sqrt(k), 1) + np.diag(np.sqrt(k), -1)
    x = np.linalg.eigvalsh(J)

    def orthonormal(x):
        p_prev, p = np.zeros_like(x), np.ones_like(x)
        ssum = p * p
        for j in range(n):
            p_next = (x * p - np.sqrt(j) * p_prev) / np.sqrt(j + 1)
            if j < n - 1:
                ssum = ssum + p_next * p_next
            p_prev, p = p, p_next
        return p, p_prev, ssum          # p_n, p_{n-1}, sum_{k<n} p_k^2

    for _ in range(3):
        pn, pn1, _ = orthonormal(x)
        x = x - pn / (np.sqrt(n) * pn1)
    _, _, ssum = orthonormal(x)
    w = 1.0 / ssum
    # the rule is symmetric about 0: enforce it exactly
    x = 0.5 * (x - x[::-1])
    w = 0.5 * (w + w[::-1])
    w = w / w.sum()
    return x, w


def gauss_hermite_streams(n1d: int = 32) -> tuple[list[np.ndarray], np.ndarray]:
    """Tensor grid over (x, y, gamma0): streams 0, 1, 3 carry nodes; weights."""
    x, w = gauss_hermite(n1d)
    X, Y, G = np.meshgrid(x, x, x, indexing="ij")
    WX, WY, WG = np.meshgrid(w, w, w, indexing="ij")
    n = n1d ** 3
    z = np.zeros(n)
    xi = [X.ravel().copy(), Y.ravel().copy(), z.copy(), G.ravel().copy(),
          z.copy(), z.copy(), z.copy(), z.copy()]
    return xi, (WX * WY * WG).ravel()


def workload_inputs(wl: Workload, n: int | None = None):
    """Streams and weights for a workload (n overrides the sample count)."""
    n = wl.n if n is None else n
    if wl.name.startswith("gh"):
        return gauss_hermite_streams(round(wl.n ** (1 / 3)))
    dt = np.float32 if wl.dtype == "f32" else np.float64
    xi = sample_streams(n, wl.seed, dtype=dt, flat_energy=bool(wl.beam.flat_energy))
    w = None
    if wl.weighted:
        w = rng(wl.seed + 1).uniform(0.5, 1.5, n).astype(dt)
    return xi, w


# ---------------------------------------------------------------------------
# Batched shots
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class BatchWorkload:
    name: str
    lasers: tuple
    beams: tuple
    counts: np.ndarray        # samples per shot
    offsets: np.ndarray       # n_shots + 1, exclusive prefix sums of counts
    ranges: np.ndarray        # (n_shots, 2) spectrum range per shot
    bins: Bins
    seed: int


def batch_shots(n_shots: int = 4096, seed: int = 0x23080903, log10_range=(3.0, 6.0),
                n_phase: int = 512, n_bins: int = 512, model_mix: bool = False) -> BatchWorkload:
    """Independent shots with per-shot parameters drawn from seed:
    n_s = round(10^U[lo, hi]); a0 ~ U[5, 50]; W0 ~ U[2, 10] um; dx, dy ~ N(0, 2) um;
    delay ~ N(0, 30) fs; gamma_mean ~ U[1e3, 2e4]; rel_spread ~ U[0.01, 0.2];
    sigma_perp = 3 um, sigma_z = 10 um, 1 mrad.  Spectrum range per shot
    [0, 1.2 gamma_mean (1 + 4 s)].  model_mix alternates the quantum and
    classical models (even shots quantum)."""
    g = rng(seed)
    lo, hi = log10_range
    counts = np.rint(10.0 ** g.uniform(lo, hi, n_shots)).astype(np.int64)
    a0 = g.uniform(5, 50, n_shots)
    w0 = g.uniform(2, 10, n_shots)
    dx = g.normal(0, 2, n_shots)
    dy = g.normal(0, 2, n_shots)
    delay = g.normal(0, 30, n_shots)
    gm = g.uniform(1e3, 2e4, n_shots)
    sp = g.uniform(0.01, 0.2, n_shots)
    lasers, beams, ranges = [], [], []
    for k in range(n_shots):
        model = MODEL_QFP if (not model_mix or k % 2 == 0) else MODEL_LL
        lasers.append(Laser(lambda_um=0.8, a0=float(a0[k]), w0_um=float(w0[k]), tau_fs=30.0,
                            model=model, dx_um=float(dx[k]), dy_um=float(dy[k]),
                            delay_fs=float(delay[k]), n_phase=n_phase))
        beams.append(Beam(gamma_mean=float(gm[k]), rel_spread=float(sp[k]), sigma_x_um=3.0,
                          sigma_y_um=3.0, sigma_z_um=10.0, div_rad=1.0e-3))
        ranges.append((0.0, 1.2 * gm[k] * (1 + 4 * sp[k])))
    offsets = np.zeros(n_shots + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    return BatchWorkload(name=f"batch{n_shots}_qfp{n_phase}", lasers=tuple(lasers),
                         beams=tuple(beams), counts=counts, offsets=offsets,
                         ranges=np.array(ranges), bins=Bins(n_bins=n_bins, lo=0.0, hi=1.0),
                         seed=seed)
