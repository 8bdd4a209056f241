"""Pins of the FP64 oracle to what the paper and mathematics fix.

None of these retypes the oracle's own formula: each compares it with an
independent route (a brute-force integration of the equation of motion, the
exact quantum-synchrotron spectrum through scipy's Bessel functions, a library
ODE solver, the paper's Table 1/2 closed forms, printed values, invariants).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import constants as SC
from scipy.integrate import quad, solve_ivp
from scipy.special import i0, kv

import oracle
from paper_2308_09348_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_values():
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# constants
# --------------------------------------------------------------------------

def test_omega0_matches_appendix_a():
    """Appendix A prints omega0 = 2.35e15 s^-1 for lambda = 0.8 um."""
    pv = paper_values()["omega0_per_s_at_0p8um"]
    c = oracle.constants(I.Laser(lambda_um=0.8))
    omega0_per_s = c["omega0"] * 1e15
    assert abs(omega0_per_s / pv["value"] - 1.0) < pv["rel_tol"]


def test_rc_and_schwinger_potential_from_si_constants():
    """R_c = r_e omega0/c and a_S = m c^2/(hbar omega0) via scipy.constants
    (the oracle uses CODATA 2018; later CODATA releases move them by ~1e-9)."""
    lam = 0.8e-6
    omega0 = 2 * math.pi * SC.c / lam
    re = SC.physical_constants["classical electron radius"][0]
    Rc = re * omega0 / SC.c
    aS = SC.m_e * SC.c ** 2 / (SC.hbar * omega0)
    c = oracle.constants(I.Laser(lambda_um=0.8))
    assert abs(c["Rc"] / Rc - 1) < 1e-8
    assert abs(c["aS"] / aS - 1) < 1e-8
    # alpha = R_c a_S (r_e = alpha lambdabar_c)
    assert abs(c["Rc"] * c["aS"] / SC.alpha - 1) < 1e-8


def test_envelope_fwhm_and_window():
    """Gaussian and sin^2 envelopes: intensity FWHM equals omega0 tau."""
    for env in (I.ENV_GAUSS, I.ENV_SIN2):
        L = I.Laser(tau_fs=30.0, envelope=env, n_phase=200000)
        phi, G, h = oracle.phase_grid(L)
        inten = G ** 2          # G is the field envelope
        above = phi[inten >= 0.5]
        c = oracle.constants(L)
        fwhm = above[-1] - above[0]
        assert abs(fwhm / c["Phi"] - 1) < 1e-3
        # midpoint nodes cover the window exactly
        assert abs(phi[0] - h / 2 - c["win_lo"]) < 1e-9 * c["Phi"]
        assert abs(phi[-1] + h / 2 - c["win_hi"]) < 1e-9 * c["Phi"]
        # c_RR uses the analytic integral of G^2; the midpoint sum agrees
        # (Gaussian: up to the 3e-8 truncation of the window)
        intG2 = (G ** 2).sum() * h
        assert abs((2 / 3) * c["Rc"] * intG2 / c["cRR"] - 1) < 1e-7


# --------------------------------------------------------------------------
# classical energy loss (Eq. 3) vs brute force of the LL equation of motion
# --------------------------------------------------------------------------

@pytest.mark.slow
def test_ll_closed_form_vs_rk4_equation_of_motion():
    from ll_brute_force import integrate, psi_derivs
    lam = 0.8
    Phi = 10 * 2 * math.pi                        # 10-cycle intensity FWHM
    tau_fs = Phi / (0.299792458 * 2 * math.pi / lam)
    laser = I.Laser(lambda_um=lam, tau_fs=tau_fs, a0=1.0)
    c = oracle.constants(laser)
    assert abs(c["Phi"] / Phi - 1) < 1e-12
    g0 = np.array([100.0, 500.0, 2000.0] * 3)
    a0 = np.repeat([1.0, 5.0, 10.0], 3)
    h0, hf, gf, ux, uz = integrate(g0, a0, Phi, c["Rc"], steps_per_cycle=200)
    # (1) the brute force reproduces the exact light-front law
    #     1/h_f = 1/h_0 + (2/3) R_c int psi'^2 dphi  (Di Piazza's solution)
    I1 = np.array([quad(lambda p: psi_derivs(p, a, Phi)[0] ** 2, -3 * Phi, 3 * Phi,
                        limit=2000)[0] for a in a0])
    exact = 1 / (1 / h0 + (2 / 3) * c["Rc"] * I1)
    assert np.max(np.abs(hf / exact - 1)) < 1e-6
    # (2) the oracle's cycle-averaged closed form: 1/gamma_f - 1/gamma_0 =
    #     c_RR a0^2 must equal 2 (1/h_f - 1/h_0) up to the envelope-gradient
    #     term int G'^2 / int G^2 = 2 ln2 / Phi^2 of the exact integral
    d_rk4 = 2 * (1 / hf - 1 / h0)
    d_oracle = c["cRR"] * a0 ** 2
    eps = 2 * math.log(2) / Phi ** 2
    assert np.max(np.abs(d_oracle / d_rk4 - 1 / (1 + eps))) < 2e-6
    # and the oracle's final energy (per-sample path, LL model)
    for i in range(len(g0)):
        L = I.Laser(lambda_um=lam, tau_fs=tau_fs, a0=a0[i], model=I.MODEL_LL)
        B = I.Beam(gamma_mean=g0[i], rel_spread=0.0, sigma_x_um=0.0, sigma_y_um=0.0)
        s = oracle.evaluate(L, B, None, [np.zeros(1)] * 8)
        assert abs(s["mu"][0] / gf[i] - 1) < 2e-3


# --------------------------------------------------------------------------
# quantum corrections (Eq. 6) vs the exact quantum-synchrotron spectrum
# --------------------------------------------------------------------------

def _Ki13(y):
    return quad(lambda s: kv(1.0 / 3.0, s), y, np.inf, limit=200)[0]


def _spectrum_F(xi, chi):
    """Quantum synchrotron emission spectrum (Baier-Katkov/Ritus), up to the
    prefactor alpha m c^2 / (sqrt3 pi hbar gamma); xi = photon energy fraction."""
    y = 2 * xi / (3 * chi * (1 - xi))
    return (1 - xi + 1 / (1 - xi)) * kv(2.0 / 3.0, y) - _Ki13(y)


def _exact_moments(chi):
    lo, hi = math.log(1e-12), math.log(1 - 1e-15)
    pts = [p for p in (math.log(min(chi, 0.5) * 0.01), math.log(min(chi, 0.5)), math.log(0.9))
           if lo < p < hi]
    m1 = quad(lambda t: math.exp(2 * t) * _spectrum_F(math.exp(t), chi), lo, hi, points=pts,
              limit=400)[0]
    m2 = quad(lambda t: math.exp(3 * t) * _spectrum_F(math.exp(t), chi), lo, hi, points=pts,
              limit=400)[0]
    return m1, m2


CHIS = [0.003, 0.03, 0.3, 1.0, 3.0, 10.0]


@pytest.fixture(scope="module")
def exact_moments():
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        return {chi: _exact_moments(chi) for chi in CHIS}


def test_gaunt_fit_vs_exact_power(exact_moments):
    for chi in CHIS:
        m1, _ = exact_moments[chi]
        g_exact = m1 / (math.sqrt(3) * math.pi) / ((2 / 3) * chi ** 2)
        g, _ = oracle.gaunt(chi)
        assert abs(g / g_exact - 1) < 0.02, (chi, g, g_exact)


def test_gaunt_limits_and_derivative():
    assert oracle.gaunt(0.0)[0] == 1.0
    chis = np.logspace(-4, 3, 200)
    gs = np.array([oracle.gaunt(c)[0] for c in chis])
    assert np.all(np.diff(gs) < 0)
    # large-chi tail ~ chi^(-4/3)
    s = math.log(oracle.gaunt(2e5)[0] / oracle.gaunt(1e5)[0]) / math.log(2)
    assert abs(s + 4 / 3) < 0.01
    # analytic derivative vs central difference
    for chi in (1e-3, 0.1, 1.0, 7.0):
        hh = chi * 1e-6
        fd = (oracle.gaunt(chi + hh)[0] - oracle.gaunt(chi - hh)[0]) / (2 * hh)
        assert abs(oracle.gaunt(chi)[1] / fd - 1) < 1e-6


def test_h2_fit_vs_exact_second_moment(exact_moments):
    assert oracle.h2(0.0) == 1.0
    for chi in CHIS:
        _, m2 = exact_moments[chi]
        h_exact = m2 / (math.sqrt(3) * math.pi) / (
            (55 / (16 * math.sqrt(3))) * chi * (2 / 3) * chi ** 2)
        assert abs(oracle.h2(chi) / h_exact - 1) < 0.006, (chi, oracle.h2(chi), h_exact)
    s = math.log(oracle.h2(2e5) / oracle.h2(1e5)) / math.log(2)
    assert abs(s + 7 / 3) < 0.01


def test_h2_fit_wide_range():
    """The fit's stated range, 1e-5 <= chi <= 300, at its ends and beyond
    the fixture's points."""
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        for chi in (1e-5, 1e-4, 0.1, 30.0, 100.0, 300.0):
            _, m2 = _exact_moments(chi)
            h_exact = m2 / (math.sqrt(3) * math.pi) / (
                (55 / (16 * math.sqrt(3))) * chi * (2 / 3) * chi ** 2)
            assert abs(oracle.h2(chi) / h_exact - 1) < 0.006, (chi, oracle.h2(chi), h_exact)
    # decreasing from h(0) = 1
    hs = np.array([oracle.h2(c) for c in np.logspace(-6, 6, 400)])
    assert np.all(np.diff(hs) < 0) and hs[0] < 1.0


def test_fp_rates_absolute_vs_exact_spectrum(exact_moments):
    """D1 and D2 per unit phase against the absolute emission moments.

    Per unit time the exact spectrum gives d<gamma>/dt = -(alpha m c^2 /
    (sqrt3 pi hbar)) m1 and d<dgamma^2>/dt = gamma (alpha m c^2/(sqrt3 pi hbar))
    m2; the phase advances at 2 omega0 for a head-on electron (the factor 2 of
    Eq. 1), and chi = 2 gamma a / a_S (Eq. 6) is taken at the rms field A/sqrt2.
    """
    L = I.Laser(lambda_um=0.8)
    c = oracle.constants(L)
    aS = c["aS"]
    for chi in CHIS:
        mu = 4000.0
        A = chi * aS / (2 * mu) * math.sqrt(2)
        r = oracle.qfp_rates(L, mu, A)
        assert abs(r["chi"] / chi - 1) < 1e-12
        m1, m2 = exact_moments[chi]
        D1_exact = -SC.alpha * aS * m1 / (2 * math.sqrt(3) * math.pi)
        D2_exact = mu * SC.alpha * aS * m2 / (2 * math.sqrt(3) * math.pi)
        assert abs(r["D1"] / D1_exact - 1) < 0.02, chi
        assert abs(r["D2"] / D2_exact - 1) < 0.02, chi
        # dD1/dgamma against a central difference of D1 in gamma at fixed A
        hh = mu * 1e-6
        fd = (oracle.qfp_rates(L, mu + hh, A)["D1"] - oracle.qfp_rates(L, mu - hh, A)["D1"]) / (2 * hh)
        assert abs(r["dD1"] / fd - 1) < 1e-6


# cycle-resolved chi: Gaunt and diffusion factors averaged over the cycle

def _cos_power_mean(p):
    """Cycle mean of |cos psi|^p in closed form (a Beta integral)."""
    from scipy.special import gamma
    return gamma((p + 1) / 2) / (math.sqrt(math.pi) * gamma(p / 2 + 1))


def test_cycle_factors_limits_and_tails():
    """chi -> 0: G = <2 cos^2> = 1, S = 2, H = 2 sqrt2 <|cos|^3>; large chi:
    g ~ chi^-4/3 and h ~ chi^-7/3 make G/g(sqrt2 chi) and H/h(sqrt2 chi)
    tend to 2 <|cos|^(2/3)> and 2 sqrt2 <|cos|^(2/3)>."""
    G, S, H = oracle.cycle_factors(0.0)
    assert abs(G - 1) < 1e-14 and abs(S - 2) < 1e-14
    assert abs(H / (2 * math.sqrt(2) * _cos_power_mean(3)) - 1) < 1e-14
    chi = 1e6
    G, S, H = oracle.cycle_factors(chi)
    r = 2 * _cos_power_mean(2 / 3)
    assert abs(G / oracle.gaunt(math.sqrt(2) * chi)[0] / r - 1) < 0.01
    assert abs(H / oracle.h2(math.sqrt(2) * chi) / (math.sqrt(2) * r) - 1) < 0.01
    # S = 2G + chi G' -> (2 - 4/3) G in the power-law tail
    assert abs(S / G - 2 / 3) < 0.01


def test_cycle_factors_vs_adaptive_quadrature_and_differences():
    for chi in (1e-3, 0.1, 1.0, 5.0, 40.0):
        G, S, H = oracle.cycle_factors(chi)
        qg = quad(lambda p: 2 * math.cos(p) ** 2 * oracle.gaunt(math.sqrt(2) * chi * math.cos(p))[0],
                  0, math.pi / 2, epsabs=0, epsrel=1e-13)[0] * 2 / math.pi
        qh = quad(lambda p: 2 * math.sqrt(2) * math.cos(p) ** 3 *
                  oracle.h2(math.sqrt(2) * chi * math.cos(p)), 0, math.pi / 2, epsabs=0,
                  epsrel=1e-13)[0] * 2 / math.pi
        assert abs(G / qg - 1) < 1e-12 and abs(H / qh - 1) < 1e-12, chi
        hh = chi * 1e-5
        dG = (oracle.cycle_factors(chi + hh)[0] - oracle.cycle_factors(chi - hh)[0]) / (2 * hh)
        assert abs(S / (2 * G + chi * dG) - 1) < 1e-8, chi


def test_cycle_gaunt_vs_cycle_mean_of_exact_power():
    """The cycle-resolved mean loss equals the cycle mean of the exact
    quantum-synchrotron power (to the 2 % of the Gaunt fit)."""
    import warnings
    xs, ws = np.polynomial.legendre.leggauss(8)
    ps = (xs + 1) * math.pi / 4
    for chi in (0.3, 3.0):
        acc = 0.0
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            for p, w in zip(ps, ws):
                ci = math.sqrt(2) * chi * math.cos(p)
                m1, _ = _exact_moments(ci)
                g_exact = m1 / (math.sqrt(3) * math.pi) / ((2 / 3) * ci ** 2)
                acc += w * math.pi / 4 * 2 * math.cos(p) ** 2 * g_exact
        G_exact = acc * 2 / math.pi
        assert abs(oracle.cycle_factors(chi)[0] / G_exact - 1) < 0.03, chi


def test_cycle_resolved_integration_vs_library_ode_solver():
    """QFP with cycle-resolved chi: the phase sum converges (second order) to
    a DOP853 solve with the same rates; the variant lowers the loss."""
    a0, g0 = 30.0, 4000.0
    Lc = I.Laser(a0=a0, model=I.MODEL_QFP, n_phase=512, variant=I.VAR_CYCLE_CHI)
    c = oracle.constants(Lc)
    Phi = c["Phi"]

    def f(phi, y):
        r = oracle.qfp_rates(Lc, y[0], a0 * math.exp(-2 * math.log(2) * (phi / Phi) ** 2))
        return [r["D1"], 2 * r["dD1"] * y[1] + r["D2"]]

    sol = solve_ivp(f, (c["win_lo"], c["win_hi"]), [g0, 0.0], method="DOP853", rtol=1e-11,
                    atol=1e-9)
    mu_ref, V_ref = sol.y[0, -1], sol.y[1, -1]
    errs = []
    for N in (256, 512, 1024):
        mu, V = oracle.qfp_integrate(I.Laser(**{**Lc.__dict__, "n_phase": N}), a0, g0)
        errs.append((abs(mu / mu_ref - 1), abs(V / V_ref - 1)))
    assert errs[1][0] < 2e-5 and errs[1][1] < 2e-4
    for (m1, v1), (m2, v2) in zip(errs, errs[1:]):
        assert 3.0 < m1 / m2 < 5.0 and 3.0 < v1 / v2 < 5.0
    mu_std, _ = oracle.qfp_integrate(I.Laser(a0=a0, model=I.MODEL_QFP, n_phase=512), a0, g0)
    assert mu_ref > mu_std * 1.005


# photon spectrum (Sec. 4): LCFA quantum-synchrotron emission along the phase

def test_bessel_pair_vs_library():
    """K_{2/3} against scipy's modified Bessel function; the tail integral of
    K_{1/3} against mpmath's (30 digits)."""
    import mpmath
    from scipy.special import kv
    for y in np.logspace(-8, 1.7, 25):
        k23, _ = oracle.bessel_pair(y)
        assert abs(k23 / kv(2 / 3, y) - 1) < 1e-13, y
    mpmath.mp.dps = 30
    for y in (1e-8, 1e-3, 0.1, 1.0, 5.0, 20.0):
        _, ki = oracle.bessel_pair(y)
        ref = mpmath.quad(lambda t: mpmath.besselk(mpmath.mpf(1) / 3, t), [y, y + 1, y + 10,
                                                                           mpmath.inf])
        assert abs(ki / float(ref) - 1) < 1e-12, y


def _rate_moments(aS, mu, chi):
    """Photon number and energy emitted per unit phase: integrals of the
    oracle's rate over eps in (0, mu), in the variable xi = eps/mu."""
    # in t = ln xi, with break points around the spectrum's scale xi ~ chi
    lo, hi = math.log(1e-14), math.log(1 - 1e-14)
    pts = sorted(p for p in (math.log(min(chi, 0.5) * f) for f in (0.01, 0.1, 1.0, 10.0))
                 if lo < p < hi)

    def r(t):
        x = math.exp(t)
        return oracle.photon_rate(aS, mu, chi, x * mu) * mu * x
    f0 = quad(r, lo, hi, points=pts, limit=400, epsrel=1e-11)[0]
    f1 = quad(lambda t: r(t) * math.exp(t) * mu, lo, hi, points=pts, limit=400,
              epsrel=1e-11)[0]
    return f0, f1


def test_photon_rate_classical_limits():
    """chi -> 0: the emitted energy per phase is the classical loss
    K mu^2 = alpha a_S chi^2/3 (Larmor, Eq. 3's rate), and the photon number
    per phase the classical 5 alpha a_S chi/(4 sqrt3 mu) (Gamma-function
    integrals of K_nu)."""
    L = I.Laser(lambda_um=0.8)
    aS = oracle.constants(L)["aS"]
    mu = 3000.0
    for chi in (1e-4, 1e-3):
        n, e = _rate_moments(aS, mu, chi)
        e_cl = SC.alpha * aS * chi ** 2 / 3
        n_cl = 5 * SC.alpha * aS * chi / (4 * math.sqrt(3) * mu)
        assert abs(e / e_cl - 1) < 10 * chi, chi        # O(chi) quantum corrections
        assert abs(n / n_cl - 1) < 10 * chi, chi


def test_photon_rate_energy_equals_gaunt_loss():
    """At any chi the emitted energy per phase equals the mean loss of the
    model, K mu^2 g(chi), to the 2 % of the Gaunt fit."""
    L = I.Laser(lambda_um=0.8)
    aS = oracle.constants(L)["aS"]
    mu = 3000.0
    for chi in (0.03, 0.3, 1.0, 3.0):
        _, e = _rate_moments(aS, mu, chi)
        g, _ = oracle.gaunt(chi)
        assert abs(e / (SC.alpha * aS * chi ** 2 / 3 * g) - 1) < 0.02, chi


def test_beam_photon_spectrum_energy_balance():
    """The energy carried by the beam's photon spectrum equals the energy the
    electrons lose in the same model (Gaunt-fit accuracy, log-bin
    quadrature)."""
    n = 16
    L = I.Laser(a0=20.0, w0_um=3.0, model=I.MODEL_QFP, n_phase=128)
    B = I.Beam(gamma_mean=3000.0, rel_spread=0.05, sigma_x_um=1.0, sigma_y_um=1.0,
               sigma_z_um=2.0, div_rad=0.0)
    xi = I.sample_streams(n, 31, dtype=np.float64)
    pb = I.Bins(n_bins=400, lo=1e-6, hi=3500.0, log_spaced=1)
    S = oracle.photon_spectrum(L, B, pb, xi)
    edges = pb.lo * (pb.hi / pb.lo) ** (np.arange(401) / 400)
    centres = np.sqrt(edges[1:] * edges[:-1])
    e_ph = float(np.sum(S * centres * np.diff(edges)))
    rec = oracle.evaluate(L, B, None, xi)
    e_el = float(np.sum(rec["gamma0"] - rec["mu"]))
    assert e_el > 10 * n                                   # a real interaction
    assert abs(e_ph / e_el - 1) < 0.03, (e_ph, e_el)


def test_photon_divergence_plane_wave_sin2_closed_form():
    """Eq. 7 in a plane wave with a sin^2 envelope, classical regime: photons
    are emitted in proportion to chi ~ A, so their mean square angle along
    the polarisation is <A^2/(2 mu^2)> weighted by A, a0^2 (int G^3/int G)
    /(2 gamma^2) = (5/16) a0^2/gamma^2 (Beta integrals of sin^2n), plus the
    1/gamma^2 cone; across it the cone alone."""
    g0, a0 = 1000.0, 2.0
    L = I.Laser(a0=a0, w0_um=3.0, envelope=I.ENV_SIN2, model=I.MODEL_QFP, n_phase=256)
    Bpw = I.Beam(gamma_mean=g0, rel_spread=0.0, sigma_x_um=0.0, sigma_y_um=0.0,
                 sigma_z_um=0.0, div_rad=0.0)
    pb = I.Bins(n_bins=240, lo=1e-9, hi=g0, log_spaced=1)
    S, T = oracle.photon_spectrum_angles(L, Bpw, pb, [np.zeros(1)] * 8)
    edges = pb.lo * (pb.hi / pb.lo) ** (np.arange(241) / 240)
    de = np.diff(edges)
    N, Tx, Ty = (S * de).sum(), (T[0] * de).sum(), (T[1] * de).sum()
    assert abs(Tx / N * g0 ** 2 / (5 / 16 * a0 ** 2 + 1) - 1) < 0.02
    assert abs(Ty / N * g0 ** 2 - 1) < 0.02


# plane-wave reconstruction (Eq. 5)

def test_pw_reconstruction_converges_to_direct_spectrum():
    """Classical model, monoenergetic misaligned beam: weighting plane-wave
    spectra at the a-bin centres by the beam's a_eff histogram (Eq. 5)
    reproduces the directly integrated 3D spectrum, with a distribution
    distance that shrinks at first order in the a-grid spacing; weight is
    conserved exactly."""
    g0, amax, n = 2000.0, 10.5, 4000
    L = I.Laser(a0=10.0, w0_um=3.0, dx_um=1.0, delay_fs=20.0, model=I.MODEL_LL)
    Bm = I.Beam(gamma_mean=g0, rel_spread=0.0, sigma_x_um=2.0, sigma_y_um=2.0,
                sigma_z_um=5.0, div_rad=0.0)
    Bpw = I.Beam(gamma_mean=g0, rel_spread=0.0, sigma_x_um=0.0, sigma_y_um=0.0,
                 sigma_z_um=0.0, div_rad=0.0)
    xi = I.sample_streams(n, 5, dtype=np.float64)
    D = []
    for na in (25, 50, 100):
        bins = I.Bins(n_bins=400, lo=0.0, hi=2100.0, n_aeff=na, aeff_max=amax)
        r = oracle.scatter(L, Bm, bins, xi)
        pw = np.array([oracle.scatter(I.Laser(a0=(k + 0.5) * amax / na, w0_um=3.0,
                                              model=I.MODEL_LL), Bpw, bins,
                                      [np.zeros(1)] * 8)["spectrum"] for k in range(na)])
        rec = oracle.pw_reconstruct(r["aeff_hist"], pw)[0]
        assert rec.sum() == r["spectrum"].sum() == n
        D.append(np.max(np.abs(np.cumsum(r["spectrum"]) - np.cumsum(rec))) / n)
    assert D[0] > D[1] > D[2] and D[2] < 0.01 and D[0] / D[2] > 3, D


def test_spread_below_eq9_bound_for_long_pulses():
    """Eq. 9 bounds sigma_f^2 for long pulses; the FP model stays below it
    and within an order of magnitude of it."""
    pv = paper_values()["eq9_bound"]
    for tau in (100.0, 300.0):
        for a0 in (5.0, 20.0, 50.0):
            for g0 in (1000.0, 4000.0, 10000.0):
                L = I.Laser(a0=a0, tau_fs=tau, model=I.MODEL_QFP, n_phase=2048)
                mu, V = oracle.qfp_integrate(L, a0, g0)
                I22 = 1.37e18 * a0 ** 2 / 0.8 ** 2 / 1e22
                bound = pv["c1"] * math.sqrt(I22) * g0 ** 3 / (1 + pv["c2"] * g0 * I22 * tau) ** 3
                assert 0.1 * bound < V <= bound, (tau, a0, g0, V, bound)


# --------------------------------------------------------------------------
# phase integration
# --------------------------------------------------------------------------

@pytest.mark.parametrize("env", [I.ENV_GAUSS, I.ENV_SIN2])
def test_qfp_classical_limit_equals_eq3(env):
    """a_S -> infinity gives g = 1, D2 = 0: the integrator must reproduce
    the closed form of Eq. 3 (to the Gaussian window truncation)."""
    for a0, g0 in ((10.0, 1957.0), (30.0, 4000.0), (100.0, 20000.0)):
        L = I.Laser(a0=a0, tau_fs=30.0, envelope=env, model=I.MODEL_QFP, n_phase=512)
        mu, V = oracle.qfp_integrate(L, a0, g0, 0.0, 1e12, 0.0)
        cRR = oracle.constants(L)["cRR"]
        closed = g0 / (1 + cRR * g0 * a0 ** 2)
        assert abs(mu / closed - 1) < 1e-7
        assert V == 0.0


def test_qfp_zero_intensity_is_identity():
    L = I.Laser(a0=0.0, model=I.MODEL_QFP, n_phase=64)
    for g0 in (1.0, 1957.0, 12345.678):
        mu, V = oracle.qfp_integrate(L, 0.0, g0)
        assert mu == g0 and V == 0.0


def test_variance_transport_classical_closed_form():
    """With D2 = 0 and g = 1 an initial variance V0 is carried by the
    linearised flow: V_f = V0 (d gamma_f / d gamma_0)^2 = V0/(1+c g0 a^2)^4.
    The scheme is second order: the error quarters when N doubles."""
    a0, g0, V0 = 20.0, 3000.0, 100.0
    errs = []
    for N in (256, 512, 1024, 2048):
        L = I.Laser(a0=a0, model=I.MODEL_QFP, n_phase=N)
        cRR = oracle.constants(L)["cRR"]
        exact = V0 / (1 + cRR * g0 * a0 ** 2) ** 4
        _, V = oracle.qfp_integrate(L, a0, g0, V0, 1e12, 0.0)
        errs.append(abs(V / exact - 1))
    assert errs[1] < 5e-4
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.5 < e1 / e2 < 4.5


def test_qfp_integrator_vs_library_ode_solver():
    """The phase sum converges (second order) to a high-accuracy DOP853 solve
    of d<gamma>/dphi = D1, dV/dphi = 2 dD1 V + D2 with the same rates."""
    a0, g0 = 30.0, 4000.0
    Lref = I.Laser(a0=a0, model=I.MODEL_QFP, n_phase=512)
    c = oracle.constants(Lref)
    Phi = c["Phi"]

    def G(phi):
        return math.exp(-2 * math.log(2) * (phi / Phi) ** 2)

    def f(phi, y):
        r = oracle.qfp_rates(Lref, y[0], a0 * G(phi))
        return [r["D1"], 2 * r["dD1"] * y[1] + r["D2"]]

    sol = solve_ivp(f, (c["win_lo"], c["win_hi"]), [g0, 0.0], method="DOP853", rtol=1e-11,
                    atol=1e-9)
    mu_ref, V_ref = sol.y[0, -1], sol.y[1, -1]
    errs = []
    for N in (256, 512, 1024):
        L = I.Laser(a0=a0, model=I.MODEL_QFP, n_phase=N)
        mu, V = oracle.qfp_integrate(L, a0, g0)
        errs.append((abs(mu / mu_ref - 1), abs(V / V_ref - 1)))
    assert errs[1][0] < 2e-5 and errs[1][1] < 2e-4     # 512 steps
    for (m1, v1), (m2, v2) in zip(errs, errs[1:]):
        assert 3.0 < m1 / m2 < 5.0 and 3.0 < v1 / v2 < 5.0


# --------------------------------------------------------------------------
# per-cell focus: Eq. 2 along the electron's path
# --------------------------------------------------------------------------

def _path_sample(L, B, v):
    """One decoded sample and the local field seen along its straight path,
    parameterised by time.  The electron sits at (x, y, z) at t = 0 and moves
    with velocity c(theta_x, theta_y, -1); the pulse envelope moves along +z
    with its peak at z = 0 at t = delay.  Returns gamma0 and the functions
    psi(t) (envelope phase from the peak) and a(t) (Eq. 2 at the electron)."""
    c = oracle.constants(L)
    k, om, zR = c["k"], c["omega0"], c["zR"]
    cl = SC.c * 1e6 / 1e15                                  # um / fs
    x = B.dx_um + B.sigma_x_um * v[0]
    y = B.dy_um + B.sigma_y_um * v[1]
    z = B.sigma_z_um * v[2]
    g0 = B.gamma_mean * (1 + B.rel_spread * v[3])
    thx, thy = B.div_rad * v[4], B.div_rad * v[5]

    def psi(t):                      # omega0 (t - delay) - k z_e(t)
        return om * (t - L.delay_fs) - k * (z - cl * t)

    def a(t):
        ze = z - cl * t
        xe, ye = x + thx * cl * t - L.dx_um, y + thy * cl * t - L.dy_um
        q = 1 + (ze / zR) ** 2
        return L.a0 / math.sqrt(q) * math.exp(-(xe * xe + ye * ye) / (L.w0_um ** 2 * q))

    # times at which psi spans the window (psi is linear in t, slope 2 omega0)
    t_lo = (c["win_lo"] + om * L.delay_fs + k * z) / (2 * om)
    t_hi = (c["win_hi"] + om * L.delay_fs + k * z) / (2 * om)
    return g0, psi, a, (t_lo, t_hi), c


def _focus_case(model, n_phase, variant=I.VAR_CELL_FOCUS, w0=2.5, div=5e-3):
    L = I.Laser(a0=20.0, w0_um=w0, tau_fs=30.0, dx_um=1.5, dy_um=-0.7, delay_fs=40.0,
                model=model, n_phase=n_phase, variant=variant)
    B = I.Beam(gamma_mean=4000.0, rel_spread=0.0, sigma_x_um=3.0, sigma_y_um=3.0,
               sigma_z_um=10.0, div_rad=div)
    V = np.array([[0.3, -0.8, 1.2, 0.0, 1.0, -0.5, 0, 0],
                  [-1.1, 0.4, -0.9, 0.0, -1.5, 0.7, 0, 0],
                  [0.0, 0.0, 2.0, 0.0, 0.2, 0.1, 0, 0],
                  [0.7, 0.9, -2.2, 0.0, 0.0, -1.2, 0, 0]])
    return L, B, V


def test_per_cell_focus_ll_vs_time_domain_quadrature():
    """LL with the per-cell focus: 1/gamma_f - 1/gamma0 equals the adaptive
    quadrature, over time along the straight path, of (2/3) R_c (a G)^2
    dpsi/dt; and differs from the crossing focus for these geometries."""
    L, B, V = _focus_case(I.MODEL_LL, 4096, w0=1.5)
    rec = oracle.evaluate(L, B, None, [V[:, k].copy() for k in range(8)])
    Lx = I.Laser(**{**L.__dict__, "variant": 0})
    rec_x = oracle.evaluate(Lx, B, None, [V[:, k].copy() for k in range(8)])
    for s, v in enumerate(V):
        g0, psi, a, (t0, t1), c = _path_sample(L, B, v)
        Phi = c["Phi"]
        dpsi = 2 * c["omega0"]

        def integrand(t):
            G = math.exp(-2 * math.log(2) * (psi(t) / Phi) ** 2)
            return (2 / 3) * c["Rc"] * (a(t) * G) ** 2 * dpsi

        du_ref = quad(integrand, t0, t1, epsabs=0, epsrel=1e-12, limit=400)[0]
        du = 1 / rec["mu"][s] - 1 / rec["gamma0"][s]
        assert abs(du / du_ref - 1) < 1e-6, (s, du, du_ref)
        du_x = 1 / rec_x["mu"][s] - 1 / rec_x["gamma0"][s]
        assert abs(du_x / du_ref - 1) > 1e-3, (s, du_x / du_ref - 1)   # the variant matters


def test_per_cell_focus_qfp_vs_library_ode_solver():
    """QFP with the per-cell focus: the phase sum converges (second order) to
    a DOP853 solve over time of the moment equations with the field a(t) G
    seen along the path."""
    L, B, V = _focus_case(I.MODEL_QFP, 512)
    v = V[0]
    g0, psi, a, (t0, t1), c = _path_sample(L, B, v)
    Phi, dpsi = c["Phi"], 2 * c["omega0"]

    def f(t, y):
        G = math.exp(-2 * math.log(2) * (psi(t) / Phi) ** 2)
        r = oracle.qfp_rates(L, y[0], a(t) * G)
        return [dpsi * r["D1"], dpsi * (2 * r["dD1"] * y[1] + r["D2"])]

    sol = solve_ivp(f, (t0, t1), [g0, 0.0], method="DOP853", rtol=1e-11, atol=1e-9)
    mu_ref, V_ref = sol.y[0, -1], sol.y[1, -1]
    errs = []
    for N in (512, 1024, 2048):
        LN = I.Laser(**{**L.__dict__, "n_phase": N})
        r = oracle.evaluate(LN, B, None, [np.array([x]) for x in v])
        errs.append((abs(r["mu"][0] / mu_ref - 1), abs(r["V"][0] / V_ref - 1)))
    assert errs[0][0] < 2e-5 and errs[0][1] < 2e-4
    for (m1, v1), (m2, v2) in zip(errs, errs[1:]):
        assert 3.0 < m1 / m2 < 5.0 and 3.0 < v1 / v2 < 5.0


@pytest.mark.parametrize("model", [I.MODEL_LL, I.MODEL_QFP])
def test_per_cell_focus_reduces_to_crossing_for_straight_path_in_long_focus(model):
    """No divergence and a Rayleigh length 1e4 times the path: the field is
    the same in every cell, so both focus readings agree (LL to the midpoint
    rule and window truncation of the G^2 integral, QFP exactly)."""
    L, B, V = _focus_case(model, 2048, w0=250.0, div=0.0)
    Lx = I.Laser(**{**L.__dict__, "variant": 0})
    xi = [V[:, k].copy() for k in range(8)]
    r, rx = oracle.evaluate(L, B, None, xi), oracle.evaluate(Lx, B, None, xi)
    tol = 1e-7 if model == I.MODEL_LL else 1e-9
    np.testing.assert_allclose(r["mu"], rx["mu"], rtol=tol)
    np.testing.assert_allclose(r["V"], rx["V"], rtol=1e-7, atol=0)


# --------------------------------------------------------------------------
# whole-beam integration: Table 1 and Table 2 closed forms
# --------------------------------------------------------------------------

def _hist_vs_density(hist, edges, density, n_total, z=5.0, floor=3.0):
    """Compare histogram masses with the integral of an analytic density
    over each bin: |h - N p| <= z sqrt(N p) + floor."""
    for b in range(len(hist)):
        p = quad(density, edges[b], edges[b + 1], limit=200)[0]
        tol = z * math.sqrt(max(n_total * p, 1.0)) + floor
        assert abs(hist[b] - n_total * p) <= tol, (b, hist[b], n_total * p)


def _short_beam_inputs(n, seed, sigma, dx=0.0, delay=0.0, a0=12.0, w0=2.0, lam=1.0):
    L = I.Laser(lambda_um=lam, a0=a0, w0_um=w0, dx_um=dx, delay_fs=delay, model=I.MODEL_LL)
    B = I.Beam(gamma_mean=5000.0, rel_spread=0.0, sigma_x_um=sigma, sigma_y_um=sigma,
               sigma_z_um=0.0, div_rad=0.0)
    xi = I.sample_streams(n, seed, dtype=np.float64)
    return L, B, xi


def test_table1_short_beam_aligned():
    """Short beam, aligned: P(a_eff < A) = (A/a0)^(W0^2/R^2), R = sqrt2 sigma."""
    n, sigma, a0, w0 = 1 << 16, 1.5, 12.0, 2.0
    L, B, xi = _short_beam_inputs(n, 11, sigma, a0=a0, w0=w0)
    bins = I.Bins(n_bins=1, lo=0, hi=1e9, n_aeff=48, aeff_max=a0)
    r = oracle.scatter(L, B, bins, xi)
    R2 = 2 * sigma ** 2
    k = w0 ** 2 / R2
    edges = np.linspace(0, a0, 49)
    _hist_vs_density(r["aeff_hist"], edges, lambda a: k / a * (a / a0) ** k, n)


def test_table1_short_beam_transverse_offset():
    """Table 1 Short beam with a transverse offset (the I0 term)."""
    n, sigma, a0, w0, d = 1 << 16, 1.5, 12.0, 2.0, 2.0
    L, B, xi = _short_beam_inputs(n, 12, sigma, dx=d, a0=a0, w0=w0)
    bins = I.Bins(n_bins=1, lo=0, hi=1e9, n_aeff=48, aeff_max=a0)
    r = oracle.scatter(L, B, bins, xi)
    R = math.sqrt(2) * sigma
    k = w0 ** 2 / R ** 2

    def dens(a):
        lg = math.log(a0 / a)
        return k / a * (a / a0) ** k * i0(2 * (d / R) * (w0 / R) * math.sqrt(lg)) * math.exp(-d * d / R ** 2)

    edges = np.linspace(0, a0, 49)
    _hist_vs_density(r["aeff_hist"], edges, dens, n)


def test_table1_short_beam_delay():
    """Longitudinal (temporal) offset: W0 -> W and a0 -> a_par with
    Delta_par = -c delay / 2 (the collision point moves by half the lag)."""
    n, sigma, a0, w0, lam, delay = 1 << 16, 1.5, 12.0, 2.0, 1.0, 60.0
    L, B, xi = _short_beam_inputs(n, 13, sigma, delay=delay, a0=a0, w0=w0, lam=lam)
    zR = math.pi * w0 ** 2 / lam
    dpar = 0.299792458 * delay / 2
    W = w0 * math.sqrt(1 + (dpar / zR) ** 2)
    apar = a0 / math.sqrt(1 + (dpar / zR) ** 2)
    bins = I.Bins(n_bins=1, lo=0, hi=1e9, n_aeff=48, aeff_max=a0)
    r = oracle.scatter(L, B, bins, xi)
    R2 = 2 * sigma ** 2
    k = W ** 2 / R2
    edges = np.linspace(0, a0, 49)

    def dens(a):
        return k / a * (a * W / (a0 * w0)) ** k if a < apar else 0.0

    _hist_vs_density(r["aeff_hist"], edges, dens, n)
    assert r["aeff_hist"][edges[:-1] > apar].sum() == 0


def test_table1_thin_beam():
    """Thin beam (R << W0), flat-top length L: dN/da = (2 N z_R / L)
    (a0^2/a^2) / sqrt(a0^2 - a^2) on both branches (aligned)."""
    n, a0, w0, lam, Lb = 1 << 16, 12.0, 2.0, 1.0, 60.0
    L = I.Laser(lambda_um=lam, a0=a0, w0_um=w0, model=I.MODEL_LL)
    B = I.Beam(gamma_mean=5000.0, rel_spread=0.0, sigma_x_um=0.0, sigma_y_um=0.0,
               sigma_z_um=Lb / (2 * math.sqrt(3)))
    xi = I.sample_streams(n, 14, dtype=np.float64)
    xi[2] = I.rng(99).uniform(-math.sqrt(3), math.sqrt(3), n)   # flat-top in z
    zR = math.pi * w0 ** 2 / lam
    az = a0 / math.sqrt(1 + (Lb / (4 * zR)) ** 2)
    bins = I.Bins(n_bins=1, lo=0, hi=1e9, n_aeff=64, aeff_max=a0)
    r = oracle.scatter(L, B, bins, xi)
    edges = np.linspace(0, a0, 65)

    def dens(a):
        if a <= az or a >= a0:
            return 0.0
        return 2 * (2 * zR / Lb) * (a0 ** 2 / a ** 2) / math.sqrt(a0 ** 2 - a ** 2)

    _hist_vs_density(r["aeff_hist"], edges, dens, n)


def test_table2_short_beam_ll_spectrum():
    """Table 2 Short beam: dN/dgamma = N (W0^2/2R^2) (g0/g)/(g0-g)
    ((g0-g)/(c_RR g0 g a0^2))^(W0^2/2R^2) above gamma_min."""
    n, sigma, a0, w0, g0 = 1 << 16, 1.5, 12.0, 2.0, 5000.0
    L, B, xi = _short_beam_inputs(n, 15, sigma, a0=a0, w0=w0, lam=0.8)
    cRR = oracle.constants(L)["cRR"]
    gmin = g0 / (1 + cRR * g0 * a0 ** 2)
    bins = I.Bins(n_bins=64, lo=gmin * 0.9, hi=g0 * 1.0001)
    r = oracle.scatter(L, B, bins, xi)
    k = w0 ** 2 / (2 * 2 * sigma ** 2)

    def dens(g):
        if g <= gmin or g >= g0:
            return 0.0
        return k * (g0 / g) / (g0 - g) * ((g0 - g) / (cRR * g0 * g * a0 ** 2)) ** k

    edges = np.linspace(bins.lo, bins.hi, bins.n_bins + 1)
    _hist_vs_density(r["spectrum"], edges, dens, n)


def test_table2_thin_beam_ll_spectrum():
    """Table 2 Thin beam: dN/dgamma = (2 N z_R/L) g0/(g0-g)^(3/2)
    c_RR g0 a0^2 / sqrt(c_RR g g0 a0^2 + g - g0), on gamma_min < gamma < gamma_z
    (the printed theta(gamma - gamma_z) has its support inverted: a_eff runs
    from a_z up to a0, so gamma_f runs from gamma_min up to gamma_z)."""
    n, a0, w0, lam, Lb, g0 = 1 << 16, 12.0, 2.0, 0.8, 60.0, 5000.0
    L = I.Laser(lambda_um=lam, a0=a0, w0_um=w0, model=I.MODEL_LL)
    B = I.Beam(gamma_mean=g0, rel_spread=0.0, sigma_x_um=0.0, sigma_y_um=0.0,
               sigma_z_um=Lb / (2 * math.sqrt(3)))
    xi = I.sample_streams(n, 16, dtype=np.float64)
    xi[2] = I.rng(98).uniform(-math.sqrt(3), math.sqrt(3), n)
    c = oracle.constants(L)
    cRR, zR = c["cRR"], c["zR"]
    az = a0 / math.sqrt(1 + (Lb / (4 * zR)) ** 2)
    gmin = g0 / (1 + cRR * g0 * a0 ** 2)
    gz = g0 / (1 + cRR * g0 * az ** 2)
    bins = I.Bins(n_bins=48, lo=gmin, hi=gz)

    def dens(g):
        if g <= gmin or g >= gz:
            return 0.0
        return (2 * zR / Lb) * g0 / (g0 - g) ** 1.5 * cRR * g0 * a0 ** 2 / math.sqrt(
            cRR * g * g0 * a0 ** 2 + g - g0)

    r = oracle.scatter(L, B, bins, xi)
    edges = np.linspace(bins.lo, bins.hi, bins.n_bins + 1)
    _hist_vs_density(r["spectrum"], edges, dens, n)


# the analytic fast path: Table 1 / Table 2 closed forms evaluated on a grid

def test_bessel_i0_vs_scipy():
    for x in (0.0, 1e-3, 0.5, 3.0, 29.9, 30.1, 100.0, 600.0):
        assert abs(oracle.bessel_i0(x) / i0(x) - 1) < 1e-14, x


@pytest.mark.parametrize("case", ["aligned", "offset", "delay"])
def test_analytic_short_beam_vs_monte_carlo(case):
    n, sigma, a0, w0, lam = 1 << 16, 1.5, 12.0, 2.0, 1.0
    dx = 2.0 if case == "offset" else 0.0
    delay = 60.0 if case == "delay" else 0.0
    L, B, xi = _short_beam_inputs(n, 21, sigma, dx=dx, delay=delay, a0=a0, w0=w0, lam=lam)
    r = oracle.scatter(L, B, I.Bins(n_bins=1, lo=0, hi=1e9, n_aeff=48, aeff_max=a0), xi)
    par = dict(radius=math.sqrt(2) * sigma, d_perp=dx, d_par=-0.299792458 * delay / 2, n=n)
    edges = np.linspace(0, a0, 49)
    _hist_vs_density(r["aeff_hist"], edges,
                     lambda a: float(oracle.analytic_aeff(L, "short", [a], **par)[0]) / n, n)


def test_analytic_thin_beam_vs_monte_carlo_with_offset():
    """Thin beam with the collision centre off the focal plane (one branch
    leaves the beam's span)."""
    n, a0, w0, lam, Lb, dpar = 1 << 16, 12.0, 2.0, 1.0, 60.0, 9.0
    L = I.Laser(lambda_um=lam, a0=a0, w0_um=w0, model=I.MODEL_LL,
                delay_fs=-2 * dpar / 0.299792458)
    B = I.Beam(gamma_mean=5000.0, rel_spread=0.0, sigma_x_um=0.0, sigma_y_um=0.0,
               sigma_z_um=Lb / (2 * math.sqrt(3)))
    xi = I.sample_streams(n, 22, dtype=np.float64)
    xi[2] = I.rng(97).uniform(-math.sqrt(3), math.sqrt(3), n)
    r = oracle.scatter(L, B, I.Bins(n_bins=1, lo=0, hi=1e9, n_aeff=64, aeff_max=a0), xi)
    edges = np.linspace(0, a0, 65)
    par = dict(length=Lb, d_par=dpar, n=n)
    _hist_vs_density(r["aeff_hist"], edges,
                     lambda a: float(oracle.analytic_aeff(L, "thin", [a], **par)[0]) / n, n)


def test_analytic_wide_beam_vs_monte_carlo():
    """Wide beam: uniform density across a box much wider than the spot,
    flat-top length, collision centre off the focal plane."""
    n, a0, w0, lam, Lb, dpar, X = 1 << 17, 12.0, 2.0, 1.0, 60.0, 6.0, 12.0
    L = I.Laser(lambda_um=lam, a0=a0, w0_um=w0, model=I.MODEL_LL,
                delay_fs=-2 * dpar / 0.299792458)
    B = I.Beam(gamma_mean=5000.0, rel_spread=0.0, sigma_x_um=X, sigma_y_um=X,
               sigma_z_um=Lb / (2 * math.sqrt(3)))
    xi = I.sample_streams(n, 23, dtype=np.float64)
    g = I.rng(96)
    xi[0], xi[1] = g.uniform(-1, 1, n), g.uniform(-1, 1, n)
    xi[2] = g.uniform(-math.sqrt(3), math.sqrt(3), n)
    r = oracle.scatter(L, B, I.Bins(n_bins=1, lo=0, hi=1e9, n_aeff=48, aeff_max=a0), xi)
    nb = n / ((2 * X) ** 2 * Lb)
    edges = np.linspace(0, a0, 49)
    par = dict(length=Lb, d_par=dpar, n=nb)
    # bins above 1.5: the box covers every electron with a_eff > 1.5
    dens = lambda a: float(oracle.analytic_aeff(L, "wide", [a], **par)[0]) / n
    _hist_vs_density(r["aeff_hist"][6:], edges[6:], dens, n)


@pytest.mark.parametrize("geom", ["short", "thin"])
def test_analytic_ll_spectrum_vs_monte_carlo(geom):
    """Table 2 via Eq. 6: the classical spectrum of the short and thin beams."""
    n, a0, w0, lam, g0 = 1 << 16, 12.0, 2.0, 0.8, 5000.0
    if geom == "short":
        sigma = 1.5
        L, B, xi = _short_beam_inputs(n, 24, sigma, a0=a0, w0=w0, lam=lam)
        par = dict(radius=math.sqrt(2) * sigma, n=n)
    else:
        Lb = 60.0
        L = I.Laser(lambda_um=lam, a0=a0, w0_um=w0, model=I.MODEL_LL)
        B = I.Beam(gamma_mean=g0, rel_spread=0.0, sigma_x_um=0.0, sigma_y_um=0.0,
                   sigma_z_um=Lb / (2 * math.sqrt(3)))
        xi = I.sample_streams(n, 25, dtype=np.float64)
        xi[2] = I.rng(95).uniform(-math.sqrt(3), math.sqrt(3), n)
        par = dict(length=Lb, n=n)
    cRR = oracle.constants(L)["cRR"]
    gmin = g0 / (1 + cRR * g0 * a0 ** 2)
    bins = I.Bins(n_bins=48, lo=gmin * 0.98, hi=g0 * 1.0001)
    r = oracle.scatter(L, B, bins, xi)
    edges = np.linspace(bins.lo, bins.hi, 49)
    _hist_vs_density(r["spectrum"], edges,
                     lambda g: float(oracle.analytic_ll(L, geom, g0, [g], **par)[0]) / n, n)


# --------------------------------------------------------------------------
# invariants of the whole-beam integration
# --------------------------------------------------------------------------

def _qfp_workload(n=2048, seed=5):
    wl = I.full_qfp(n)
    xi, _ = I.workload_inputs(wl, n)
    return wl, [x.astype(np.float64) for x in xi]


def test_zero_intensity_spectrum_is_initial_histogram():
    wl, xi = _qfp_workload()
    for model in (I.MODEL_LL, I.MODEL_QFP):
        L = I.Laser(**{**wl.laser.__dict__, "a0": 0.0, "model": model})
        s = oracle.evaluate(L, wl.beam, wl.bins, xi)
        assert np.array_equal(s["mu"], s["gamma0"])
        assert np.all(s["V"] == 0)
        r = oracle.scatter(L, wl.beam, wl.bins, xi)
        h, _ = np.histogram(s["gamma0"], bins=wl.bins.n_bins, range=(wl.bins.lo, wl.bins.hi))
        assert np.array_equal(r["spectrum"], h.astype(float))


def test_weight_conservation_and_consistency():
    wl, xi = _qfp_workload()
    w = I.rng(3).uniform(0.2, 2.0, len(xi[0]))
    r = oracle.scatter(wl.laser, wl.beam, wl.bins, xi, w)
    m = r["moments"]
    assert abs(r["spectrum"].sum() + m["under"] + m["over"] - w.sum()) < 1e-9
    assert abs(r["divmap"].sum() + m["map_out"] - w.sum()) < 1e-9
    assert abs(r["aeff_hist"].sum() - w[np.asarray(
        oracle.evaluate(wl.laser, wl.beam, wl.bins, xi)["abin"]) < wl.bins.n_aeff].sum()) < 1e-9
    # moments against the per-sample records (law of total variance)
    s = oracle.evaluate(wl.laser, wl.beam, wl.bins, xi)
    W = w.sum()
    mean = (w * s["mu"]).sum() / W
    var = (w * (s["mu"] - mean) ** 2).sum() / W + (w * s["V"]).sum() / W
    assert abs(m["mean"] / mean - 1) < 1e-12
    assert abs(m["spread"] / math.sqrt(var) - 1) < 1e-10
    thx0 = wl.beam.div_rad * xi[4]
    assert abs(m["div_x"] ** 2 / ((w * (thx0 ** 2 + s["theta_e"] ** 2)).sum() / W) - 1) < 1e-12


def _mc_finalize_case(n, seed):
    """A quantum beam whose energy spread is mostly the per-electron Fokker-
    Planck variance and whose x divergence is mostly the Eq. 8 broadening,
    with the initial angles still a visible share, and uneven weights."""
    L = I.Laser(lambda_um=0.8, a0=40.0, w0_um=4.0, tau_fs=30.0, model=I.MODEL_QFP, dx_um=1.0,
                delay_fs=10.0, n_phase=16)
    B = I.Beam(gamma_mean=6000.0, rel_spread=0.002, sigma_x_um=1.0, sigma_y_um=1.0,
               sigma_z_um=5.0, div_rad=6e-3)
    bins = I.Bins(n_bins=64, lo=0.0, hi=9000.0)
    xi = [x.astype(np.float64) for x in I.sample_streams(n, seed)]
    w = I.rng(seed + 1).uniform(0.25, 1.75, n)
    return L, B, bins, xi, w


@pytest.mark.slow
def test_moment_finalize_vs_realised_monte_carlo():
    """The whole-beam moments against the weighted sample moments of the
    REALISED per-electron outcomes over 2^20 samples (Sec. 1 observables,
    Eq. 8): the law-of-total-variance spread must equal the spread of the
    realised energies gamma_out = mu + sqrt(V) xi7, and div_x / div_y the rms
    of the realised angles theta_x = theta_x0 + theta_e xi6 and theta_y.  The
    expectations and the Monte Carlo noise are computed here in numpy from
    the per-sample records; the moment struct is only the thing checked.
    The case is chosen so that dropping <V> from the spread, dropping either
    term of div_x, or putting theta_e on the y axis each misses by many
    standard deviations."""
    n = 1 << 20
    L, B, bins, xi, w = _mc_finalize_case(n, seed=0x2308)
    m = oracle.scatter(L, B, bins, xi, w)["moments"]
    s = oracle.evaluate(L, B, bins, xi)
    W = w.sum()
    g, mu, V = s["gamma_out"], s["mu"], s["V"]
    # realised sample moments
    mean_r = (w * g).sum() / W
    var_r = (w * (g - mean_r) ** 2).sum() / W
    thx2_r = (w * s["theta_x"] ** 2).sum() / W
    thy2_r = (w * s["theta_y"] ** 2).sum() / W
    # the noise of each estimator over xi6, xi7 given the samples' mu, V,
    # theta_x0, theta_e: mean_r - <mu> = sum w sqrt(V) xi7 / W;
    # var_r - [<(mu - m)^2> + <V>] = sum w [2 (mu - m) sqrt(V) xi7 + V (xi7^2 - 1)] / W
    # (+ O(1/N)); thx2_r - <thx0^2 + te^2> = sum w [2 thx0 te xi6 + te^2 (xi6^2 - 1)] / W
    mu_m = (w * mu).sum() / W
    d = mu - mu_m
    sd_mean = math.sqrt((w ** 2 * V).sum()) / W
    sd_var = math.sqrt((w ** 2 * (4 * d * d * V + 2 * V * V)).sum()) / W
    thx0 = B.div_rad * xi[4]
    te = s["theta_e"]
    sd_thx = math.sqrt((w ** 2 * (4 * thx0 ** 2 * te ** 2 + 2 * te ** 4)).sum()) / W
    z = 5.0
    print("mean", m["mean"], mean_r, "spread^2", m["spread"] ** 2, var_r, "+-", sd_var,
          "div_x^2", m["div_x"] ** 2, thx2_r, "+-", sd_thx)
    assert abs(m["W"] - W) <= 1e-9 * W
    assert abs(m["mean"] - mean_r) <= z * sd_mean
    assert abs(m["spread"] ** 2 - var_r) <= z * sd_var + 1e-6 * var_r
    assert abs(m["div_x"] ** 2 - thx2_r) <= z * sd_thx
    # the y angle carries no broadening: exact
    assert abs(m["div_y"] ** 2 / thy2_r - 1) <= 1e-12
    assert abs(m["div"] ** 2 / (thx2_r + thy2_r) - 1) <= 10 * z * sd_thx / thx2_r
    assert abs(m["rel_spread"] - m["spread"] / m["mean"]) <= 1e-15 * m["rel_spread"]
    # the case discriminates: each plausible slip misses by > 20 sigma
    assert abs((w * d * d).sum() / W - var_r) > 20 * sd_var          # <V> dropped
    assert abs((w * V).sum() / W - var_r) > 20 * sd_var              # spread of mu dropped
    assert abs((w * thx0 ** 2).sum() / W - thx2_r) > 20 * sd_thx      # theta_e dropped
    assert abs((w * te ** 2).sum() / W - thx2_r) > 20 * sd_thx        # theta_x0 dropped
    assert (w * te ** 2).sum() / W > 1e-3 * thy2_r                   # theta_e on y (exact check)


def test_eq8_coefficient_and_scaling():
    """Eq. 8: theta_e = kappa sqrt(2/pi) a sigma / gamma^2 per electron, with
    a -> a_eff, sigma -> sqrt(V), gamma -> mu.  The coefficient is the one the
    paper prints (tests/golden); a least-squares fit of log theta_e on
    log a_eff, log sqrt(V) and log mu over a beam with wide ranges of all
    three must give exponents 1, 1, -2 and the printed coefficient, and the
    prefactor kappa must scale theta_e linearly."""
    c_paper = paper_values()["eq8_theta_e_coefficient"]["value"]
    assert abs(c_paper - math.sqrt(2 / math.pi)) < 1e-15
    n = 4096
    L = I.Laser(lambda_um=0.8, a0=60.0, w0_um=3.0, tau_fs=30.0, model=I.MODEL_QFP, n_phase=24)
    B = I.Beam(gamma_mean=5000.0, rel_spread=0.3, sigma_x_um=3.0, sigma_y_um=3.0,
               sigma_z_um=20.0, div_rad=1e-3)
    xi = [x.astype(np.float64) for x in I.sample_streams(n, 77)]
    s = oracle.evaluate(L, B, None, xi)
    ok = s["V"] > 0
    assert ok.mean() > 0.99
    a, sv, mu, te = s["aeff"][ok], np.sqrt(s["V"][ok]), s["mu"][ok], s["theta_e"][ok]
    # the three regressors must vary independently over this beam
    X = np.column_stack([np.ones(a.size), np.log(a), np.log(sv), np.log(mu)])
    assert np.linalg.cond(X[:, 1:] - X[:, 1:].mean(0)) < 1e3
    coef, *_ = np.linalg.lstsq(X, np.log(te), rcond=None)
    print("log-fit coefficients:", coef, "exp(c0):", math.exp(coef[0]))
    assert np.allclose(coef[1:], [1.0, 1.0, -2.0], atol=1e-9)
    assert abs(math.exp(coef[0]) / c_paper - 1) < 1e-9
    L2 = I.Laser(**{**L.__dict__, "div_prefactor": 2.5})
    s2 = oracle.evaluate(L2, B, None, xi)
    np.testing.assert_array_equal(s2["mu"], s["mu"])
    np.testing.assert_allclose(s2["theta_e"], 2.5 * s["theta_e"], rtol=1e-15)
    # the classical model has no broadening
    s3 = oracle.evaluate(I.Laser(**{**L.__dict__, "model": I.MODEL_LL}), B, None, xi)
    assert np.all(s3["theta_e"] == 0)


def test_transverse_offset_mirror_symmetry():
    """+dx on a sample set equals -dx on its x-mirrored set, bit for bit;
    the divergence map mirrors in theta_x."""
    wl, xi = _qfp_workload(1024)
    B = I.Beam(**{**wl.beam.__dict__, "dx_um": 0.0})
    L1 = I.Laser(**{**wl.laser.__dict__, "dx_um": 2.0})
    L2 = I.Laser(**{**wl.laser.__dict__, "dx_um": -2.0})
    xm = list(xi)
    for k in (0, 4, 6):
        xm[k] = -xi[k]
    r1 = oracle.scatter(L1, B, wl.bins, xi)
    r2 = oracle.scatter(L2, B, wl.bins, xm)
    assert np.array_equal(r1["spectrum"], r2["spectrum"])
    assert r1["moments"] == r2["moments"]
    s1 = oracle.evaluate(L1, B, wl.bins, xi)
    s2 = oracle.evaluate(L2, B, wl.bins, xm)
    assert np.array_equal(s1["aeff"], s2["aeff"]) and np.array_equal(s1["mu"], s2["mu"])
    assert np.array_equal(s1["theta_x"], -s2["theta_x"])


def test_delay_mirror_symmetry():
    """+delay with z-mirrored samples equals -delay, bit for bit, at zero
    divergence."""
    wl, xi = _qfp_workload(1024)
    B = I.Beam(**{**wl.beam.__dict__, "div_rad": 0.0})
    L1 = I.Laser(**{**wl.laser.__dict__, "delay_fs": 40.0})
    L2 = I.Laser(**{**wl.laser.__dict__, "delay_fs": -40.0})
    xm = list(xi)
    xm[2] = -xi[2]
    s1 = oracle.evaluate(L1, B, wl.bins, xi)
    s2 = oracle.evaluate(L2, B, wl.bins, xm)
    assert np.array_equal(s1["aeff"], s2["aeff"])
    assert np.array_equal(s1["mu"], s2["mu"]) and np.array_equal(s1["V"], s2["V"])


def test_classical_divergence_unchanged():
    """Classical model: the final angle is the initial angle (S11 reading)."""
    wl, xi = _qfp_workload(512)
    L = I.Laser(**{**wl.laser.__dict__, "model": I.MODEL_LL})
    s = oracle.evaluate(L, wl.beam, wl.bins, xi)
    assert np.array_equal(s["theta_x"], wl.beam.div_rad * xi[4])
    assert np.all(s["theta_e"] == 0)


def test_bin_rule_half_open_edges():
    L = I.Laser(a0=0.0)
    B = I.Beam(gamma_mean=1.0, rel_spread=1.0, sigma_x_um=0, sigma_y_um=0)
    bins = I.Bins(n_bins=4, lo=0.0, hi=8.0)
    # gamma0 = 1 + xi3 -> values exactly on edges and outside
    g = np.array([0.0, 1.9999, 2.0, 3.0, 6.0, 7.9999, 8.0, 9.0, -0.5])
    xi = [np.zeros_like(g)] * 8
    xi = list(xi)
    xi[3] = g - 1.0
    s = oracle.evaluate(L, B, bins, xi)
    # gamma0 is clamped at 1: the -0.5 and 0.0 entries land in bin 0
    assert list(s["bin"]) == [0, 0, 1, 1, 3, 3, 4, 4, 0]
    Lg = I.Bins(n_bins=3, lo=1.0, hi=1000.0, log_spaced=1)
    xi[3] = np.array([1.0, 10.5, 99.0, 101.0, 999.0, 1000.0, 2000.0, 1.5, 2.0]) - 1.0
    s = oracle.evaluate(L, B, Lg, xi)
    assert list(s["bin"][[1, 2, 3, 4, 6]]) == [1, 1, 2, 2, 3]


def test_gauss_hermite_rule_exactness():
    x, w = I.gauss_hermite(32)
    assert abs(w.sum() - 1) < 1e-14
    for k in range(0, 64):
        exact = 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2, dtype=np.float64)))
        val = float(np.sum(w * x ** k))
        scale = float(np.sum(w * np.abs(x) ** k))
        assert abs(val - exact) <= 1e-11 * scale, k


# --------------------------------------------------------------------------
# gradients: the oracle's dual-number gradient vs central differences of its
# plain forward (independent code paths: dual arithmetic vs plain doubles)
# --------------------------------------------------------------------------

LASER_PARAMS = ("a0", "w0_um", "dx_um", "dy_um", "delay_fs")
BEAM_PARAMS = ("gamma_mean", "rel_spread", "div_rad")


def _loss_plain(L, B, bins, sigma, xi, w, dm, dS):
    r = oracle.scatter(L, B, bins, xi, w)
    S = oracle.smooth_spectrum(L, B, bins, sigma, xi, w)
    return sum(dm.get(k, 0.0) * r["moments"][k] for k in dm) + float(np.dot(dS, S))


def _perturbed(L, B, name, value):
    if name in LASER_PARAMS:
        return I.Laser(**{**L.__dict__, name: value}), B
    return L, I.Beam(**{**B.__dict__, name: value})


@pytest.mark.parametrize("model,variant", [(I.MODEL_LL, 0), (I.MODEL_QFP, 0),
                                           (I.MODEL_LL, I.VAR_CELL_FOCUS),
                                           (I.MODEL_QFP, I.VAR_CELL_FOCUS),
                                           (I.MODEL_QFP, I.VAR_CYCLE_CHI),
                                           (I.MODEL_QFP, I.VAR_CELL_FOCUS | I.VAR_CYCLE_CHI)])
def test_oracle_gradient_vs_central_differences(model, variant):
    """The oracle's dual-number gradient (every step differentiated in dual
    arithmetic, the model variants included) against Richardson central
    differences of its plain forward (a separate code path)."""
    n = 300 if not variant & I.VAR_CYCLE_CHI else 120
    wl = I.full_qfp(n)
    L = I.Laser(**{**wl.laser.__dict__, "model": model, "n_phase": 48, "dy_um": 0.7,
                   "variant": variant})
    if variant & I.VAR_CELL_FOCUS:
        # a focus tight enough that the path through it matters, and angles
        # that move the electron sideways over the pulse
        L = I.Laser(**{**L.__dict__, "w0_um": 2.0})
    B = wl.beam
    if variant & I.VAR_CELL_FOCUS:
        B = I.Beam(**{**B.__dict__, "div_rad": 5e-3})
    xi, _ = I.workload_inputs(wl, n)
    xi = [a.astype(np.float64) for a in xi]
    w = I.rng(31).uniform(0.5, 1.5, n)
    bins = I.Bins(n_bins=128, lo=0.0, hi=6720.0)
    sigma = 2.0
    rg = I.rng(32)
    dm = {k: float(rg.normal()) for k in ("mean", "spread", "rel_spread", "div_x", "div_y", "div",
                                          "mean_aeff", "mean_gamma0")}
    dm["mean"] *= 1e-3
    dm["spread"] *= 1e-3
    dm["div_x"] *= 1e3
    dm["div_y"] *= 1e3
    dm["div"] *= 1e3
    dS = rg.normal(size=bins.n_bins) * 1e-2
    g = oracle.grad(L, B, bins, sigma, xi, w, dL_dm=dm, dL_dS=dS)["grad"]
    scale = {"a0": 30.0, "w0_um": 2.5, "dx_um": 1.0, "dy_um": 1.0, "delay_fs": 10.0,
             "gamma_mean": 4000.0, "rel_spread": 0.1, "div_rad": B.div_rad}
    for k, name in enumerate(oracle.GRAD_PARAMS):
        base = getattr(L, name) if name in LASER_PARAMS else getattr(B, name)
        h = 1e-4 * scale[name]

        def D(hh):
            lp = _loss_plain(*_perturbed(L, B, name, base + hh), bins, sigma, xi, w, dm, dS)
            lm = _loss_plain(*_perturbed(L, B, name, base - hh), bins, sigma, xi, w, dm, dS)
            return (lp - lm) / (2 * hh)

        fd = (4 * D(h / 2) - D(h)) / 3          # Richardson: O(h^4)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-9 * np.max(np.abs(g) * np.array(
            [scale[p] for p in oracle.GRAD_PARAMS])) / scale[name], (name, g[k], fd)


def test_oracle_smoothed_spectrum_conserves_weight():
    """Away from the range ends the smoothed spectrum keeps the total weight
    up to the mass beyond the 6-sigma truncation, erfc(6/sqrt2) = 1.97e-9
    (the bin-centre sum of a Gaussian of width 2 bins is exact to 1e-12)."""
    n = 500
    wl = I.full_qfp(n)
    L = I.Laser(**{**wl.laser.__dict__, "model": I.MODEL_LL})
    xi, _ = I.workload_inputs(wl, n)
    xi = [a.astype(np.float64) for a in xi]
    bins = I.Bins(n_bins=400, lo=-2000.0, hi=10000.0)
    S = oracle.smooth_spectrum(L, wl.beam, bins, 2.0, xi)
    from scipy.special import erfc
    # (the included bins are whole bins, so the cut sits within half a bin of 6 sigma)
    assert abs(S.sum() / n - (1 - erfc(6 / math.sqrt(2)))) < 1e-10


def test_continuum_mode_is_second_order_and_extrapolates():
    """The oracle's continuum-accurate mode (N, 2N, 4N cells, Richardson for
    the second-order scheme) against an independent evaluation on 4096 cells:
    where the 256-cell error is resolvable, the extrapolated value removes at
    least 95 % of it (median over samples), and the summed error over the
    samples falls by 4 (order 2 within 0.2) per halving of the cell (at 128
    cells the mean energy is still short of the asymptote: order 1.7)."""
    from dataclasses import replace
    wl = I.full_qfp(96)
    L = replace(wl.laser, n_phase=256)
    xi, _ = I.workload_inputs(wl, 96)
    xi = [a.astype(np.float64) for a in xi]
    r = oracle.continuum(L, wl.beam, xi, levels=3)
    assert r["grids"] == [256, 512, 1024]
    fine = oracle.evaluate(replace(L, n_phase=4096), wl.beam, None, xi)
    grids = [oracle.evaluate(replace(L, n_phase=n), wl.beam, None, xi) for n in (256, 512, 1024)]
    for f in ("mu", "V"):
        np.testing.assert_array_equal(r[f], grids[0][f])
        d0 = np.abs(r[f] - fine[f])
        dc = np.abs(r[f + "_c"] - fine[f])
        sel = d0 > 1e-11 * np.abs(fine[f])
        assert sel.sum() >= 20, (f, sel.sum())
        assert np.median(dc[sel] / d0[sel]) < 0.05, (f, np.median(dc[sel] / d0[sel]))
        e = [np.abs(g[f] - fine[f])[sel].sum() for g in grids]
        for k in (0, 1):
            assert abs(math.log2(e[k] / e[k + 1]) - 2.0) < 0.2, (f, k, e)
