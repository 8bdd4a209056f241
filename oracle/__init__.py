"""FP64 CPU oracle for the QScatter beam phase-space integration.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(the CUDA library and its Python binding) never does.  The oracle shares no
code with the CUDA path: it is plain C (``qs_oracle.c``) compiled with gcc,
loaded here through ctypes, plus argument marshalling.

Every function cites the passage of arXiv 2308.09348 it follows in the C
source.  Parity pins: ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qs_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libqs_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double: no contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class QsoLaser(C.Structure):
    _fields_ = [("lambda_um", C.c_double), ("a0", C.c_double), ("w0_um", C.c_double),
                ("tau_fs", C.c_double), ("dx_um", C.c_double), ("dy_um", C.c_double),
                ("delay_fs", C.c_double), ("div_prefactor", C.c_double),
                ("envelope", C.c_int32), ("model", C.c_int32), ("n_phase", C.c_int32),
                ("variant", C.c_int32)]


class QsoBeam(C.Structure):
    _fields_ = [("gamma_mean", C.c_double), ("rel_spread", C.c_double),
                ("gamma_lo", C.c_double), ("gamma_hi", C.c_double),
                ("sigma_x_um", C.c_double), ("sigma_y_um", C.c_double), ("sigma_z_um", C.c_double),
                ("div_rad", C.c_double), ("dx_um", C.c_double), ("dy_um", C.c_double),
                ("flat_energy", C.c_int32), ("pad", C.c_int32)]


class QsoBins(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("log_spaced", C.c_int32), ("lo", C.c_double),
                ("hi", C.c_double), ("n_tx", C.c_int32), ("n_ty", C.c_int32),
                ("theta_max", C.c_double), ("n_aeff", C.c_int32), ("pad", C.c_int32),
                ("aeff_max", C.c_double)]


class QsoMoments(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("W", "mean", "spread", "rel_spread", "div_x", "div_y",
                                          "div", "mean_aeff", "under", "over", "map_out",
                                          "mean_gamma0")]


SAMPLE_DTYPE = np.dtype([("gamma0", "f8"), ("aeff", "f8"), ("mu", "f8"), ("V", "f8"),
                         ("theta_e", "f8"), ("theta_x", "f8"), ("theta_y", "f8"),
                         ("gamma_out", "f8"), ("bin", "i4"), ("ix", "i4"), ("iy", "i4"),
                         ("abin", "i4")])

_DP = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.qso_constants.argtypes = [C.POINTER(QsoLaser), _DP]
            L.qso_phase_grid.argtypes = [C.POINTER(QsoLaser), _DP, _DP, _DP]
            L.qso_gaunt.argtypes = [C.c_double, _DP, _DP]
            L.qso_h2.argtypes = [C.c_double]
            L.qso_h2.restype = C.c_double
            L.qso_cycle_factors.argtypes = [C.c_double, _DP, _DP, _DP]
            L.qso_bessel_pair.argtypes = [C.c_double, _DP, _DP]
            L.qso_photon_rate.argtypes = [C.c_double] * 4
            L.qso_photon_rate.restype = C.c_double
            L.qso_photon_spectrum.argtypes = [C.POINTER(QsoLaser), C.POINTER(QsoBeam),
                                              C.POINTER(QsoBins), C.c_int64, C.POINTER(_DP),
                                              _DP, _DP]
            L.qso_photon_spectrum.restype = C.c_int
            L.qso_photon_spectrum2.argtypes = [C.POINTER(QsoLaser), C.POINTER(QsoBeam),
                                               C.POINTER(QsoBins), C.c_int64, C.POINTER(_DP),
                                               _DP, _DP, _DP]
            L.qso_photon_spectrum2.restype = C.c_int
            L.qso_pw_reconstruct.argtypes = [C.c_int, C.c_int, C.c_int, _DP, _DP, _DP]
            L.qso_bessel_i0.argtypes = [C.c_double]
            L.qso_bessel_i0.restype = C.c_double
            L.qso_analytic_aeff.argtypes = [C.POINTER(QsoLaser), C.c_int, _DP, C.c_int, _DP, _DP]
            L.qso_analytic_ll.argtypes = [C.POINTER(QsoLaser), C.c_int, _DP, C.c_double, C.c_int,
                                          _DP, _DP]
            L.qso_qfp_rates.argtypes = [C.POINTER(QsoLaser), C.c_double, C.c_double, C.c_double, _DP]
            L.qso_qfp_integrate.argtypes = [C.POINTER(QsoLaser), C.c_double, C.c_double, C.c_double,
                                            C.c_double, C.c_double, _DP, _DP]
            L.qso_eval.argtypes = [C.POINTER(QsoLaser), C.POINTER(QsoBeam), C.POINTER(QsoBins),
                                   C.c_int64, C.POINTER(_DP), C.c_void_p]
            L.qso_scatter.argtypes = [C.POINTER(QsoLaser), C.POINTER(QsoBeam), C.POINTER(QsoBins),
                                      C.c_int64, C.POINTER(_DP), _DP, _DP, _DP, _DP,
                                      C.POINTER(QsoMoments)]
            L.qso_scatter.restype = C.c_int
            L.qso_grad.argtypes = [C.POINTER(QsoLaser), C.POINTER(QsoBeam), C.POINTER(QsoBins),
                                   C.c_double, C.c_int64, C.POINTER(_DP), _DP, _DP, _DP, _DP,
                                   _DP, C.POINTER(QsoMoments)]
            L.qso_grad.restype = C.c_int
            L.qso_smooth_spectrum.argtypes = [C.POINTER(QsoLaser), C.POINTER(QsoBeam),
                                              C.POINTER(QsoBins), C.c_double, C.c_int64,
                                              C.POINTER(_DP), _DP, _DP]
            L.qso_smooth_spectrum.restype = C.c_int
            _lib = L
    return _lib


# ---- marshalling from the workload descriptions (inputs.Laser/Beam/Bins) ----

def _laser(p) -> QsoLaser:
    return QsoLaser(p.lambda_um, p.a0, p.w0_um, p.tau_fs, p.dx_um, p.dy_um, p.delay_fs,
                    p.div_prefactor, int(p.envelope), int(p.model), int(p.n_phase),
                    int(getattr(p, "variant", 0)))


def _beam(b) -> QsoBeam:
    return QsoBeam(b.gamma_mean, b.rel_spread, b.gamma_lo, b.gamma_hi, b.sigma_x_um,
                   b.sigma_y_um, b.sigma_z_um, b.div_rad, b.dx_um, b.dy_um,
                   int(b.flat_energy), 0)


def _bins(b) -> QsoBins:
    return QsoBins(int(b.n_bins), int(b.log_spaced), b.lo, b.hi, int(b.n_tx), int(b.n_ty),
                   b.theta_max, int(b.n_aeff), 0, b.aeff_max)


def _ptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _streams(xi, n):
    arrs = []
    for k in range(8):
        a = xi[k] if k < len(xi) else None
        if a is None:
            arrs.append(None)
        else:
            a = np.ascontiguousarray(a, dtype=np.float64)
            assert a.shape == (n,)
            arrs.append(a)
    ptrs = (_DP * 8)(*[(_ptr(a) if a is not None else _DP()) for a in arrs])
    return arrs, ptrs


CONSTANT_NAMES = ("k", "omega0", "zR", "Rc", "aS", "Phi", "PhiT", "win_lo", "win_hi", "cRR")


def constants(laser) -> dict:
    out = np.zeros(10)
    lib().qso_constants(C.byref(_laser(laser)), _ptr(out))
    return dict(zip(CONSTANT_NAMES, out.tolist()))


def phase_grid(laser):
    n = int(laser.n_phase)
    phi = np.zeros(n)
    G = np.zeros(n)
    h = np.zeros(1)
    lib().qso_phase_grid(C.byref(_laser(laser)), _ptr(phi), _ptr(G), _ptr(h))
    return phi, G, float(h[0])


def gaunt(chi: float):
    g = np.zeros(1)
    gp = np.zeros(1)
    lib().qso_gaunt(float(chi), _ptr(g), _ptr(gp))
    return float(g[0]), float(gp[0])


def h2(chi: float) -> float:
    return float(lib().qso_h2(float(chi)))


def cycle_factors(chi: float):
    """Cycle-resolved Gaunt and diffusion factors (G, S = 2G + chi G', H)."""
    G, S, H = C.c_double(), C.c_double(), C.c_double()
    lib().qso_cycle_factors(float(chi), C.byref(G), C.byref(S), C.byref(H))
    return G.value, S.value, H.value


def qfp_rates(laser, mu: float, A: float, aS_scale: float = 1.0) -> dict:
    out = np.zeros(4)
    lib().qso_qfp_rates(C.byref(_laser(laser)), float(mu), float(A), float(aS_scale), _ptr(out))
    return dict(D1=out[0], dD1=out[1], D2=out[2], chi=out[3])


def qfp_integrate(laser, aeff: float, gamma0: float, V0: float = 0.0, aS_scale: float = 1.0,
                  d2_scale: float = 1.0):
    mu = np.zeros(1)
    V = np.zeros(1)
    lib().qso_qfp_integrate(C.byref(_laser(laser)), float(aeff), float(gamma0), float(V0),
                            float(aS_scale), float(d2_scale), _ptr(mu), _ptr(V))
    return float(mu[0]), float(V[0])


def evaluate(laser, beam, bins, xi) -> np.ndarray:
    """Per-sample evaluation; ``xi`` is a list of up to 8 arrays (None = zeros)."""
    n = next(len(a) for a in xi if a is not None)
    arrs, ptrs = _streams(xi, n)
    out = np.zeros(n, dtype=SAMPLE_DTYPE)
    bn = _bins(bins) if bins is not None else None
    lib().qso_eval(C.byref(_laser(laser)), C.byref(_beam(beam)),
                   C.byref(bn) if bn is not None else None, n, ptrs,
                   out.ctypes.data_as(C.c_void_p))
    return out


def continuum(laser, beam, xi, levels: int = 3) -> dict:
    """Continuum-accurate mode of the phase integration (Eq. 6 with the
    Fokker-Planck closure): every sample evaluated with n_phase, 2 n_phase,
    ... (``levels`` doublings of the midpoint grid over the same window, at
    most 4096 cells) and Richardson-extrapolated for the scheme's second
    order, f_c = (4 f(2N) - f(N)) / 3 from the two finest grids.  Returns the
    per-sample mean energy and variance at n_phase (``mu``, ``V``), their
    extrapolated continuum values (``mu_c``, ``V_c``), the discretisation
    error of n_phase relative to them (``err_mu``, ``err_V``) and the
    observed order log2(|f(N) - f(2N)| / |f(2N) - f(4N)|) per sample
    (``order``, NaN where the differences vanish)."""
    from dataclasses import replace
    n0 = int(laser.n_phase)
    grids = [n0 << k for k in range(levels)]
    if levels < 2 or grids[-1] > 4096:
        raise ValueError("continuum: 2 to log2(4096 / n_phase) + 1 levels")
    rec = [evaluate(replace(laser, n_phase=n), beam, None, xi) for n in grids]
    out = {"n_phase": n0, "grids": grids}
    for f in ("mu", "V"):
        v = [r[f].astype(np.float64) for r in rec]
        fc = (4.0 * v[-1] - v[-2]) / 3.0
        out[f] = v[0]
        out[f + "_c"] = fc
        with np.errstate(divide="ignore", invalid="ignore"):
            out["err_" + f] = np.abs(v[0] - fc) / np.abs(fc)
            if levels >= 3:
                out["order_" + f] = np.log2(np.abs(v[0] - v[1]) / np.abs(v[1] - v[2]))
    return out


def scatter(laser, beam, bins, xi, w=None) -> dict:
    """Whole-beam integration: spectrum, divergence map, a_eff histogram, moments."""
    n = next(len(a) for a in xi if a is not None)
    arrs, ptrs = _streams(xi, n)
    w64 = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    spec = np.zeros(max(int(bins.n_bins), 0))
    nmap = int(bins.n_tx) * int(bins.n_ty) if (bins.n_tx > 0 and bins.n_ty > 0) else 0
    dmap = np.zeros(nmap)
    ah = np.zeros(max(int(bins.n_aeff), 0))
    m = QsoMoments()
    rc = lib().qso_scatter(C.byref(_laser(laser)), C.byref(_beam(beam)), C.byref(_bins(bins)), n,
                           ptrs, _ptr(w64), _ptr(spec) if spec.size else None,
                           _ptr(dmap) if dmap.size else None, _ptr(ah) if ah.size else None,
                           C.byref(m))
    if rc != 0:
        raise MemoryError("oracle scatter: allocation failed")
    mom = {k: getattr(m, k) for k, _ in QsoMoments._fields_}
    return dict(spectrum=spec, divmap=dmap.reshape(int(bins.n_ty), int(bins.n_tx)) if nmap else dmap,
                aeff_hist=ah, moments=mom)


# parameter order of the gradient
GRAD_PARAMS = ("a0", "w0_um", "dx_um", "dy_um", "delay_fs", "gamma_mean", "rel_spread", "div_rad")
MOMENT_NAMES = tuple(k for k, _ in QsoMoments._fields_)


def smooth_spectrum(laser, beam, bins, sigma_bins, xi, w=None) -> np.ndarray:
    """Kernel-smoothed spectrum (plain FP64 evaluation)."""
    n = next(len(a) for a in xi if a is not None)
    arrs, ptrs = _streams(xi, n)
    w64 = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    S = np.zeros(int(bins.n_bins))
    rc = lib().qso_smooth_spectrum(C.byref(_laser(laser)), C.byref(_beam(beam)),
                                   C.byref(_bins(bins)), float(sigma_bins), n, ptrs, _ptr(w64),
                                   _ptr(S))
    if rc != 0:
        raise ValueError("smoothed spectrum needs uniform bins and sigma_bins > 0")
    return S


def grad(laser, beam, bins, sigma_bins, xi, w=None, dL_dm=None, dL_dS=None) -> dict:
    """Forward-mode (dual number) gradient of L = dL_dm . m + dL_dS . S with
    respect to GRAD_PARAMS; also returns the forward smoothed spectrum and
    moments.  dL_dm: dict by moment name or array of 13 (qso_moments order)."""
    n = next(len(a) for a in xi if a is not None)
    arrs, ptrs = _streams(xi, n)
    w64 = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    dm = np.zeros(13)
    if isinstance(dL_dm, dict):
        for k, v in dL_dm.items():
            dm[MOMENT_NAMES.index(k)] = v
    elif dL_dm is not None:
        dm[:] = dL_dm
    dS = None if dL_dS is None else np.ascontiguousarray(dL_dS, dtype=np.float64)
    g = np.zeros(8)
    S = np.zeros(int(bins.n_bins))
    m = QsoMoments()
    rc = lib().qso_grad(C.byref(_laser(laser)), C.byref(_beam(beam)), C.byref(_bins(bins)),
                        float(sigma_bins), n, ptrs, _ptr(w64), _ptr(dm), _ptr(dS), _ptr(g),
                        _ptr(S), C.byref(m))
    if rc != 0:
        raise ValueError("oracle gradient: bad arguments (uniform bins, sigma_bins > 0)")
    return dict(grad=g, smooth=S, moments={k: getattr(m, k) for k in MOMENT_NAMES})


def bessel_pair(y: float):
    """(K_{2/3}(y), integral of K_{1/3} from y to infinity)."""
    a, b = C.c_double(), C.c_double()
    lib().qso_bessel_pair(float(y), C.byref(a), C.byref(b))
    return a.value, b.value


def photon_rate(aS: float, mu: float, chi: float, eps: float) -> float:
    """Photons per unit phase and unit photon energy (m c^2) of an electron of
    mean energy mu at chi (LCFA quantum-synchrotron spectrum)."""
    return lib().qso_photon_rate(float(aS), float(mu), float(chi), float(eps))


def photon_spectrum_angles(laser, beam, pbins, xi, w=None):
    """(S, T): the photon spectrum and its angle-weighted moments T[0] (x,
    the polarisation axis) and T[1] (y); T/S is the mean square photon angle
    at each bin centre (Eq. 7)."""
    n = next(len(a) for a in xi if a is not None)
    arrs, ptrs = _streams(xi, n)
    w64 = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(int(pbins.n_bins))
    th = np.zeros(2 * int(pbins.n_bins))
    rc = lib().qso_photon_spectrum2(C.byref(_laser(laser)), C.byref(_beam(beam)),
                                    C.byref(_bins(pbins)), n, ptrs, _ptr(w64), _ptr(out),
                                    _ptr(th))
    if rc != 0:
        raise ValueError("photon spectrum needs the quantum model and valid bins")
    return out, th.reshape(2, -1)


def photon_spectrum(laser, beam, pbins, xi, w=None) -> np.ndarray:
    """Beam photon spectrum dN/deps at the centres of the photon-energy bins
    ``pbins`` (n_bins, lo, hi, log_spaced; eps in m c^2)."""
    n = next(len(a) for a in xi if a is not None)
    arrs, ptrs = _streams(xi, n)
    w64 = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(int(pbins.n_bins))
    rc = lib().qso_photon_spectrum(C.byref(_laser(laser)), C.byref(_beam(beam)),
                                   C.byref(_bins(pbins)), n, ptrs, _ptr(w64), _ptr(out))
    if rc != 0:
        raise ValueError("photon spectrum needs the quantum model and valid bins")
    return out


def pw_reconstruct(hist, pw) -> np.ndarray:
    """Eq. 5: out[s, b] = sum_k hist[s, k] pw[k, b] (hist: shots x a-bins,
    pw: a-bins x energy bins)."""
    hist = np.ascontiguousarray(np.atleast_2d(hist), dtype=np.float64)
    pw = np.ascontiguousarray(pw, dtype=np.float64)
    ns, na = hist.shape
    nb = pw.shape[1]
    assert pw.shape[0] == na
    out = np.zeros((ns, nb))
    lib().qso_pw_reconstruct(ns, na, nb, _ptr(hist), _ptr(pw), _ptr(out))
    return out


GEOMETRIES = {"short": 0, "thin": 1, "wide": 2}


def bessel_i0(x: float) -> float:
    return lib().qso_bessel_i0(float(x))


def _geom_par(radius=0.0, length=0.0, d_perp=0.0, d_par=0.0, n=1.0):
    return np.array([radius, length, d_perp, d_par, n], dtype=np.float64)


def analytic_aeff(laser, geom, a, **par) -> np.ndarray:
    """Table 1: dN/da_eff on the grid ``a`` for an idealised beam ("short":
    radius R in the collision plane; "thin": on axis, flat-top length; "wide":
    uniform density n across the laser) with offsets d_perp, d_par."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros_like(a)
    lib().qso_analytic_aeff(C.byref(_laser(laser)), GEOMETRIES[geom], _ptr(_geom_par(**par)),
                            a.size, _ptr(a), _ptr(out))
    return out


def analytic_ll(laser, geom, gamma0, g, **par) -> np.ndarray:
    """Table 2 (via Eq. 6): the classical final-energy density dN/dgamma."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros_like(g)
    lib().qso_analytic_ll(C.byref(_laser(laser)), GEOMETRIES[geom], _ptr(_geom_par(**par)),
                          float(gamma0), g.size, _ptr(g), _ptr(out))
    return out
