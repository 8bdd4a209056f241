"""Thin ctypes binding of libqscatter (argument marshalling only).

Every step of the beam phase-space integration runs in the library's CUDA
kernels; this module converts workload descriptions and torch tensors into
the C structs of ``include/qscatter.h`` and calls the entry points of the same
names.  There is no CPU fallback: if the shared library is missing or fails to
load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import inputs as _inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqscatter.so")

(QS_OK, QS_ERR_INVALID_ARG, QS_ERR_CUDA, QS_ERR_WORKSPACE, QS_ERR_UNSUPPORTED, QS_ERR_TIMEOUT,
 QS_ERR_NONFINITE) = range(7)
QS_F32, QS_F64 = 0, 1
QS_EXEC_CHECK_FINITE = 1


class QsError(RuntimeError):
    def __init__(self, status: int, fn: str):
        msg = _lib().qs_status_string(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{fn}: {msg} (status {status})")
        self.status = status


class qs_laser(C.Structure):
    _fields_ = [("lambda_um", C.c_double), ("a0", C.c_double), ("w0_um", C.c_double),
                ("tau_fs", C.c_double), ("dx_um", C.c_double), ("dy_um", C.c_double),
                ("delay_fs", C.c_double), ("div_prefactor", C.c_double),
                ("envelope", C.c_int32), ("model", C.c_int32), ("n_phase", C.c_int32),
                ("variant", C.c_int32)]


class qs_beam(C.Structure):
    _fields_ = [("gamma_mean", C.c_double), ("rel_spread", C.c_double),
                ("gamma_lo", C.c_double), ("gamma_hi", C.c_double),
                ("sigma_x_um", C.c_double), ("sigma_y_um", C.c_double),
                ("sigma_z_um", C.c_double), ("div_rad", C.c_double),
                ("dx_um", C.c_double), ("dy_um", C.c_double),
                ("flat_energy", C.c_int32), ("reserved", C.c_int32)]


class qs_samples(C.Structure):
    _fields_ = [("n", C.c_int64), ("xi", C.c_void_p * 8), ("w", C.c_void_p),
                ("dtype", C.c_int32), ("reserved", C.c_int32)]


class qs_bins(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("log_spaced", C.c_int32), ("lo", C.c_double),
                ("hi", C.c_double), ("n_tx", C.c_int32), ("n_ty", C.c_int32),
                ("theta_max", C.c_double), ("n_aeff", C.c_int32), ("reserved", C.c_int32),
                ("aeff_max", C.c_double), ("smooth_sigma_bins", C.c_double)]


MOMENT_FIELDS = ("W", "mean", "spread", "rel_spread", "div_x", "div_y", "div", "mean_aeff",
                 "under", "over", "map_out", "mean_gamma0", "nonfinite")


class qs_moments(C.Structure):
    _fields_ = [(k, C.c_double) for k in MOMENT_FIELDS]


class qs_exec(C.Structure):
    _fields_ = [("precision", C.c_int32), ("weight_frac_bits", C.c_int32),
                ("block", C.c_int32), ("grid", C.c_int32), ("tile", C.c_int32),
                ("flags", C.c_int32), ("ev_start", C.c_void_p), ("ev_stop", C.c_void_p)]


class qs_geometry(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("radius_um", C.c_double),
                ("length_um", C.c_double), ("d_perp_um", C.c_double), ("d_par_um", C.c_double),
                ("count", C.c_double)]


GEOMETRIES = {"short": 0, "thin": 1, "wide": 2}


def make_geometry(geom, radius=0.0, length=0.0, d_perp=0.0, d_par=0.0, n=1.0) -> qs_geometry:
    return qs_geometry(GEOMETRIES[geom], 0, float(radius), float(length), float(d_perp),
                       float(d_par), float(n))


class qs_sample_out(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("gamma0", "aeff", "mu", "V", "theta_e", "theta_x",
                                          "theta_y", "gamma_out", "bin", "ix", "iy", "abin")]


_LIB = None
_lock = threading.Lock()
_VP = C.c_void_p


def _lib():
    global _LIB
    with _lock:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libqscatter is not built ({LIB_PATH} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            L.qs_version.restype = C.c_int32
            L.qs_status_string.argtypes = [C.c_int32]
            L.qs_status_string.restype = C.c_char_p
            L.qs_workspace_bytes.argtypes = [C.POINTER(qs_bins), C.POINTER(qs_exec), C.c_int64]
            L.qs_workspace_bytes.restype = C.c_size_t
            L.qs_scatter.argtypes = [C.POINTER(qs_laser), C.POINTER(qs_beam),
                                     C.POINTER(qs_samples), C.POINTER(qs_bins),
                                     C.POINTER(qs_exec), _VP, _VP, _VP, _VP, _VP, _VP,
                                     C.c_size_t, _VP]
            L.qs_scatter.restype = C.c_int32
            L.qs_eval_samples.argtypes = [C.POINTER(qs_laser), C.POINTER(qs_beam),
                                          C.POINTER(qs_samples), C.POINTER(qs_bins),
                                          C.POINTER(qs_exec), C.POINTER(qs_sample_out), _VP]
            L.qs_eval_samples.restype = C.c_int32
            L.qs_scatter_noalloc.argtypes = [C.POINTER(qs_laser), C.POINTER(qs_beam),
                                             C.POINTER(qs_samples), C.POINTER(qs_bins),
                                             C.POINTER(qs_exec), _VP, _VP, _VP, _VP, _VP, _VP]
            L.qs_scatter_noalloc.restype = C.c_int32
            L.qs_scatter_grad.argtypes = [C.POINTER(qs_laser), C.POINTER(qs_beam),
                                          C.POINTER(qs_samples), C.POINTER(qs_bins),
                                          C.POINTER(qs_exec), _VP, _VP, _VP, _VP, _VP,
                                          C.c_size_t, _VP]
            L.qs_scatter_grad.restype = C.c_int32
            L.qs_host_workspace_bytes.argtypes = [C.POINTER(qs_bins), C.POINTER(qs_exec),
                                                  C.POINTER(qs_samples), C.c_int64]
            L.qs_host_workspace_bytes.restype = C.c_size_t
            L.qs_scatter_host.argtypes = [C.POINTER(qs_laser), C.POINTER(qs_beam),
                                          C.POINTER(qs_samples), C.POINTER(qs_bins),
                                          C.POINTER(qs_exec), C.c_int64, _VP, _VP, _VP, _VP,
                                          _VP, _VP, C.c_size_t, _VP]
            L.qs_scatter_host.restype = C.c_int32
            L.qs_batch_workspace_bytes.argtypes = [C.c_int32, C.c_int64, C.POINTER(qs_bins),
                                                   C.c_int32, C.POINTER(qs_exec), C.c_int32]
            L.qs_batch_workspace_bytes.restype = C.c_size_t
            L.qs_scatter_batch.argtypes = [C.c_int32, _VP, _VP, _VP, C.POINTER(qs_samples),
                                           C.POINTER(qs_bins), _VP, C.c_int32,
                                           C.POINTER(qs_exec), _VP, _VP, _VP, _VP, _VP, _VP,
                                           C.c_size_t, _VP]
            L.qs_scatter_batch.restype = C.c_int32
            L.qs_scatter_grad_batch.argtypes = [C.c_int32, _VP, _VP, _VP, C.POINTER(qs_samples),
                                                C.POINTER(qs_bins), _VP, C.c_int32,
                                                C.POINTER(qs_exec), _VP, _VP, _VP, _VP, _VP,
                                                C.c_size_t, _VP]
            L.qs_scatter_grad_batch.restype = C.c_int32
            L.qs_photon_workspace_bytes.argtypes = [C.POINTER(qs_bins), C.POINTER(qs_exec),
                                                    C.c_int64]
            L.qs_photon_workspace_bytes.restype = C.c_size_t
            L.qs_photon_spectrum.argtypes = [C.POINTER(qs_laser), C.POINTER(qs_beam),
                                             C.POINTER(qs_samples), C.POINTER(qs_bins),
                                             C.POINTER(qs_exec), _VP, _VP, _VP, C.c_size_t, _VP]
            L.qs_photon_spectrum.restype = C.c_int32
            L.qs_pw_reconstruct.argtypes = [C.c_int32, C.c_int32, C.c_int32, _VP, _VP, _VP, _VP]
            L.qs_pw_reconstruct.restype = C.c_int32
            L.qs_analytic_aeff.argtypes = [C.POINTER(qs_laser), C.POINTER(qs_geometry),
                                           C.c_int64, _VP, _VP, _VP]
            L.qs_analytic_aeff.restype = C.c_int32
            L.qs_analytic_ll_spectrum.argtypes = [C.POINTER(qs_laser), C.POINTER(qs_geometry),
                                                  C.c_double, C.c_int64, _VP, _VP, _VP]
            L.qs_analytic_ll_spectrum.restype = C.c_int32
            L.qs_unit_rates_scratch_bytes.restype = C.c_size_t
            L.qs_unit_rates.argtypes = [C.POINTER(C.c_double), _VP, C.c_size_t, _VP]
            L.qs_unit_rates.restype = C.c_int32
            _LIB = L
    return _LIB


def lib():
    """The loaded shared library (raises if it is not built)."""
    return _lib()


# ---- descriptor marshalling ---------------------------------------------

def make_laser(p: _inputs.Laser) -> qs_laser:
    return qs_laser(p.lambda_um, p.a0, p.w0_um, p.tau_fs, p.dx_um, p.dy_um, p.delay_fs,
                    p.div_prefactor, int(p.envelope), int(p.model), int(p.n_phase),
                    int(p.variant))


def make_beam(b: _inputs.Beam) -> qs_beam:
    return qs_beam(b.gamma_mean, b.rel_spread, b.gamma_lo, b.gamma_hi, b.sigma_x_um,
                   b.sigma_y_um, b.sigma_z_um, b.div_rad, b.dx_um, b.dy_um,
                   int(b.flat_energy), 0)


def make_bins(b: _inputs.Bins) -> qs_bins:
    return qs_bins(int(b.n_bins), int(b.log_spaced), b.lo, b.hi, int(b.n_tx), int(b.n_ty),
                   b.theta_max, int(b.n_aeff), 0, b.aeff_max, float(b.smooth_sigma_bins))


def _event_handle(ev):
    """cudaEvent_t of a torch.cuda.Event (torch creates it at first record)."""
    if ev.cuda_event == 0:
        ev.record()
    return ev.cuda_event


def make_exec(precision="f32", weight_frac_bits=0, block=0, grid=0, events=None,
              tile=0, check_finite=False) -> qs_exec:
    prec = QS_F64 if precision in ("f64", QS_F64, torch.float64) else QS_F32
    e0, e1 = (None, None) if events is None else (_event_handle(events[0]),
                                                  _event_handle(events[1]))
    flags = QS_EXEC_CHECK_FINITE if check_finite else 0
    return qs_exec(prec, int(weight_frac_bits), int(block), int(grid), int(tile), flags, e0, e1)


def make_samples(xi, w=None) -> tuple[qs_samples, list]:
    """xi: list of up to 8 CUDA tensors (None = zeros) of one float dtype."""
    xs = list(xi) + [None] * (8 - len(xi))
    ref = next((t for t in xs if t is not None), None)
    if ref is None:
        raise ValueError("at least one sample stream is required")
    dt = ref.dtype
    if dt not in (torch.float32, torch.float64):
        raise TypeError("sample streams must be float32 or float64")
    n = ref.numel()
    keep = []
    ptrs = []
    for t in xs:
        if t is None:
            ptrs.append(None)
            continue
        if t.dtype != dt or t.numel() != n or not t.is_cuda:
            raise ValueError("sample streams must be CUDA tensors of one dtype and length")
        t = t.contiguous()
        keep.append(t)
        ptrs.append(t.data_ptr())
    wp = None
    if w is not None:
        if w.dtype != dt or w.numel() != n or not w.is_cuda:
            raise ValueError("weights must match the sample streams")
        w = w.contiguous()
        keep.append(w)
        wp = w.data_ptr()
    s = qs_samples(n, (C.c_void_p * 8)(*ptrs), wp, QS_F32 if dt == torch.float32 else QS_F64, 0)
    return s, keep


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check(status: int, fn: str):
    if status != QS_OK:
        raise QsError(status, fn)


# ---- entry points ---------------------------------------------------------

def workspace_bytes(bins: _inputs.Bins, n: int, precision="f32", block=0, grid=0) -> int:
    b = make_bins(bins)
    e = make_exec(precision, 0, block, grid)
    v = _lib().qs_workspace_bytes(C.byref(b), C.byref(e), int(n))
    if v == 0:
        raise QsError(QS_ERR_INVALID_ARG, "qs_workspace_bytes")
    return int(v)


class Outputs:
    """Device buffers of one qs_scatter call (reusable across calls)."""

    def __init__(self, bins: _inputs.Bins, n: int, device=None, precision="f32", block=0,
                 grid=0):
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.bins = bins
        self.spectrum = torch.zeros(max(bins.n_bins, 0), dtype=torch.float64, device=dev)
        nmap = bins.n_tx * bins.n_ty if (bins.n_tx > 0 and bins.n_ty > 0) else 0
        self.divmap = torch.zeros(nmap, dtype=torch.float64, device=dev)
        self.aeff_hist = torch.zeros(max(bins.n_aeff, 0), dtype=torch.float64, device=dev)
        self.spec_smooth = torch.zeros(max(bins.n_bins, 0) if bins.smooth_sigma_bins > 0 else 0,
                                       dtype=torch.float64, device=dev)
        self.moments = torch.zeros(len(MOMENT_FIELDS), dtype=torch.float64, device=dev)
        nbytes = workspace_bytes(bins, n, precision, block, grid)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        self.ws_bytes = nbytes

    def moments_dict(self) -> dict:
        v = self.moments.cpu().tolist()
        return dict(zip(MOMENT_FIELDS, v))

    def result(self) -> dict:
        nm = self.divmap
        if self.bins.n_tx > 0:
            nm = nm.view(self.bins.n_ty, self.bins.n_tx)
        return dict(spectrum=self.spectrum, divmap=nm, aeff_hist=self.aeff_hist,
                    spec_smooth=self.spec_smooth, moments=self.moments_dict())


def _ptr_or_none(t):
    return t.data_ptr() if (t is not None and t.numel() > 0) else None


def qs_scatter(laser, beam, xi, bins, w=None, precision="f32", out: Outputs | None = None,
               block=0, grid=0, weight_frac_bits=0, stream=None, kernel_events=None,
               check_finite=False) -> Outputs:
    """Integrate the beam phase space: spectra + moments (asynchronous).

    ``kernel_events``: optional (start, stop) torch.cuda.Event pair recorded
    around the evaluation kernel on the call's stream.  ``check_finite``:
    wait for the call and raise QsError (QS_ERR_NONFINITE) if samples were
    excluded as non-finite (the outputs are written all the same)."""
    s, keep = make_samples(xi, w)
    if out is None:
        out = Outputs(bins, s.n, keep[0].device, precision, block, grid)
    L, B, Bn = make_laser(laser), make_beam(beam), make_bins(bins)
    E = make_exec(precision, weight_frac_bits, block, grid, kernel_events,
                  check_finite=check_finite)
    st = _lib().qs_scatter(C.byref(L), C.byref(B), C.byref(s), C.byref(Bn), C.byref(E),
                           _ptr_or_none(out.spectrum), _ptr_or_none(out.divmap),
                           _ptr_or_none(out.aeff_hist), _ptr_or_none(out.spec_smooth),
                           out.moments.data_ptr(), out.ws_ptr, out.ws_bytes, _stream_ptr(stream))
    _check(st, "qs_scatter")
    return out


SAMPLE_FIELDS_F = ("gamma0", "aeff", "mu", "V", "theta_e", "theta_x", "theta_y", "gamma_out")
SAMPLE_FIELDS_I = ("bin", "ix", "iy", "abin")


def qs_eval_samples(laser, beam, xi, bins=None, precision="f32", stream=None) -> dict:
    """Per-sample records (dict of CUDA tensors)."""
    s, keep = make_samples(xi, None)
    dev = keep[0].device
    n = s.n
    res = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in SAMPLE_FIELDS_F}
    res.update({k: torch.empty(n, dtype=torch.int32, device=dev) for k in SAMPLE_FIELDS_I})
    o = qs_sample_out(*[res[k].data_ptr() if n else None
                        for k in SAMPLE_FIELDS_F + SAMPLE_FIELDS_I])
    L, B = make_laser(laser), make_beam(beam)
    Bn = make_bins(bins) if bins is not None else None
    E = make_exec(precision)
    st = _lib().qs_eval_samples(C.byref(L), C.byref(B), C.byref(s),
                                C.byref(Bn) if Bn is not None else None, C.byref(E),
                                C.byref(o), _stream_ptr(stream))
    _check(st, "qs_eval_samples")
    return res


class _OutputsNoWorkspace(Outputs):
    """Output buffers only (qs_scatter_noalloc needs no workspace)."""

    def __init__(self, bins: _inputs.Bins, device):
        self.bins = bins
        self.spectrum = torch.zeros(max(bins.n_bins, 0), dtype=torch.float64, device=device)
        nmap = bins.n_tx * bins.n_ty if (bins.n_tx > 0 and bins.n_ty > 0) else 0
        self.divmap = torch.zeros(nmap, dtype=torch.float64, device=device)
        self.aeff_hist = torch.zeros(max(bins.n_aeff, 0), dtype=torch.float64, device=device)
        self.spec_smooth = torch.zeros(max(bins.n_bins, 0) if bins.smooth_sigma_bins > 0 else 0,
                                       dtype=torch.float64, device=device)
        self.moments = torch.zeros(len(MOMENT_FIELDS), dtype=torch.float64, device=device)
        self.workspace = None
        self.ws_ptr = None
        self.ws_bytes = 0


def qs_scatter_noalloc(laser, beam, xi, bins, w=None, precision="f32", out: Outputs | None = None,
                       block=0, grid=0, weight_frac_bits=0, stream=None) -> Outputs:
    """qs_scatter without a workspace: the library's static device scratch is
    used (for callers that cannot allocate device memory).  ``out`` supplies
    the output buffers; its workspace, if any, is not touched."""
    s, keep = make_samples(xi, w)
    if out is None:
        out = _OutputsNoWorkspace(bins, keep[0].device)
    L, B, Bn = make_laser(laser), make_beam(beam), make_bins(bins)
    E = make_exec(precision, weight_frac_bits, block, grid)
    st = _lib().qs_scatter_noalloc(C.byref(L), C.byref(B), C.byref(s), C.byref(Bn), C.byref(E),
                                   _ptr_or_none(out.spectrum), _ptr_or_none(out.divmap),
                                   _ptr_or_none(out.aeff_hist), _ptr_or_none(out.spec_smooth),
                                   out.moments.data_ptr(), _stream_ptr(stream))
    _check(st, "qs_scatter_noalloc")
    return out


def qs_photon_spectrum(laser, beam, xi, pbins, w=None, precision="f32", out=None,
                       workspace=None, block=0, grid=0, stream=None, kernel_events=None,
                       theta2=None):
    """Photon spectrum dN/deps (eps in m c^2) of the beam at the centres of
    the photon-energy bins ``pbins`` (n_bins, lo, hi, log_spaced).  With
    ``theta2`` (a 2 x n_bins float64 device tensor, or True to allocate one)
    also the angle-weighted sums of Eq. 7; returns (spectrum, theta2) then."""
    s, keep = make_samples(xi, w)
    dev = keep[0].device
    Bn = make_bins(pbins)
    E = make_exec(precision, 0, block, grid, kernel_events)
    if out is None:
        out = torch.zeros(int(pbins.n_bins), dtype=torch.float64, device=dev)
    nbytes = int(_lib().qs_photon_workspace_bytes(C.byref(Bn), C.byref(E), s.n))
    if nbytes == 0:
        _check(QS_ERR_INVALID_ARG, "qs_photon_workspace_bytes")
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    L, B = make_laser(laser), make_beam(beam)
    if theta2 is True:
        theta2 = torch.zeros(2, int(pbins.n_bins), dtype=torch.float64, device=dev)
    st = _lib().qs_photon_spectrum(C.byref(L), C.byref(B), C.byref(s), C.byref(Bn), C.byref(E),
                                   out.data_ptr(), None if theta2 is None else theta2.data_ptr(),
                                   workspace.data_ptr(), nbytes, _stream_ptr(stream))
    _check(st, "qs_photon_spectrum")
    return out if theta2 is None else (out, theta2)


GRAD_PARAMS = ("a0", "w0_um", "dx_um", "dy_um", "delay_fs", "gamma_mean", "rel_spread", "div_rad")


def qs_scatter_grad(laser, beam, xi, bins, moments, dL_dmoments, dL_dsmooth=None, w=None,
                    precision="f32", out: Outputs | None = None, block=0, grid=0,
                    stream=None) -> torch.Tensor:
    """Gradient (8 doubles, GRAD_PARAMS order) of a loss given its upstream
    gradient with respect to the 13 moments (and the smoothed spectrum)."""
    s, keep = make_samples(xi, w)
    dev = keep[0].device
    if out is None:
        out = Outputs(bins, s.n, dev, precision, block, grid)
    mom = moments.to(device=dev, dtype=torch.float64).contiguous()
    dm = dL_dmoments.to(device=dev, dtype=torch.float64).contiguous()
    dS = None if dL_dsmooth is None else dL_dsmooth.to(device=dev, dtype=torch.float64).contiguous()
    g = torch.empty(8, dtype=torch.float64, device=dev)
    L, B, Bn = make_laser(laser), make_beam(beam), make_bins(bins)
    E = make_exec(precision, 0, block, grid)
    st = _lib().qs_scatter_grad(C.byref(L), C.byref(B), C.byref(s), C.byref(Bn), C.byref(E),
                                mom.data_ptr(), dm.data_ptr(),
                                dS.data_ptr() if dS is not None else None, g.data_ptr(),
                                out.ws_ptr, out.ws_bytes, _stream_ptr(stream))
    _check(st, "qs_scatter_grad")
    return g


# ---- batched shots ----------------------------------------------------------

def _struct_array_to_device(structs, ctype, device) -> torch.Tensor:
    arr = (ctype * len(structs))(*structs)
    raw = bytes(memoryview(arr).cast("B"))
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


class Batch:
    """Device-side descriptors, outputs and workspace of one qs_scatter_batch
    problem shape (reusable across calls and capturable in a CUDA graph).
    With ``bins.smooth_sigma_bins > 0`` the kernel-smoothed spectra are
    produced too, with ``bins.n_tx > 0`` the divergence maps (``divmaps``,
    n_shots x n_ty x n_tx) and with ``bins.n_aeff > 0`` the a_eff histograms
    (``aeff_hists``); ``grad`` runs the batched adjoint
    (qs_scatter_grad_batch) over the same workspace."""

    # columns of the 8 gradient parameters in the device descriptor arrays
    # viewed as float64 rows (qs_laser: 10 doubles, qs_beam: 11 doubles)
    LASER_COLS = (1, 2, 4, 5, 6)       # a0, w0_um, dx_um, dy_um, delay_fs
    BEAM_COLS = (0, 1, 7)              # gamma_mean, rel_spread, div_rad

    def __init__(self, lasers, beams, offsets, bins: _inputs.Bins, n_total: int, device=None,
                 ranges=None, precision="f32", tile=0, block=0, grid=0, max_phase=None,
                 grad_block=0):
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.n_shots = len(lasers)
        assert len(beams) == self.n_shots
        self.bins = bins
        self.precision = precision
        self.tile, self.block, self.grid, self.grad_block = tile, block, grid, grad_block
        # phase cells are used by the quantum model and by the per-cell focus
        self.max_phase = int(max_phase or max(
            int(l.n_phase) if (l.model == _inputs.MODEL_QFP or l.variant & _inputs.VAR_CELL_FOCUS)
            else 1 for l in lasers))
        self.d_lasers = _struct_array_to_device([make_laser(l) for l in lasers], qs_laser, dev)
        self.d_beams = _struct_array_to_device([make_beam(b) for b in beams], qs_beam, dev)
        if offsets is None:          # parameter sweep: every shot uses all samples
            self.d_offsets = None
        else:
            off = torch.as_tensor(offsets, dtype=torch.int64)
            assert off.numel() == self.n_shots + 1
            self.d_offsets = off.to(dev)
        self.d_ranges = None if ranges is None else torch.as_tensor(
            ranges, dtype=torch.float64).reshape(-1, 2).contiguous().to(dev)
        nb = max(bins.n_bins, 0)
        self.spectra = torch.zeros(self.n_shots, nb, dtype=torch.float64, device=dev)
        self.spec_smooth = torch.zeros(self.n_shots, nb if bins.smooth_sigma_bins > 0 else 0,
                                       dtype=torch.float64, device=dev)
        # per-shot divergence maps (n_shots x n_ty x n_tx, each laid out as
        # qs_scatter's map) and a_eff histograms, when the bins ask for them
        self.divmaps = torch.zeros(self.n_shots, max(bins.n_ty, 0) if bins.n_tx > 0 else 0,
                                   max(bins.n_tx, 0), dtype=torch.float64, device=dev)
        self.aeff_hists = torch.zeros(self.n_shots, max(bins.n_aeff, 0), dtype=torch.float64,
                                      device=dev)
        self.moments = torch.zeros(self.n_shots, len(MOMENT_FIELDS), dtype=torch.float64, device=dev)
        self.grads = torch.zeros(self.n_shots, len(GRAD_PARAMS), dtype=torch.float64, device=dev)
        e = make_exec(precision, 0, block, grid, None, tile)
        b = make_bins(bins)
        nbytes = _lib().qs_batch_workspace_bytes(self.n_shots, int(n_total), C.byref(b),
                                                 self.max_phase, C.byref(e),
                                                 1 if self.d_offsets is None else 0)
        if nbytes == 0:
            raise QsError(QS_ERR_INVALID_ARG, "qs_batch_workspace_bytes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        self.ws_ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        self.ws_bytes = nbytes

    def _common(self):
        return (self.n_shots, self.d_lasers.data_ptr(), self.d_beams.data_ptr(),
                self.d_offsets.data_ptr() if self.d_offsets is not None else None)

    def run(self, xi, w=None, stream=None, check_finite=False):
        s, keep = make_samples(xi, w)
        self._keep = keep
        b = make_bins(self.bins)
        e = make_exec(self.precision, 0, self.block, self.grid, None, self.tile, check_finite)
        st = _lib().qs_scatter_batch(
            *self._common(), C.byref(s), C.byref(b),
            self.d_ranges.data_ptr() if self.d_ranges is not None else None, self.max_phase,
            C.byref(e), self.spectra.data_ptr() if self.spectra.numel() else None,
            self.spec_smooth.data_ptr() if self.spec_smooth.numel() else None,
            self.divmaps.data_ptr() if self.divmaps.numel() else None,
            self.aeff_hists.data_ptr() if self.aeff_hists.numel() else None,
            self.moments.data_ptr(), self.ws_ptr, self.ws_bytes, _stream_ptr(stream))
        _check(st, "qs_scatter_batch")
        return self

    def grad(self, xi, dL_dmoments, dL_dsmooth=None, w=None, moments=None, out=None,
             stream=None) -> torch.Tensor:
        """Per-shot gradients (n_shots x 8, GRAD_PARAMS order) of a loss
        given its upstream gradient with respect to every shot's 13 moments
        (n_shots x 13) and smoothed spectrum (n_shots x n_bins); ``moments``:
        the forward moments (default: those of the last run)."""
        s, keep = make_samples(xi, w)
        dev = self.moments.device
        mom = (self.moments if moments is None else moments).to(dev, torch.float64).contiguous()
        dm = dL_dmoments.to(dev, torch.float64).contiguous()
        dS = None if dL_dsmooth is None else dL_dsmooth.to(dev, torch.float64).contiguous()
        g = self.grads if out is None else out
        b = make_bins(self.bins)
        e = make_exec(self.precision, 0, self.grad_block, self.grid, None, self.tile)
        st = _lib().qs_scatter_grad_batch(
            *self._common(), C.byref(s), C.byref(b),
            self.d_ranges.data_ptr() if self.d_ranges is not None else None, self.max_phase,
            C.byref(e), mom.data_ptr(), dm.data_ptr(),
            dS.data_ptr() if dS is not None else None, g.data_ptr(), self.ws_ptr, self.ws_bytes,
            _stream_ptr(stream))
        _check(st, "qs_scatter_grad_batch")
        self._keep_grad = (keep, mom, dm, dS)
        return g

    def params(self) -> torch.Tensor:
        """The shots' 8 gradient parameters (n_shots x 8, device)."""
        L = self.d_lasers.view(torch.float64).view(self.n_shots, -1)
        Bm = self.d_beams.view(torch.float64).view(self.n_shots, -1)
        return torch.cat([L[:, list(self.LASER_COLS)], Bm[:, list(self.BEAM_COLS)]], dim=1)

    def set_params(self, theta: torch.Tensor):
        """Writes the shots' 8 gradient parameters (n_shots x 8) into the device
        descriptors (the other descriptor fields are kept)."""
        t = theta.to(self.d_lasers.device, torch.float64)
        L = self.d_lasers.view(torch.float64).view(self.n_shots, -1)
        Bm = self.d_beams.view(torch.float64).view(self.n_shots, -1)
        L[:, list(self.LASER_COLS)] = t[:, :5]
        Bm[:, list(self.BEAM_COLS)] = t[:, 5:]

    def moments_dicts(self) -> list[dict]:
        return [dict(zip(MOMENT_FIELDS, row)) for row in self.moments.cpu().tolist()]


# ---- plane-wave reconstruction (Eq. 5) ------------------------------------

def pw_table(laser, beam, bins, n_a: int, a_max: float, xi, w=None, precision="f32",
             stream=None) -> torch.Tensor:
    """Plane-wave spectra per unit weight, n_a x bins.n_bins, at the a-bin
    centres a_k = (k + 1/2) a_max / n_a (those of an a_eff histogram with
    n_aeff = n_a, aeff_max = a_max): one qs_scatter_batch sweep over the
    shared samples xi, each shot the laser at a0 = a_k with no misalignment
    and the beam reduced to its energy distribution at the focus."""
    from dataclasses import replace
    lasers = [replace(laser, a0=(k + 0.5) * a_max / n_a, dx_um=0.0, dy_um=0.0, delay_fs=0.0,
                      variant=0) for k in range(n_a)]
    b0 = replace(beam, sigma_x_um=0.0, sigma_y_um=0.0, sigma_z_um=0.0, div_rad=0.0, dx_um=0.0,
                 dy_um=0.0)
    sb = _inputs.Bins(n_bins=bins.n_bins, lo=bins.lo, hi=bins.hi, log_spaced=bins.log_spaced)
    n = int(xi[0].numel())
    bt = Batch(lasers, [b0] * n_a, None, sb, n, xi[0].device, precision=precision)
    bt.run(xi, w, stream=stream)
    W = bt.moments[:, 0].clamp_min(1e-300)
    return bt.spectra / W[:, None]


def qs_pw_reconstruct(hist, pw, out=None, stream=None) -> torch.Tensor:
    """Eq. 5 on the device: out[s, b] = sum_k hist[s, k] pw[k, b] (hist: shots
    x n_a or one histogram, pw: n_a x bins; float64 device tensors)."""
    h = hist.reshape(-1, hist.shape[-1]).to(torch.float64).contiguous()
    p = pw.to(torch.float64).contiguous()
    ns, na = h.shape
    nb = p.shape[1]
    if p.shape[0] != na:
        raise QsError(QS_ERR_INVALID_ARG, "qs_pw_reconstruct")
    if out is None:
        out = torch.zeros(ns, nb, dtype=torch.float64, device=p.device)
    st = _lib().qs_pw_reconstruct(ns, na, nb, h.data_ptr(), p.data_ptr(), out.data_ptr(),
                                  _stream_ptr(stream))
    _check(st, "qs_pw_reconstruct")
    return out


# ---- unit rates -----------------------------------------------------------

UNIT_RATE_FIELDS = ("fma", "lg2", "ex2", "rcp", "dfma", "sms", "sm_max_mhz", "fma2")


def unit_rates(stream=None) -> dict:
    """Measured operations per SM per clock of the FP32 FMA, MUFU lg2 / ex2 /
    rcp and FP64 FMA pipes (at the maximum SM clock), the SM count and that
    clock, and the packed f32x2 FMA in lane-operations (qs_unit_rates)."""
    nbytes = int(_lib().qs_unit_rates_scratch_bytes())
    scratch = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
    out = (C.c_double * 8)()
    st = _lib().qs_unit_rates(out, scratch.data_ptr(), nbytes, _stream_ptr(stream))
    _check(st, "qs_unit_rates")
    return dict(zip(UNIT_RATE_FIELDS, list(out)))


# ---- analytic fast path (Table 1, Table 2) ---------------------------------

def analytic_aeff(laser, geom, a, stream=None, **par) -> torch.Tensor:
    """Table 1 dN/da_eff on the device grid ``a`` (float64) for an idealised
    beam: "short" (radius, d_perp, d_par, n), "thin" or "wide" (length,
    d_par, n; n is the density for "wide")."""
    x = a.to(torch.float64).contiguous()
    out = torch.empty_like(x)
    g = make_geometry(geom, **par)
    st = _lib().qs_analytic_aeff(C.byref(make_laser(laser)), C.byref(g), x.numel(),
                                 x.data_ptr(), out.data_ptr(), _stream_ptr(stream))
    _check(st, "qs_analytic_aeff")
    return out


def analytic_ll(laser, geom, gamma0, g, stream=None, **par) -> torch.Tensor:
    """Table 2 (Eq. 6 with Eq. 3): the classical dN/dgamma on the device grid ``g``."""
    x = g.to(torch.float64).contiguous()
    out = torch.empty_like(x)
    geo = make_geometry(geom, **par)
    st = _lib().qs_analytic_ll_spectrum(C.byref(make_laser(laser)), C.byref(geo), float(gamma0),
                                        x.numel(), x.data_ptr(), out.data_ptr(),
                                        _stream_ptr(stream))
    _check(st, "qs_analytic_ll_spectrum")
    return out


# ---- host-resident samples ------------------------------------------------

def make_host_samples(xi, w=None) -> tuple[qs_samples, list]:
    """xi: list of up to 8 CPU tensors (pinned for asynchronous copies)."""
    xs = list(xi) + [None] * (8 - len(xi))
    ref = next(t for t in xs if t is not None)
    dt = ref.dtype
    n = ref.numel()
    keep, ptrs = [], []
    for t in xs:
        if t is None:
            ptrs.append(None)
            continue
        if t.is_cuda or t.dtype != dt or t.numel() != n:
            raise ValueError("host sample streams must be CPU tensors of one dtype and length")
        t = t.contiguous()
        keep.append(t)
        ptrs.append(t.data_ptr())
    wp = None
    if w is not None:
        w = w.contiguous()
        keep.append(w)
        wp = w.data_ptr()
    s = qs_samples(n, (C.c_void_p * 8)(*ptrs), wp, QS_F32 if dt == torch.float32 else QS_F64, 0)
    return s, keep


class HostOutputs:
    """Pinned host outputs plus the device workspace of qs_scatter_host."""

    def __init__(self, bins: _inputs.Bins, xi_host, w=None, chunk=0, precision="f32", device=None,
                 block=0, grid=0):
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.bins = bins
        self.chunk = int(chunk)
        pin = dict(dtype=torch.float64, pin_memory=True)
        self.spectrum = torch.zeros(max(bins.n_bins, 0), **pin)
        nmap = bins.n_tx * bins.n_ty if (bins.n_tx > 0 and bins.n_ty > 0) else 0
        self.divmap = torch.zeros(nmap, **pin)
        self.aeff_hist = torch.zeros(max(bins.n_aeff, 0), **pin)
        self.spec_smooth = torch.zeros(max(bins.n_bins, 0) if bins.smooth_sigma_bins > 0 else 0,
                                       **pin)
        self.moments = torch.zeros(len(MOMENT_FIELDS), **pin)
        s, _ = make_host_samples(xi_host, w)
        e = make_exec(precision, 0, block, grid)
        b = make_bins(bins)
        nbytes = _lib().qs_host_workspace_bytes(C.byref(b), C.byref(e), C.byref(s), self.chunk)
        if nbytes == 0:
            raise QsError(QS_ERR_INVALID_ARG, "qs_host_workspace_bytes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        self.ws_ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        self.ws_bytes = nbytes

    def moments_dict(self) -> dict:
        return dict(zip(MOMENT_FIELDS, self.moments.tolist()))


def qs_scatter_host(laser, beam, xi_host, bins, w=None, precision="f32",
                    out: HostOutputs | None = None, chunk=0, block=0, grid=0,
                    weight_frac_bits=0, stream=None) -> HostOutputs:
    """Integrate host-resident samples; copies overlap the kernels.  The
    outputs in ``out`` are valid once the stream reaches the end of the call."""
    s, keep = make_host_samples(xi_host, w)
    if out is None:
        out = HostOutputs(bins, xi_host, w, chunk, precision, None, block, grid)
    L, B, Bn = make_laser(laser), make_beam(beam), make_bins(bins)
    E = make_exec(precision, weight_frac_bits, block, grid)
    hp = lambda t: t.data_ptr() if t.numel() else None  # noqa: E731
    st = _lib().qs_scatter_host(C.byref(L), C.byref(B), C.byref(s), C.byref(Bn), C.byref(E),
                                out.chunk, hp(out.spectrum), hp(out.divmap), hp(out.aeff_hist),
                                hp(out.spec_smooth), out.moments.data_ptr(), out.ws_ptr,
                                out.ws_bytes, _stream_ptr(stream))
    _check(st, "qs_scatter_host")
    out._keep = keep
    return out
