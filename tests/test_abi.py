"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and rejects invalid arguments on the host before touching a GPU."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2308_09348_gb300 import binding as B
from paper_2308_09348_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2308_09348_gb300 import build
    build.build()
    return B.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(qs_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"qs_scatter", "qs_eval_samples", "qs_workspace_bytes", "qs_version",
            "qs_status_string"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_status_strings(lib):
    assert lib.qs_version() == 10
    for s in range(7):
        assert lib.qs_status_string(s)
    assert lib.qs_status_string(99) == b"unknown status"


def test_struct_sizes_match_header_layout():
    assert C.sizeof(B.qs_laser) == 8 * 8 + 4 * 4
    assert C.sizeof(B.qs_beam) == 10 * 8 + 2 * 4
    assert C.sizeof(B.qs_samples) == 8 + 8 * 8 + 8 + 2 * 4
    assert C.sizeof(B.qs_bins) == 4 * 2 + 8 * 2 + 4 * 2 + 8 + 4 * 2 + 8 + 8
    assert C.sizeof(B.qs_moments) == 13 * 8
    assert C.sizeof(B.qs_exec) == 24 + 2 * 8


def _call(lib, laser=None, beam=None, samples=None, bins=None, exe=None, moments=1,
          ws=256, ws_bytes=1 << 20):
    L = laser or B.make_laser(I.Laser())
    Bm = beam or B.make_beam(I.Beam())
    S = samples or B.qs_samples(0, (C.c_void_p * 8)(), None, 0, 0)
    Bn = bins or B.make_bins(I.Bins())
    return lib.qs_scatter(C.byref(L), C.byref(Bm), C.byref(S), C.byref(Bn),
                          C.byref(exe) if exe is not None else None, 256, 512, 768, 1024,
                          moments, ws, ws_bytes, None)


def test_host_validation_rejects_bad_descriptors(lib):
    bad_lasers = [I.Laser(w0_um=0.0), I.Laser(lambda_um=-1.0), I.Laser(tau_fs=float("nan")),
                  I.Laser(model=I.MODEL_QFP, n_phase=0), I.Laser(model=I.MODEL_QFP, n_phase=5000),
                  I.Laser(envelope=7), I.Laser(a0=-1.0), I.Laser(variant=4), I.Laser(variant=I.VAR_CYCLE_CHI),
                  I.Laser(variant=I.VAR_CELL_FOCUS, n_phase=0)]
    for L in bad_lasers:
        assert _call(lib, laser=B.make_laser(L)) == B.QS_ERR_INVALID_ARG, L
    bad_beams = [I.Beam(gamma_mean=0.0), I.Beam(sigma_x_um=-1.0),
                 I.Beam(flat_energy=1, gamma_lo=10.0, gamma_hi=5.0)]
    for b in bad_beams:
        assert _call(lib, beam=B.make_beam(b)) == B.QS_ERR_INVALID_ARG, b
    bad_bins = [I.Bins(n_bins=4, lo=1.0, hi=1.0), I.Bins(n_bins=4, lo=0.0, hi=1.0, log_spaced=1),
                I.Bins(n_tx=4, n_ty=0, theta_max=1.0), I.Bins(n_tx=4, n_ty=4, theta_max=0.0),
                I.Bins(n_aeff=8, aeff_max=0.0), I.Bins(n_bins=-1),
                I.Bins(n_bins=8, lo=1.0, hi=10.0, log_spaced=1, smooth_sigma_bins=2.0),
                I.Bins(n_bins=0, smooth_sigma_bins=2.0), I.Bins(smooth_sigma_bins=-1.0)]
    for b in bad_bins:
        assert _call(lib, bins=B.make_bins(b)) == B.QS_ERR_INVALID_ARG, b
    # samples: n > 0 with a required stream missing, negative n, bad dtype
    xi = (C.c_void_p * 8)(4096, 8192, 0, 12288)
    assert _call(lib, samples=B.qs_samples(10, xi, None, 0, 0)) == B.QS_ERR_INVALID_ARG
    assert _call(lib, samples=B.qs_samples(-1, (C.c_void_p * 8)(), None, 0, 0)) == B.QS_ERR_INVALID_ARG
    assert _call(lib, samples=B.qs_samples(0, (C.c_void_p * 8)(), None, 5, 0)) == B.QS_ERR_INVALID_ARG
    # misaligned stream
    xi = (C.c_void_p * 8)(4096, 8192, 12288, 16386)
    assert _call(lib, samples=B.qs_samples(10, xi, None, 1, 0)) == B.QS_ERR_INVALID_ARG
    # exec options
    for e in (B.qs_exec(3, 0, 0, 0), B.qs_exec(0, 60, 0, 0), B.qs_exec(0, 0, 48, 0),
              B.qs_exec(0, 0, 1024, 0), B.qs_exec(0, 0, 0, -1),
              B.qs_exec(0, 0, 0, 0, 0, 2), B.qs_exec(0, 0, 0, 0, 0, -1)):
        assert _call(lib, exe=e) == B.QS_ERR_INVALID_ARG
    # missing moments output
    assert _call(lib, moments=None) == B.QS_ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(B, "_LIB", None)
    with pytest.raises(RuntimeError, match="not built"):
        B.lib()
