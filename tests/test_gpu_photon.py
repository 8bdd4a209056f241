"""Photon spectrum of the beam (qs_photon_spectrum) against the oracle and
against the electrons' energy loss, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_09348_gb300 import binding as B
from paper_2308_09348_gb300 import inputs as I
from paper_2308_09348_gb300 import QsError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_09348_gb300 import build
    build.build()


def _case(n, n_phase=32, variant=0, a0=20.0, seed=31):
    L = I.Laser(a0=a0, w0_um=3.0, model=I.MODEL_QFP, n_phase=n_phase, variant=variant,
                delay_fs=10.0, dx_um=0.5)
    Bm = I.Beam(gamma_mean=3000.0, rel_spread=0.05, sigma_x_um=1.5, sigma_y_um=1.5,
                sigma_z_um=3.0, div_rad=2e-3)
    xi = I.sample_streams(n, seed, dtype=np.float32)
    return L, Bm, xi


def _dev(xi, w=None):
    return [torch.from_numpy(a).cuda() for a in xi], (None if w is None else
                                                        torch.from_numpy(w).cuda())


PB = I.Bins(n_bins=48, lo=1e-3, hi=3500.0, log_spaced=1)


@pytest.mark.parametrize("variant", [0, I.VAR_CELL_FOCUS])
def test_fp64_matches_oracle(variant):
    n = 6
    L, Bm, xi = _case(n, variant=variant)
    w = np.array([1.0, 0.5, 2.0, 0.0, 1.5, 0.25], dtype=np.float32)
    xt, wt = _dev(xi, w)
    S = B.qs_photon_spectrum(L, Bm, xt, PB, w=wt, precision="f64").cpu().numpy()
    ref = oracle.photon_spectrum(L, Bm, PB, [a.astype(np.float64) for a in xi],
                                 w.astype(np.float64))
    assert ref.max() > 0
    l1 = np.abs(S - ref).sum() / np.abs(ref).sum()
    print("FP64 photon spectrum L1 rel:", l1)
    assert l1 < 1e-11
    np.testing.assert_allclose(S, ref, rtol=1e-10, atol=1e-14 * ref.max())


def test_fp32_matches_oracle_and_is_repeatable():
    n = 101
    L, Bm, xi = _case(n, n_phase=32)
    xt, _ = _dev(xi)
    pb = I.Bins(n_bins=64, lo=1e-3, hi=3500.0, log_spaced=1)
    S = B.qs_photon_spectrum(L, Bm, xt, pb).cpu().numpy()
    S2 = B.qs_photon_spectrum(L, Bm, xt, pb).cpu().numpy()
    assert np.array_equal(S, S2)
    ref = oracle.photon_spectrum(L, Bm, pb, [a.astype(np.float64) for a in xi])
    l1 = np.abs(S - ref).sum() / np.abs(ref).sum()
    big = ref > 1e-6 * ref.max()
    rel = np.max(np.abs(S[big] / ref[big] - 1))
    print("FP32 photon spectrum L1 rel:", l1, "max rel (significant bins):", rel)
    # measured 3.0e-7 and 3.8e-7: the Bessel table's interpolation (2.3e-7)
    # and the FP32 table coordinate (~1e-6 in F); a table coordinate off by
    # 1e-3 of a node, or a coarser table, would read ~1e-5
    assert l1 < 2e-6
    assert rel < 3e-6


def test_uniform_bins_edge_sizes_and_launch_shapes():
    L, Bm, xi = _case(777, n_phase=64)
    xt, _ = _dev(xi)
    pb = I.Bins(n_bins=512, lo=0.0, hi=3200.0)
    a = B.qs_photon_spectrum(L, Bm, xt, pb).cpu().numpy()
    b = B.qs_photon_spectrum(L, Bm, xt, pb, block=128, grid=7).cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-9 * a.max())
    one = B.qs_photon_spectrum(L, Bm, xt, I.Bins(n_bins=1, lo=10.0, hi=20.0)).cpu().numpy()
    assert one.shape == (1,) and one[0] > 0
    # empty beam and a single sample
    z = B.qs_photon_spectrum(L, Bm, [x[:0] for x in xt], pb).cpu().numpy()
    assert not z.any()
    s1 = B.qs_photon_spectrum(L, Bm, [x[:1] for x in xt], pb).cpu().numpy()
    assert s1.max() > 0


def test_energy_balance_with_the_electron_loss():
    """The photons carry the energy the electrons lose (to the 2 % of the
    Gaunt fit against the exact power), on 2^16 samples."""
    n = 1 << 16
    L, Bm, xi = _case(n, n_phase=128)
    xt, _ = _dev(xi)
    pb = I.Bins(n_bins=400, lo=1e-6, hi=3600.0, log_spaced=1)
    S = B.qs_photon_spectrum(L, Bm, xt, pb).cpu().numpy()
    edges = pb.lo * (pb.hi / pb.lo) ** (np.arange(pb.n_bins + 1) / pb.n_bins)
    centres = np.sqrt(edges[1:] * edges[:-1])
    e_ph = float(np.sum(S * centres * np.diff(edges)))
    out = B.qs_scatter(L, Bm, xt, I.Bins(n_bins=16, lo=0.0, hi=4000.0), precision="f32")
    m = out.moments_dict()
    e_el = (m["mean_gamma0"] - m["mean"]) * m["W"]
    print("photon energy / electron loss:", e_ph / e_el)
    assert e_el > 10 * n
    assert abs(e_ph / e_el - 1) < 0.03


@pytest.mark.parametrize("prec,n", [("f64", 6), ("f32", 101)])
def test_angular_moments_match_oracle(prec, n):
    """Eq. 7's angle-weighted sums beside the spectrum, against the oracle."""
    L, Bm, xi = _case(n)
    xt, _ = _dev(xi)
    S, T = B.qs_photon_spectrum(L, Bm, xt, PB, precision=prec, theta2=True)
    S, T = S.cpu().numpy(), T.cpu().numpy()
    Sr, Tr = oracle.photon_spectrum_angles(L, Bm, PB, [a.astype(np.float64) for a in xi])
    tol = 1e-10 if prec == "f64" else 2e-6
    for a, r in ((S, Sr), (T[0], Tr[0]), (T[1], Tr[1])):
        l1 = np.abs(a - r).sum() / np.abs(r).sum()
        print(f"[{prec}] photon angular sums L1 rel: {l1:.3e}")
        assert l1 < tol
    # mean square angles are of order (a/gamma)^2 along x, (1/gamma)^2 + div^2 along y
    assert (T[0] * S).sum() > (T[1] * S).sum() > 0


def test_plane_wave_photon_divergence_closed_form():
    """Plane wave with a sin^2 envelope, classical regime: photon-number
    weighted mean square angle (5/16 a0^2 + 1)/gamma^2 along the
    polarisation, 1/gamma^2 across (FP32 path, all photons)."""
    g0, a0 = 1000.0, 2.0
    L = I.Laser(a0=a0, w0_um=3.0, envelope=I.ENV_SIN2, model=I.MODEL_QFP, n_phase=256)
    Bpw = I.Beam(gamma_mean=g0, rel_spread=0.0, sigma_x_um=0.0, sigma_y_um=0.0,
                 sigma_z_um=0.0, div_rad=0.0)
    pb = I.Bins(n_bins=240, lo=1e-9, hi=g0, log_spaced=1)
    xt = [torch.zeros(64, device="cuda") for _ in range(8)]
    S, T = B.qs_photon_spectrum(L, Bpw, xt, pb, theta2=True)
    S, T = S.cpu().numpy(), T.cpu().numpy()
    de = np.diff(pb.lo * (pb.hi / pb.lo) ** (np.arange(241) / 240))
    N = (S * de).sum()
    assert abs((T[0] * de).sum() / N * g0 ** 2 / (5 / 16 * a0 ** 2 + 1) - 1) < 0.02
    assert abs((T[1] * de).sum() / N * g0 ** 2 - 1) < 0.02


def test_rejected_requests():
    L, Bm, xi = _case(10)
    xt, _ = _dev(xi)
    with pytest.raises(QsError):
        B.qs_photon_spectrum(I.Laser(**{**L.__dict__, "model": I.MODEL_LL}), Bm, xt, PB)
    with pytest.raises(QsError) as e:
        B.qs_photon_spectrum(I.Laser(**{**L.__dict__, "variant": I.VAR_CYCLE_CHI}), Bm, xt, PB)
    assert e.value.status == B.QS_ERR_UNSUPPORTED
    with pytest.raises(QsError):          # angular sums: at most 256 bins
        B.qs_photon_spectrum(L, Bm, xt, I.Bins(n_bins=300, lo=0.0, hi=1.0), theta2=True)
    for pb in (I.Bins(n_bins=0, lo=0.0, hi=1.0), I.Bins(n_bins=513, lo=0.0, hi=1.0),
               I.Bins(n_bins=8, lo=0.0, hi=1.0, log_spaced=1), I.Bins(n_bins=8, lo=2.0, hi=1.0)):
        with pytest.raises(QsError):
            B.qs_photon_spectrum(L, Bm, xt, pb)
