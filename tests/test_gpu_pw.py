"""Plane-wave reconstruction (Eq. 5): the device contraction against the
oracle's, and the reconstructed 3D spectrum against the direct one."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_09348_gb300 import binding as B
from paper_2308_09348_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_09348_gb300 import build
    build.build()


@pytest.mark.parametrize("ns,na,nb", [(1, 61, 512), (37, 13, 100), (1000, 200, 33), (9, 1, 300)])
def test_contraction_matches_oracle(ns, na, nb):
    rg = I.rng(ns + na + nb)
    h = rg.uniform(0, 5, (ns, na))
    pw = rg.uniform(0, 1, (na, nb))
    out = B.qs_pw_reconstruct(torch.from_numpy(h).cuda(), torch.from_numpy(pw).cuda())
    ref = oracle.pw_reconstruct(h, pw)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-300)


def test_reconstruction_converges_to_direct_ll():
    """Monoenergetic misaligned beam, classical model, FP64 path: the
    reconstruction approaches the direct spectrum as the a-grid refines."""
    g0, amax, n = 2000.0, 10.5, 20000
    L = I.Laser(a0=10.0, w0_um=3.0, dx_um=1.0, delay_fs=20.0, model=I.MODEL_LL)
    Bm = I.Beam(gamma_mean=g0, rel_spread=0.0, sigma_x_um=2.0, sigma_y_um=2.0,
                sigma_z_um=5.0, div_rad=0.0)
    xi = [torch.from_numpy(a).cuda() for a in I.sample_streams(n, 5, dtype=np.float32)]
    x1 = [x[:64] for x in xi]
    D = []
    for na in (25, 50, 100):
        bins = I.Bins(n_bins=400, lo=0.0, hi=2100.0, n_aeff=na, aeff_max=amax)
        out = B.qs_scatter(L, Bm, xi, bins, precision="f64")
        pw = B.pw_table(L, Bm, bins, na, amax, x1, precision="f64")
        rec = B.qs_pw_reconstruct(out.aeff_hist, pw)[0].cpu().numpy()
        S = out.spectrum.cpu().numpy()
        assert abs(rec.sum() - S.sum()) < 1e-9 * n
        D.append(np.max(np.abs(np.cumsum(S) - np.cumsum(rec))) / n)
    print("CDF distances:", D)
    assert D[0] > D[1] > D[2] and D[2] < 0.01 and D[0] / D[2] > 3


def test_reconstruction_quantum_beam_with_spread():
    """Quantum model, 10 % energy spread: reconstruction from a 61-point
    plane-wave table (a from 0 to 12 in steps of 0.2, as in Sec. 3.2)
    reproduces the direct spectrum within sampling noise."""
    n, npw = 1 << 18, 1 << 16
    L = I.Laser(a0=12.0, w0_um=3.0, dx_um=1.0, delay_fs=15.0, model=I.MODEL_QFP, n_phase=256)
    Bm = I.Beam(gamma_mean=3000.0, rel_spread=0.1, sigma_x_um=2.0, sigma_y_um=2.0,
                sigma_z_um=5.0, div_rad=0.0)
    xi = [torch.from_numpy(a).cuda() for a in I.sample_streams(n, 6, dtype=np.float32)]
    xpw = [torch.from_numpy(a).cuda() for a in I.sample_streams(npw, 7, dtype=np.float32)]
    bins = I.Bins(n_bins=128, lo=0.0, hi=4500.0, n_aeff=61, aeff_max=12.2)
    out = B.qs_scatter(L, Bm, xi, bins)
    pw = B.pw_table(L, Bm, bins, 61, 12.2, xpw)
    rec = B.qs_pw_reconstruct(out.aeff_hist, pw)[0].cpu().numpy()
    S = out.spectrum.cpu().numpy()
    l1 = np.abs(S - rec).sum() / S.sum()
    c = (np.arange(128) + 0.5) * 4500.0 / 128
    dm = abs((S * c).sum() / S.sum() - (rec * c).sum() / rec.sum()) / ((S * c).sum() / S.sum())
    print("L1/W:", l1, "mean rel:", dm)
    assert l1 < 0.05 and dm < 2e-3
