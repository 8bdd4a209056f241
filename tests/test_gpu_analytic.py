"""Analytic fast path (Table 1, Table 2 via Eq. 6) on the device against the
oracle, through the C ABI."""
import math

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


CASES = [("short", dict(radius=2.1, n=1000.0)),
         ("short", dict(radius=2.1, d_perp=2.0, d_par=-4.0, n=1000.0)),
         ("short", dict(radius=0.5, d_perp=6.0, n=1.0)),           # I0 argument > 30
         ("thin", dict(length=60.0, n=500.0)),
         ("thin", dict(length=60.0, d_par=9.0, n=500.0)),
         ("thin", dict(length=20.0, d_par=30.0, n=500.0)),          # both roots on one side
         ("wide", dict(length=60.0, d_par=6.0, n=0.01)),
         ("wide", dict(length=8.0, d_par=40.0, n=0.01))]


@pytest.mark.parametrize("geom,par", CASES)
def test_aeff_density_matches_oracle(geom, par):
    L = I.Laser(a0=12.0, w0_um=2.0, lambda_um=1.0, model=I.MODEL_LL)
    a = np.concatenate([np.linspace(-1.0, 13.0, 2001), [0.0, 12.0, 1e-9]])
    out = B.analytic_aeff(L, geom, torch.from_numpy(a).cuda(), **par).cpu().numpy()
    ref = oracle.analytic_aeff(L, geom, a, **par)
    assert ref.max() > 0
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("geom,par", [CASES[0], CASES[1], CASES[3], CASES[6]])
def test_ll_spectrum_matches_oracle(geom, par):
    L = I.Laser(a0=12.0, w0_um=2.0, lambda_um=0.8, model=I.MODEL_LL)
    g0 = 5000.0
    g = np.linspace(0.0, 5100.0, 3001)
    out = B.analytic_ll(L, geom, g0, torch.from_numpy(g).cuda(), **par).cpu().numpy()
    ref = oracle.analytic_ll(L, geom, g0, g, **par)
    assert ref.max() > 0
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-300)


def test_invalid_geometry():
    L = I.Laser(model=I.MODEL_LL)
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    for geom, par in (("short", dict(radius=0.0)), ("thin", dict(length=-1.0)),
                      ("wide", dict(length=5.0, n=-1.0))):
        with pytest.raises(QsError):
            B.analytic_aeff(L, geom, x, **par)
    with pytest.raises(QsError):
        B.analytic_ll(L, "short", 0.5, x, radius=1.0)
