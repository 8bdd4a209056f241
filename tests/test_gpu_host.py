"""qs_scatter_host: host-resident samples streamed in double-buffered chunks
give the same results as qs_scatter on device-resident samples."""
import numpy as np
import pytest
import torch

from paper_2308_09348_gb300 import binding as B
from paper_2308_09348_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_09348_gb300 import build
    build.build()


@pytest.mark.parametrize("chunk", [1024, 4096, 0])
@pytest.mark.parametrize("prec,model", [("f32", I.MODEL_QFP), ("f64", I.MODEL_LL),
                                         ("f32", I.MODEL_LL)])
def test_host_equals_device(chunk, prec, model):
    n = 10_001          # several chunks and a ragged last one (for small chunks)
    wl = I.full_qfp(n)
    L = I.Laser(**{**wl.laser.__dict__, "model": model, "n_phase": 96})
    bins = I.Bins(**{**wl.bins.__dict__, "smooth_sigma_bins": 2.0})
    xi, _ = I.workload_inputs(wl, n)
    w = I.rng(5).uniform(0.5, 1.5, n).astype(np.float32)
    xh = [torch.from_numpy(a).pin_memory() for a in xi]
    wh = torch.from_numpy(w).pin_memory()
    ref = B.qs_scatter(L, wl.beam, [x.cuda() for x in xh], bins, w=wh.cuda(), precision=prec)
    out = B.qs_scatter_host(L, wl.beam, xh, bins, w=wh, precision=prec, chunk=chunk)
    torch.cuda.synchronize()
    assert torch.equal(out.spectrum, ref.spectrum.cpu())
    assert torch.equal(out.divmap, ref.divmap.cpu())
    assert torch.equal(out.aeff_hist, ref.aeff_hist.cpu())
    assert torch.equal(out.spec_smooth, ref.spec_smooth.cpu())
    # chunked launches partition the samples differently from one launch
    np.testing.assert_allclose(out.moments.numpy(), ref.moments.cpu().numpy(),
                               rtol=1e-13 if prec == "f64" else 1e-8)


def test_host_automatic_chunks_span_the_ramp():
    """chunk = 0: chunks of whole waves (1792 samples per SM) growing x3 up
    to 2^23 samples; n spans the 1-, 3- and 9-wave chunks, full chunks and a
    ragged tail."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    wave = 1792 * sms
    n = 13 * wave + (1 << 23) // wave * wave + 12_345
    wl = I.full_qfp(n)
    L = I.Laser(**{**wl.laser.__dict__, "n_phase": 32})
    xi, _ = I.workload_inputs(wl, n)
    xh = [torch.from_numpy(a).pin_memory() for a in xi]
    ref = B.qs_scatter(L, wl.beam, [x.cuda() for x in xh], wl.bins)
    out = B.qs_scatter_host(L, wl.beam, xh, wl.bins, chunk=0)
    torch.cuda.synchronize()
    assert torch.equal(out.spectrum, ref.spectrum.cpu())
    assert torch.equal(out.divmap, ref.divmap.cpu())
    assert torch.equal(out.aeff_hist, ref.aeff_hist.cpu())
    assert out.moments[0].item() == n
    np.testing.assert_allclose(out.moments.numpy(), ref.moments.cpu().numpy(), rtol=1e-8)


def test_host_pageable_memory_and_repeat():
    n = 5000
    wl = I.full_qfp(n)
    L = I.Laser(**{**wl.laser.__dict__, "n_phase": 64})
    xi, _ = I.workload_inputs(wl, n)
    xh = [torch.from_numpy(a) for a in xi]          # pageable
    ref = B.qs_scatter(L, wl.beam, [x.cuda() for x in xh], wl.bins)
    out = B.qs_scatter_host(L, wl.beam, xh, wl.bins, chunk=2048)
    torch.cuda.synchronize()
    m1 = out.moments.clone()
    assert torch.equal(out.spectrum, ref.spectrum.cpu())
    B.qs_scatter_host(L, wl.beam, xh, wl.bins, out=out)
    torch.cuda.synchronize()
    assert torch.equal(out.moments, m1)


def test_host_rejects_bad_chunk():
    n = 100
    wl = I.full_qfp(n)
    xi, _ = I.workload_inputs(wl, n)
    xh = [torch.from_numpy(a) for a in xi]
    with pytest.raises(B.QsError):
        B.qs_scatter_host(wl.laser, wl.beam, xh, wl.bins, chunk=1000)
