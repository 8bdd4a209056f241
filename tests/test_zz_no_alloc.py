"""qs_scatter_noalloc: the entry point for callers that cannot allocate
device memory (for example a plugin inside a host application that owns
every device allocation).  It keeps its scratch space in a fixed-size static
device array inside the library instead of a caller workspace.

Checked through the C ABI on the GPU: two calls in a row (different
workloads, so stale scratch contents would show) agree with qs_scatter, and a
request larger than the static scratch is refused before any launch.  This
file is collected last on purpose.
"""
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


def _inputs(wl, n, weighted):
    xi, _ = I.workload_inputs(wl, n)
    xt = [torch.from_numpy(a).cuda() for a in xi]
    w = None
    if weighted:
        w = torch.from_numpy(I.rng(21).uniform(0.5, 1.5, n).astype(np.float32)).cuda()
    return xt, w


def _same(a, b, prec):
    # identical per-sample code and launch shape: histograms are integer sums
    # and must match exactly; moments within the path's moment tolerance
    assert torch.equal(a.spectrum, b.spectrum)
    assert torch.equal(a.divmap, b.divmap)
    assert torch.equal(a.aeff_hist, b.aeff_hist)
    ma, mb = a.moments.cpu().numpy(), b.moments.cpu().numpy()
    tol = 1e-12 if prec == "f64" else 1e-5
    np.testing.assert_allclose(ma, mb, rtol=tol, atol=0)


def test_noalloc_matches_workspace_path_on_consecutive_calls():
    wl1 = I.full_qfp(20011)
    x1, _ = _inputs(wl1, 20011, False)
    wl2 = I.full_ll(7003)
    bins2 = I.Bins(n_bins=300, lo=0.0, hi=6000.0, n_tx=64, n_ty=32, theta_max=5e-3,
                   n_aeff=100, aeff_max=30.0)
    x2, w2 = _inputs(wl2, 7003, True)

    ref1 = B.qs_scatter(wl1.laser, wl1.beam, x1, wl1.bins, precision="f32")
    ref2 = B.qs_scatter(wl2.laser, wl2.beam, x2, bins2, w=w2, precision="f64")
    torch.cuda.synchronize()

    got1 = B.qs_scatter_noalloc(wl1.laser, wl1.beam, x1, wl1.bins, precision="f32")
    torch.cuda.synchronize()
    _same(got1, ref1, "f32")
    got2 = B.qs_scatter_noalloc(wl2.laser, wl2.beam, x2, bins2, w=w2, precision="f64")
    torch.cuda.synchronize()
    _same(got2, ref2, "f64")
    # and once more with the first workload: nothing left over from call 2
    got3 = B.qs_scatter_noalloc(wl1.laser, wl1.beam, x1, wl1.bins, precision="f32")
    torch.cuda.synchronize()
    _same(got3, ref1, "f32")


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    wl = I.full_qfp(1000)
    x, _ = _inputs(wl, 1000, False)
    big = I.Bins(n_bins=512, lo=0.0, hi=6720.0, n_tx=1024, n_ty=1024, theta_max=1e-2)
    assert B.workspace_bytes(big, 1000) > 1 << 20
    with pytest.raises(B.QsError) as e:
        B.qs_scatter_noalloc(wl.laser, wl.beam, x, big)
    assert e.value.status == B.QS_ERR_WORKSPACE
