"""Child process of test_gpu_reset.py: every entry point that keeps state per
device (the cycle-resolved chi tables, the photon-spectrum table, the static
scratch of qs_scatter_noalloc, the copy stream of qs_scatter_host, kernel
attributes) gives the same results before and after a cudaDeviceReset.

Runs without torch's CUDA state: device memory comes from the CUDA runtime
through ctypes, so that the reset destroys nothing this process still uses.
Prints one JSON line; exit code 0 when every result matched, 3 when the
driver did not give the new context a new id (then nothing that relies on
the context check is run after the reset), 1 on a mismatch.
"""
import ctypes as C
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2308_09348_gb300 import binding as B  # noqa: E402
from paper_2308_09348_gb300 import inputs as I  # noqa: E402

lib = B.lib()
rt = C.CDLL("libcudart.so.13")
drv = C.CDLL("libcuda.so.1")
H2D, D2H = 1, 2


def check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with {rc}")


def context_id():
    ctx = C.c_void_p()
    check(drv.cuCtxGetCurrent(C.byref(ctx)), "cuCtxGetCurrent")
    if not ctx.value:
        return None
    cid = C.c_ulonglong()
    check(drv.cuCtxGetId(ctx, C.byref(cid)), "cuCtxGetId")
    return cid.value


class Dev:
    """Device buffers of this process, freed by the reset."""

    def __init__(self):
        self.ptrs = []

    def alloc(self, nbytes):
        p = C.c_void_p()
        check(rt.cudaMalloc(C.byref(p), C.c_size_t(max(int(nbytes), 256))), "cudaMalloc")
        self.ptrs.append(p.value)
        return p.value

    def upload(self, a):
        a = np.ascontiguousarray(a)
        p = self.alloc(a.nbytes)
        check(rt.cudaMemcpy(C.c_void_p(p), a.ctypes.data_as(C.c_void_p), C.c_size_t(a.nbytes), H2D),
              "cudaMemcpy H2D")
        return p

    @staticmethod
    def download(p, n, dtype=np.float64):
        out = np.zeros(n, dtype=dtype)
        check(rt.cudaMemcpy(out.ctypes.data_as(C.c_void_p), C.c_void_p(p), C.c_size_t(out.nbytes), D2H),
              "cudaMemcpy D2H")
        return out


def run_all(xi, host_xi):
    """One call of each stateful entry point; returns their outputs."""
    d = Dev()
    n = len(xi[0])
    ptrs = [d.upload(a) for a in xi]
    S = B.qs_samples(n, (C.c_void_p * 8)(*ptrs), None, B.QS_F32, 0)
    res = {}
    wl = I.full_qfp(n)
    E = B.make_exec("f32")
    # cycle-resolved chi (tables built per context)
    Lc = B.make_laser(I.Laser(**{**wl.laser.__dict__, "n_phase": 64, "variant": I.VAR_CYCLE_CHI}))
    bins = I.Bins(n_bins=128, lo=0.0, hi=6720.0)
    Bn, Bm = B.make_bins(bins), B.make_beam(wl.beam)
    nb = lib.qs_workspace_bytes(C.byref(Bn), C.byref(E), n)
    ws, spec, mom = d.alloc(nb), d.alloc(128 * 8), d.alloc(13 * 8)
    check(lib.qs_scatter(C.byref(Lc), C.byref(Bm), C.byref(S), C.byref(Bn), C.byref(E), spec, None,
                         None, None, mom, ws, nb, None), "qs_scatter (cycle chi)")
    check(rt.cudaDeviceSynchronize(), "sync")
    res["cycle_spec"] = Dev.download(spec, 128).tolist()
    res["cycle_mom"] = Dev.download(mom, 13).tolist()
    # static scratch of qs_scatter_noalloc
    L0 = B.make_laser(I.Laser(**{**wl.laser.__dict__, "n_phase": 64}))
    spec2, mom2 = d.alloc(128 * 8), d.alloc(13 * 8)
    check(lib.qs_scatter_noalloc(C.byref(L0), C.byref(Bm), C.byref(S), C.byref(Bn), C.byref(E),
                                 spec2, None, None, None, mom2, None), "qs_scatter_noalloc")
    check(rt.cudaDeviceSynchronize(), "sync")
    res["noalloc_spec"] = Dev.download(spec2, 128).tolist()
    res["noalloc_mom"] = Dev.download(mom2, 13).tolist()
    # photon table
    pb = B.make_bins(I.Bins(n_bins=32, lo=1e-2, hi=6000.0, log_spaced=1))
    pnb = lib.qs_photon_workspace_bytes(C.byref(pb), C.byref(E), n)
    pws, pout = d.alloc(pnb), d.alloc(32 * 8)
    check(lib.qs_photon_spectrum(C.byref(L0), C.byref(Bm), C.byref(S), C.byref(pb), C.byref(E),
                                 pout, None, pws, pnb, None), "qs_photon_spectrum")
    check(rt.cudaDeviceSynchronize(), "sync")
    res["photon"] = Dev.download(pout, 32).tolist()
    # host-resident samples (copy stream and events per context)
    hp = [a.ctypes.data for a in host_xi]
    HS = B.qs_samples(n, (C.c_void_p * 8)(*hp), None, B.QS_F32, 0)
    hnb = lib.qs_host_workspace_bytes(C.byref(Bn), C.byref(E), C.byref(HS), 1024)
    hws = d.alloc(hnb + 256)
    hws = (hws + 255) // 256 * 256
    hspec = np.zeros(128)
    hmom = np.zeros(13)
    check(lib.qs_scatter_host(C.byref(L0), C.byref(Bm), C.byref(HS), C.byref(Bn), C.byref(E), 1024,
                              hspec.ctypes.data, None, None, None, hmom.ctypes.data, hws, hnb, None),
          "qs_scatter_host")
    check(rt.cudaDeviceSynchronize(), "sync")
    res["host_spec"] = hspec.tolist()
    res["host_mom"] = hmom.tolist()
    for p in d.ptrs:
        rt.cudaFree(C.c_void_p(p))
    return res


def main():
    n = 3001
    xi = I.sample_streams(n, 0x5EED, dtype=np.float32)
    host_xi = [np.ascontiguousarray(a) for a in xi]
    check(rt.cudaSetDevice(0), "cudaSetDevice")
    before = run_all(xi, host_xi)
    id0 = context_id()
    check(rt.cudaDeviceReset(), "cudaDeviceReset")
    check(rt.cudaSetDevice(0), "cudaSetDevice")
    id1 = context_id()
    if id0 is None or id1 is None or id0 == id1:
        print(json.dumps({"context_ids": [id0, id1], "skipped": "context id unchanged"}))
        return 3
    after = run_all(xi, host_xi)
    same = {k: before[k] == after[k] for k in before}
    nonzero = {k: any(v != 0 for v in before[k]) for k in before}
    print(json.dumps({"context_ids": [id0, id1], "same": same, "nonzero": nonzero}))
    return 0 if all(same.values()) and all(nonzero.values()) else 1


if __name__ == "__main__":
    sys.exit(main())
