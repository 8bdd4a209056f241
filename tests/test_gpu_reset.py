"""Per-device state across a device reset.

The library keeps a few things per device: the cycle-resolved chi tables and
the photon-spectrum table (built on the device at first use), the address of
qs_scatter_noalloc's static scratch array, the copy stream and events of
qs_scatter_host, and kernel attributes.  All of them belong to the CUDA
context, and cudaDeviceReset destroys it.  The library keys them on the
context's id, so the first call after a reset sets them up again.  Run in a
child process (tests/context_reset_child.py) that owns its device memory, so
that the reset destroys nothing this test process uses.
"""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_09348_gb300 import build
    build.build()


def test_stateful_entry_points_agree_before_and_after_a_device_reset():
    r = subprocess.run([sys.executable, os.path.join(HERE, "context_reset_child.py")],
                       capture_output=True, text=True, timeout=600)
    print(r.stdout[-2000:], r.stderr[-2000:])
    if r.returncode == 3:
        pytest.fail("the driver kept the context id across the reset: " + r.stdout.strip())
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert all(res["same"].values()) and all(res["nonzero"].values()), res
