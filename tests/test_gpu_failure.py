"""Failure detection without a GPU fault: the cooperative kernels' bounded grid barrier.

A CTA that never arrives (withheld on purpose in the diagnostic launch) makes the others' wait run
out after the given limit (1 ms here); they record the timeout and leave, the host gets
PT_ERR_DEVICE_TIMEOUT, and the context keeps working: a PT-TEBD run afterwards still matches the
oracle. No trap, assert, bad address or endless loop is involved.
"""
import time

import numpy as np
import pytest

from workloads import workload
from oracle import problem as oprob
from tests.gpu_helpers import OPS, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

PT_OK = 0
PT_ERR_DEVICE_TIMEOUT = -5
ST_TIMEOUT = 16


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05529_gb300 as pkg
    pkg.build()
    capi = pkg.load()
    capi.use_torch_allocator()
    return capi


def test_barrier_completes_when_every_cta_arrives(_lib):
    rc, st = _lib.selftest_grid_barrier(-1, 1000.0)
    assert rc == PT_OK and st == 0


def test_withheld_cta_times_out_and_the_context_survives(_lib):
    t0 = time.perf_counter()
    rc, st = _lib.selftest_grid_barrier(3, 1.0)
    dt = time.perf_counter() - t0
    assert rc == PT_ERR_DEVICE_TIMEOUT and (st & ST_TIMEOUT)
    assert dt < 5.0
    # the device is still usable: the barrier works again, and a full PT-TEBD run is correct
    assert _lib.selftest_grid_barrier(-1, 1000.0) == (PT_OK, 0)
    w = workload("xyz3_onebath", K=6)
    cis = oprob.build_inputs(w)
    eng, obs, _ = run_gpu(w, cis, OPS)
    ref = run_oracle(w, cis, OPS)[0]
    assert np.max(np.abs(obs[:, 0, :3, :] - ref.obs)) < 1e-9
    eng.destroy()
