"""Failure detection with faults injected on the host: every one ends in an error code, none in a
GPU fault, and the context keeps working afterwards.

  * a Jacobi sweep cap of 1            -> PT_ERR_SVD_NOCONV (the SVD stops, the status word says so)
  * a NaN in one two-site gate          -> PT_ERR_NAN (the guard between theta and the SVD stops the
                                           bond; no NaN reaches a pivot order or a rotation)
  * an allocator that returns NULL      -> PT_ERR_OOM from pt_tebd_init, every allocation released
  * an initial MPS wider than chi_max   -> PT_ERR_CAPACITY from pt_tebd_init
"""
import ctypes as C

import numpy as np
import pytest

from workloads import workload
from oracle import model, problem as oprob
from tests.gpu_helpers import OPS, engine_args_from_oracle, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

PT_ERR_OOM, PT_ERR_CAPACITY, PT_ERR_SVD_NOCONV, PT_ERR_NAN = -2, -3, -4, -6


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


def _still_correct():
    # the context is usable and the path still matches the oracle after the injected failure
    w = workload("xyz3_onebath", K=4)
    cis = oprob.build_inputs(w)
    eng, obs, _ = run_gpu(w, cis, OPS)
    ref = run_oracle(w, cis, OPS)[0]
    assert np.max(np.abs(obs[:, 0, :3, :] - ref.obs)) < 1e-9
    eng.destroy()


def test_sweep_cap_of_one_reports_no_convergence(_lib):
    w = workload("xyz5_twobaths", K=8)
    chains, mpos = engine_args_from_oracle(oprob.build_inputs(w))
    eng = _lib.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K, max_sweeps=1)
    eng.step(6)
    with pytest.raises(_lib.PTError) as ei:
        eng.sync()
    assert ei.value.code == PT_ERR_SVD_NOCONV
    eng.destroy()
    _still_correct()


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_nan_in_a_gate_reports_nan(_lib, precision):
    w = workload("xyz3_onebath", K=4)
    cis = oprob.build_inputs(w)
    chains, mpos = engine_args_from_oracle(cis)
    gq = np.array(chains[0]["gates_q"])
    gq[0, 3, 5] = np.nan                  # the first (odd) bond's dt/4 gate
    chains[0]["gates_q"] = gq
    eng = _lib.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, precision=precision, max_steps=w.K)
    eng.step(2)
    with pytest.raises(_lib.PTError) as ei:
        eng.sync()
    assert ei.value.code == PT_ERR_NAN
    eng.destroy()
    _still_correct()


def test_allocation_failure_reports_oom_and_releases_everything(_lib):
    import torch
    w = workload("xyz3_onebath", K=4)
    chains, mpos = engine_args_from_oracle(oprob.build_inputs(w))
    dev = torch.cuda.current_device()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated(dev)
    live = {}
    budget = [25]                              # the 26th allocation fails

    def _alloc(nbytes, ctx):
        if budget[0] <= 0:
            return None
        budget[0] -= 1
        p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch.cuda.current_stream(dev))
        live[p] = nbytes
        return p

    def _free(ptr, ctx):
        if ptr:
            live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

    fa, ff = _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)
    _lib.lib.pt_tebd_set_allocator(fa, ff, None)
    try:
        with pytest.raises(_lib.PTError) as ei:
            _lib.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K)
        assert ei.value.code == PT_ERR_OOM
        assert budget[0] == 0 and not live            # every allocation made was released
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated(dev) == base
    finally:
        _lib.use_torch_allocator(dev)
    _still_correct()


def test_initial_mps_wider_than_chi_max_is_a_capacity_error(_lib):
    w = workload("random32_stress", K=2)
    w.random_state = dict(N=6, chi=12, kappa=4, K=2)
    w.kappa_max = 4
    chains, mpos = engine_args_from_oracle(oprob.build_inputs(w))
    with pytest.raises(_lib.PTError) as ei:
        _lib.Engine(chains, mpos, chi_max=8, eps=w.eps, max_steps=2)
    assert ei.value.code == PT_ERR_CAPACITY
    assert "chi_max" in str(ei.value)
    _still_correct()
