"""GB300 (sm_103a) PT-TEBD time step: CUDA kernels behind a C ABI (include/pt_tebd.h).

``paper_2201_05529_gb300.build()`` compiles ``libpttebd.so`` in-tree;
``paper_2201_05529_gb300._capi`` is the ctypes binding (it raises if the library is missing);
``paper_2201_05529_gb300.problem`` builds the host inputs (gates, PT-MPOs) of a workload.
"""
__all__ = ["build", "load"]


def build(verbose=False, force=False):
    from .builder import build as _b
    return _b(verbose=verbose, force=force)


def load():
    from . import _capi
    return _capi
