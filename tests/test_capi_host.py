"""Host-side checks of the C ABI (no GPU work): the library builds for sm_103a, loads, and exports
every function include/pt_tebd.h declares; the binding declares the same set."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "pt_tebd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(pt_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def capi():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2201_05529_gb300 as pkg
    pkg.build()
    return pkg.load()


def test_library_exports_every_declared_symbol(capi):
    names = _header_functions()
    assert "pt_tebd_init" in names and "pt_svd_f64" in names
    missing = [n for n in names if not hasattr(capi.lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(capi):
    assert sorted(capi.EXPORTS) == _header_functions()


def test_init_rejects_bad_arguments_without_a_gpu(capi):
    import ctypes as C
    h = C.c_void_p()
    rc = capi.lib.pt_tebd_init(C.byref(h), None, 0, None, 0, None, None)
    assert rc == -1
    assert b"bad arguments" in capi.lib.pt_tebd_last_error(None)


def test_svd_scratch_size_is_positive(capi):
    assert capi.svd_scratch_bytes(256, 256, 4) >= 256 * 256 * 16 * 4
    assert capi.svd_scratch_bytes(0, 4, 1) == 0
