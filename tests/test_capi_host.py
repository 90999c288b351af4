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


def test_resume_problem_cuts_the_pt_mpos_and_carries_the_log_norm(capi):
    import numpy as np
    rng = np.random.default_rng(3)
    chis, kaps = [1, 2, 3, 1], [2, 1, 3]
    gam = [rng.normal(size=(chis[n], 4, kaps[n], chis[n + 1])) + 0j for n in range(3)]
    lam = [np.ones(c) for c in chis]
    P = [rng.normal(size=(1 if k == 0 else 2, 4, 4, 2)) + 0j for k in range(6)]
    Q = [rng.normal(size=(1 if k == 0 else 3, 4, 4, 3)) + 0j for k in range(6)]
    chains = [dict(N=3, rho0=np.zeros((3, 4)), gates_q=np.zeros((2, 16, 16)), gates_h=np.zeros((2, 16, 16)),
                   ptmpo_id=[0, -1, 1])]
    ck = [{"step": 4, "chi": np.array(chis), "kappa": np.array(kaps), "gamma": gam, "lambda": lam, "lognorm": np.array([-0.75, 0.25, 0.0, 0.5])}]
    rc, rm = capi.resume_problem(chains, [P, Q], ck)
    assert [len(x) for x in rm] == [2, 2] and rm[0][0] is P[4] and rm[1][1] is Q[5]
    d = rc[0]
    assert d["rho0"] is None and list(d["chi0"]) == chis and list(d["kappa0"]) == kaps
    assert np.array_equal(d["gamma0"][0], gam[0]) and d["gamma0"][1] is not gam[1] and list(d["lognorm0"]) == [-0.75, 0.25, 0.0, 0.5]
    assert np.array_equal(d["gamma0"][2], gam[2]) and d["ptmpo_id"] == [0, -1, 1]
    assert chains[0]["rho0"] is not None                   # the caller's dicts are not modified
    with pytest.raises(ValueError):
        capi.resume_problem(chains + chains, [P, Q], ck + [dict(ck[0], step=5)])
