"""The library's host builders (paper_2201_05529_gb300.problem) against the oracle's (CPU).

The GPU parity tests feed the oracle-built inputs through the C ABI; users and bench.py feed the
library's own builders. The two are written independently (gates from an eigendecomposition vs a
matrix exponential; two influence-functional compressors), so they are compared here: gates
element by element, PT-MPOs through the observables of the oracle's PT-TEBD run with either one.
"""
import numpy as np
import pytest

from workloads import workload
from oracle import model, problem as oprob
from paper_2201_05529_gb300 import problem as pp


@pytest.mark.parametrize("name,K", [("xyz3_onebath", 20), ("xyz5_twobaths", 12), ("xyz5_gksl", 12),
                                    ("xyz7_twospin_drive", 12)])
def test_library_builders_agree_with_the_oracle(name, K):
    w = workload(name, K=K)
    chains, mpos = pp.build_problem(w)
    ci = oprob.build_inputs(w)[0]
    assert np.max(np.abs(chains[0]["gates_q"] - np.array(ci.gates_q))) < 1e-14
    assert np.max(np.abs(chains[0]["gates_h"] - np.array(ci.gates_h))) < 1e-14
    assert np.max(np.abs(chains[0]["rho0"] - np.array(ci.rho0))) == 0.0
    if not mpos:
        return
    pts = [None if i < 0 else mpos[i] for i in chains[0]["ptmpo_id"]]
    lib_inputs = oprob.ChainInputs(ci.N, ci.rho0, ci.gates_q, ci.gates_h, pts)
    a = oprob.simulate_chain(ci, w, [model.SZ, model.SX])
    b = oprob.simulate_chain(lib_inputs, w, [model.SZ, model.SX])
    assert np.max(np.abs(a.obs - b.obs)) < 1e-11
