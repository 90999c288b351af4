"""The stored expected values under tests/golden/ (no GPU): they come from the oracle alone, and the
stored state is a valid truncated augmented MPS (unit-norm, descending bond weights within the
bond cap, the workload's augmented dimensions)."""
import ast
import json
import os

import numpy as np

from workloads import workload

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_golden_writer_calls_only_the_oracle_and_the_workloads():
    tree = ast.parse(open(os.path.join(GOLDEN, "make_random32_step1.py")).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.ImportFrom):
            mods.add(node.module.split(".")[0])
        elif isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
    assert mods <= {"json", "os", "sys", "time", "oracle", "workloads"}, mods


def test_random32_step1_is_a_valid_truncated_state():
    g = json.load(open(os.path.join(GOLDEN, "random32_step1.json")))
    w = workload("random32_stress")
    assert g["workload"] == w.name and g["K"] == w.K and g["chi_max"] == w.chi_max and g["eps"] == w.eps
    N = w.random_state["N"]
    chis, kaps = g["chis"], g["kappas"]
    assert len(chis) == N + 1 and chis[0] == chis[-1] == 1 and max(chis) <= w.chi_max
    assert kaps == [w.random_state["kappa"]] * N
    for b, lam in enumerate(g["lambda"]):
        lam = np.asarray(lam)
        assert len(lam) == chis[b]
        assert abs(np.linalg.norm(lam) - 1.0) < 1e-12
        assert np.all(np.diff(lam) <= 0) and lam[-1] > 0
    assert np.isfinite(g["lognorm"])
