"""Writes random32_step1.json: the FP64 oracle's state after the first step of the random
augmented-MPS stress workload at full size (N = 32, chi = 96, kappa = 16: the bond SVDs see D up to
1536 x 1536), for the GPU test that runs the same step. It calls only oracle/ and workloads/.

    python tests/golden/make_random32_step1.py        # about ten minutes on eight cores
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import model, problem as oprob   # noqa: E402
from workloads import workload                        # noqa: E402


def main():
    w = workload("random32_stress")
    ci = oprob.build_inputs(w)[0]
    t0 = time.time()
    r = oprob.simulate_chain(ci, w, [model.SZ, model.SX], K=1, keep_lambdas=True)
    m = r.final_mps
    out = {"workload": w.name, "K": w.K, "step": 1, "chi_max": w.chi_max, "eps": w.eps,
           "chis": [int(x) for x in r.chis[-1]], "kappas": [int(x) for x in r.kappas[-1]],
           "lognorm": float(m.lognorm),
           "lambda": [[float(x) for x in l] for l in m.lam],
           "obs_re": [[float(o.real) for o in row] for row in r.obs[1]],
           "obs_im": [[float(o.imag) for o in row] for row in r.obs[1]],
           "trace": [float(r.trace[1].real), float(r.trace[1].imag)],
           "oracle_seconds": time.time() - t0}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "random32_step1.json"), "w") as f:
        json.dump(out, f)
    print(f"written ({out['oracle_seconds']:.0f} s)")


if __name__ == "__main__":
    main()
