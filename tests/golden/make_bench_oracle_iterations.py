"""Writes bench_oracle_iterations.json: the oracle's own FGMRES iteration count for the
bench workload (elliptic membrane N=256, kappa_s=1e4, weighted additive CAV V-cycle with
2+2 sweeps, alpha=0.85, rtol 1e-10 relative to ||b||).  Calls only oracle/ and the seeded
workload generator; the bench's reference arm scales its per-iteration timing by it.

    OMP_NUM_THREADS=1 python tests/golden/make_bench_oracle_iterations.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import ib_workloads as W  # noqa: E402
from oracle import fgmres, multigrid  # noqa: E402

NU, ALPHA = 2, 0.85

if __name__ == "__main__":
    rec = W.config2(256, 1e4)
    t0 = time.time()
    levels = multigrid.build_hierarchy(rec, 8, "cav")
    K = levels[0].KE
    b = rec.rhs()
    _, info = fgmres.fgmres(lambda v: K @ v, b,
                            lambda r: multigrid.vcycle(levels, r, NU, NU, "additive", ALPHA),
                            rtol=1e-10, maxit=150)
    out = {"workload": rec.name, "nu": NU, "alpha": ALPHA, "iters": info["iters"],
           "converged": bool(info["converged"]), "relres_true": info["relres_true"],
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "bench_oracle_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)
