"""Writes bench_oracle_iterations.json: the oracle's own FGMRES iteration counts for the
bench workload (elliptic membrane N=256, kappa_s=1e4, rtol 1e-10 relative to ||b||) with the
bench's two V-cycles: the weighted additive CAV sweep on every level (2+2 sweeps, alpha 0.85),
and the class-by-class multiplicative sweep on the finest level (1+1) with the additive one
below it (4+4).  Calls only oracle/ and the seeded workload generator; the bench's CPU
baseline and reference arm scale their per-iteration timings by these counts.

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
NU_BELOW = 4

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
    L = len(levels) - 1
    modes = ["coloured"] + ["additive"] * (L - 1)
    nus = [1] + [NU_BELOW] * (L - 1)
    t0 = time.time()
    _, info = fgmres.fgmres(lambda v: K @ v, b,
                            lambda r: multigrid.vcycle(levels, r, nus, nus, modes, ALPHA),
                            rtol=1e-10, maxit=150)
    out["coloured_finest"] = {"modes": modes, "nu": nus, "alpha": ALPHA, "iters": info["iters"],
                              "converged": bool(info["converged"]), "relres_true": info["relres_true"],
                              "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "bench_oracle_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)
