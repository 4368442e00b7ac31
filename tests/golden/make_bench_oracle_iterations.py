"""Writes bench_oracle_iterations.json: the oracle's own FGMRES iteration counts for the
bench workload (elliptic membrane N=256, kappa_s=1e4, rtol 1e-10 relative to ||b||) with the
bench's two V-cycles: the weighted additive CAV sweep on every level (2+2 sweeps, alpha 0.85),
and the class-by-class multiplicative sweep on the finest level (1+1) with the additive one
below it (4+4); for a coarsest grid of 8 x 8 (the top-level keys) and of 32 x 32 (under
"coarsest_32").  With --post-only, only the form that sweeps the finest level once after the
coarse correction and not before it (0+1, additive 4+4 below) is computed, under the key
"coloured_finest_post_only" of each coarsest grid named.  Calls only oracle/ and the seeded
workload generator; the bench's CPU baseline and reference arm scale their per-iteration
timings by these counts.

    OMP_NUM_THREADS=1 python tests/golden/make_bench_oracle_iterations.py [--post-only] [coarsest ...]
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

def counts(rec, coarsest: int) -> dict:
    t0 = time.time()
    levels = multigrid.build_hierarchy(rec, coarsest, "cav")
    K = levels[0].KE
    b = rec.rhs()
    _, info = fgmres.fgmres(lambda v: K @ v, b,
                            lambda r: multigrid.vcycle(levels, r, NU, NU, "additive", ALPHA),
                            rtol=1e-10, maxit=150)
    out = {"workload": rec.name, "coarsest_N": coarsest, "nu": NU, "alpha": ALPHA, "iters": info["iters"],
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
    return out


def post_only_counts(rec, coarsest: int) -> dict:
    """The coloured finest level swept once after the coarse correction only (0+1)."""
    t0 = time.time()
    levels = multigrid.build_hierarchy(rec, coarsest, "cav")
    K = levels[0].KE
    b = rec.rhs()
    L = len(levels) - 1
    modes = ["coloured"] + ["additive"] * (L - 1)
    pre = [0] + [NU_BELOW] * (L - 1)
    post = [1] + [NU_BELOW] * (L - 1)
    _, info = fgmres.fgmres(lambda v: K @ v, b,
                            lambda r: multigrid.vcycle(levels, r, pre, post, modes, ALPHA),
                            rtol=1e-10, maxit=150)
    return {"modes": modes, "nu_pre": pre, "nu_post": post, "alpha": ALPHA, "iters": info["iters"],
            "converged": bool(info["converged"]), "relres_true": info["relres_true"],
            "oracle_seconds": round(time.time() - t0, 1)}


if __name__ == "__main__":
    rec = W.config2(256, 1e4)
    path = os.path.join(HERE, "bench_oracle_iterations.json")
    post_only = "--post-only" in sys.argv[1:]
    which = [int(a) for a in sys.argv[1:] if a != "--post-only"] or [8, 32]
    out = {}
    if os.path.exists(path):
        with open(path) as f:
            out = json.load(f)
    for c in which:
        if post_only:
            res = post_only_counts(rec, c)
            (out if c == 8 else out[f"coarsest_{c}"])["coloured_finest_post_only"] = res
            with open(path, "w") as f:
                json.dump(out, f, indent=1)
            print(c, res, flush=True)
            continue
        res = counts(rec, c)
        if c == 8:
            keep = {k: v for k, v in out.items() if k.startswith("coarsest_")}
            out = dict(res, **keep)
        else:
            out[f"coarsest_{c}"] = res
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(c, res, flush=True)
