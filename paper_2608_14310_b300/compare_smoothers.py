"""CAV against the box smoother B(4,2) on the paper's target-point and beam set-ups (Sec. 5.2):
FGMRES iterations, set-up time and solves/s on one GPU, both with the class-by-class
multiplicative sweep (one sweep per side, FP64 inverses), the first step's right-hand side
assembled on the device, 1e-10 drop relative to ||r_0||, at most 150 iterations.

Times are wall clock around the blocking calls (the solve returns when its result is on the
host): set-up once, then the median of three solves after one warm-up solve.  One JSON line
per (set-up, N, patch family).

    python -m paper_2608_14310_b300.compare_smoothers
"""
import json
import time

import numpy as np
import torch

import ib_workloads as W
from paper_2608_14310_b300 import api

SETUPS = {"target": W.paper_target_rows, "beam": W.paper_beam}


def main(sizes=(32, 64, 128, 256)):
    torch.cuda.set_device(0)
    for law in ("target", "beam"):
        for N in sizes:
            s = SETUPS[law](N)
            sys_ = api.ib_setup(s)
            b = torch.zeros(3 * N * N, dtype=torch.float64, device="cuda")
            api.ib_step_rhs(sys_, None, None, b)
            for kind in ("cav", "box"):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = api.cav_setup(sys_, kind=kind, coarsest_N=8, nu_pre=1, nu_post=1, precision="fp64",
                                  smoother="coloured", krylov_capacity=150)
                torch.cuda.synchronize()
                setup_ms = 1e3 * (time.perf_counter() - t0)
                ts = []
                for _ in range(4):
                    x = torch.zeros_like(b)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    info = api.fgmres_solve(sys_, h, b, x, rtol=1e-10, maxit=150, rel_to=1, history=False)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)
                solve = float(np.median(ts[1:]))
                lv = api.cav_get_level_info(h, 0)
                print(json.dumps({"law": law, "N": N, "kind": kind, "iters": info["iters"],
                                  "converged": info["converged"], "setup_ms": round(setup_ms, 2),
                                  "solve_ms": round(1e3 * solve, 3), "solves_per_s": round(1.0 / solve, 1),
                                  "ms_per_iter": round(1e3 * solve / max(info["iters"], 1), 4),
                                  "n_colours_l0": lv["n_colours"], "patches_l0": lv["n_patches"],
                                  "sum_n2_l0": lv["enlarged_sum_n2"]}), flush=True)
                h.close()


if __name__ == "__main__":
    main()
