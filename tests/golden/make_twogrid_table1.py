"""Write twogrid_table1.json: the two-grid spectra of Sec. 5.1, Table 1 (membrane, N = 16 with
an 8 x 8 coarse grid, mu = 1e-2, one sweep per side) computed by the oracle alone, for the
paper's lexicographic multiplicative CAV sweep and for the class-by-class order the CUDA path
uses, next to the values the paper prints.  Run from the repository root:

    python tests/golden/make_twogrid_table1.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ib_workloads as W  # noqa: E402
from oracle import multigrid, twogrid  # noqa: E402

# Table 1 of the paper: rho(T) and min / max |lambda(B^TG K_E)| per spring stiffness
PAPER = {"1e2": (0.0816, 0.9357, 1.0486), "1e3": (0.1233, 0.9471, 1.1233), "1e4": (0.3518, 0.8470, 1.3518),
         "1e5": (0.4684, 0.8090, 1.4684), "1e6": (0.5916, 0.8326, 1.5916)}


def main():
    out = {"workload": "paper membrane (ellipse 0.23 x 0.27, spacing about h/2), N = 16, coarsest 8, "
                       "mu = 1e-2, dt = h/2, 1+1 sweeps", "entries": {}}
    for key in PAPER:
        s = W.paper_membrane(16, float(key))
        levels = multigrid.build_hierarchy(s, 8)
        K = levels[0].KE
        row = {"paper": dict(zip(("rho_T", "min_abs_lambda", "max_abs_lambda"), PAPER[key]))}
        for mode in ("multiplicative", "coloured"):
            BK = twogrid.preconditioned_operator(lambda v: K @ v,
                                                 lambda r: multigrid.vcycle(levels, r, 1, 1, mode), K.shape[0])
            row[mode] = twogrid.spectrum_summary(BK, 16)
        out["entries"][key] = row
        print(key, row, flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "twogrid_table1.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
