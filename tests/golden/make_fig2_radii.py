"""Write fig2_radii.json: the two-grid spectra of Sec. 5.1, Fig. 2 (membrane, N = 32 with a
16 x 16 coarse grid, kappa_s = 1e4, one multiplicative sweep per side) computed by the oracle
alone, for B(1,0) and B(4,2) at mu = 1 and B(4,2) and CAV at mu = 1e-2, next to the spectral
radii the paper prints.  One patch order per run: "multiplicative" (the paper's lexicographic
order) or "coloured" (the class-by-class order the CUDA path uses); each run merges its
entries into the file.  Dense B^TG K_E of order 3072 per case, about half an hour per order
on one CPU socket.  Run from the repository root:

    python tests/golden/make_fig2_radii.py multiplicative
    python tests/golden/make_fig2_radii.py coloured
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ib_workloads as W  # noqa: E402
from oracle import multigrid, twogrid  # noqa: E402

# Fig. 2 of the paper: (panel, patch family, viscosity, printed spectral radius)
PAPER = [("a", "vanka", 1.0, 0.88), ("c", "box", 1.0, 0.13), ("d", "box", 1e-2, 0.81), ("e", "cav", 1e-2, 0.14)]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fig2_radii.json")


def main(mode):
    assert mode in ("multiplicative", "coloured")
    out = {"workload": "paper membrane (ellipse 0.23 x 0.27, spacing about h/2), N = 32, coarsest 16, "
                       "kappa_s = 1e4, dt = h/2, 1+1 sweeps; B(4,2) with restricted injection", "entries": {}}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    for panel, kind, mu, rho in PAPER:
        s = W.paper_membrane(32, 1e4, mu=mu)
        levels = multigrid.build_hierarchy(s, 16, kind)
        K = levels[0].KE
        BK = twogrid.preconditioned_operator(lambda v: K @ v,
                                             lambda r: multigrid.vcycle(levels, r, 1, 1, mode), K.shape[0])
        row = out["entries"].setdefault(panel, {"kind": kind, "mu": mu, "paper_rho_T": rho})
        row[mode] = twogrid.spectrum_summary(BK, 32)
        print(panel, mode, row[mode], flush=True)
        # re-read before writing: the other order may have finished a panel meanwhile
        cur = out
        if os.path.exists(OUT):
            with open(OUT) as f:
                cur = json.load(f)
            cur["entries"].setdefault(panel, {"kind": kind, "mu": mu, "paper_rho_T": rho})[mode] = row[mode]
        with open(OUT, "w") as f:
            json.dump(cur, f, indent=1)
        out = cur


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "multiplicative")
