"""The paper's own experiments (Sec. 5.1, 5.2; Table 2) through the CUDA path with the
coloured multiplicative CAV smoother, one sweep per side: the first backward-Euler step's
system of each set-up is solved by FGMRES to a 1e-10 drop relative to ||r_0|| (zero guess).

  * the GPU assembles its own right-hand side (ib_step_rhs); it equals the oracle's to 1e-9
    (the beam's fourth difference of X cancels about eight digits at N = 64, so summation
    order shows at that level);
  * the GPU's iteration count equals the oracle's (same smoother and class order) within one;
  * both stay within three of the count the paper prints for its lexicographic sweep (marker
    placement and the patch order differ from the paper's, which it does not fully state);
  * at N = 128 (no oracle run: too slow for the suite) the GPU solve converges; its count is
    printed beside the paper's (beam 18 against 11 is a recorded deviation, not a pin).
"""
import numpy as np
import pytest

import ib_workloads as W
from oracle import fgmres as ofg, ib as oib, multigrid as omg
from tests.gpu_helpers import gpu_hierarchy, host, rel, torch_dev

pytestmark = pytest.mark.gpu

SETUPS = {"membrane": W.paper_membrane, "beam": W.paper_beam, "target": W.paper_target_rows}
# (law, N, the paper's printed FGMRES count with CAV)
WITH_ORACLE = [("membrane", 16, 9), ("membrane", 32, 10), ("membrane", 64, 11),
               ("beam", 32, 9), ("beam", 64, 10), ("target", 32, 10), ("target", 64, 13)]
GPU_ONLY = [("beam", 128, 11), ("target", 128, 15)]


def _gpu_solve(s):
    from paper_2608_14310_b300 import api
    sys_, h = gpu_hierarchy(s, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, precision="fp64",
                            smoother="coloured")
    b = torch_dev(np.zeros(3 * s.N * s.N))
    api.ib_step_rhs(sys_, None, None, b)
    x = torch_dev(np.zeros(3 * s.N * s.N))
    info = api.fgmres_solve(sys_, h, b, x, rtol=1e-10, maxit=150, rel_to=1)
    return host(b), info


@pytest.mark.parametrize("law,N,paper", WITH_ORACLE)
def test_paper_counts_against_oracle(law, N, paper):
    s = SETUPS[law](N)
    bo = oib.first_step_rhs(s)
    levels = omg.build_hierarchy(s, 8)
    K = levels[0].KE
    _, io = ofg.fgmres(lambda v: K @ v, bo, lambda r: omg.vcycle(levels, r, 1, 1, "coloured"),
                       rtol=1e-10, maxit=150, ref="r0")
    bg, info = _gpu_solve(s)
    assert rel(bg, bo) <= 1e-9
    assert info["converged"] == 1 and io["converged"]
    assert abs(info["iters"] - io["iters"]) <= 1, (info["iters"], io["iters"])
    assert abs(info["iters"] - paper) <= 3, (info["iters"], paper)
    print(f"{law} N={N}: gpu {info['iters']} oracle {io['iters']} paper {paper}")


@pytest.mark.parametrize("law,N,paper", GPU_ONLY)
def test_paper_counts_large(law, N, paper):
    s = SETUPS[law](N)
    _, info = _gpu_solve(s)
    assert info["converged"] == 1 and info["relres_true"] <= 2e-10, info
    print(f"{law} N={N}: gpu {info['iters']} paper {paper}")
