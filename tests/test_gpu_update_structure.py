"""ib_update_structure: a system handle moved to a new configuration (the next Newton iterate
or time step, Sec. 5.3) behaves as a system set up at that configuration, and hierarchies built
before the move keep preconditioning with the configuration they were built from.

  * after the update, y = K_E x equals the oracle's K_E at the new markers (1e-13 of max|y|);
  * a hierarchy built before the update still brings FGMRES to 1e-10 on the new system (a
    lagged preconditioner; true residual from the oracle's K_E);
  * a hierarchy rebuilt after the update gives the same iterations and bits as one built on
    a system set up from scratch at the new configuration.
"""
from dataclasses import replace

import numpy as np
import pytest

import ib_workloads as W
from oracle import multigrid as omg
from tests.gpu_helpers import host, torch_dev

pytestmark = pytest.mark.gpu


def test_update_structure():
    from paper_2608_14310_b300 import api
    rec1 = W.membrane_ellipse(32, 1e4)
    # a nearby configuration, as between Newton iterates or time steps (h = 1/32)
    rec2 = replace(rec1, X=rec1.X + np.array([0.002, -0.001]))
    sysm = api.ib_setup(rec1)
    h_old = api.cav_setup(sysm, nu_pre=1, nu_post=1, precision="fp64", smoother="coloured")
    api.ib_update_structure(sysm, rec2)
    K2 = omg.build_hierarchy(rec2, 8, "cav", factor=False)[0].KE
    x = np.random.default_rng(5).standard_normal(K2.shape[0])
    y = torch_dev(np.zeros(x.size))
    api.ib_apply(sysm, torch_dev(x), y)
    want = K2 @ x
    assert np.abs(host(y) - want).max() <= 1e-13 * np.abs(want).max()
    b = rec2.rhs()
    xl = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(sysm, h_old, torch_dev(b), xl, rtol=1e-10, maxit=150)
    res = np.linalg.norm(b - K2 @ host(xl)) / np.linalg.norm(b)
    assert info["converged"] == 1 and res <= 2e-10, (info, res)
    h_new = api.cav_setup(sysm, nu_pre=1, nu_post=1, precision="fp64", smoother="coloured")
    fresh = api.ib_setup(rec2)
    h_fresh = api.cav_setup(fresh, nu_pre=1, nu_post=1, precision="fp64", smoother="coloured")
    outs = []
    for s, h in ((sysm, h_new), (fresh, h_fresh)):
        xs = torch_dev(np.zeros(b.size))
        inf = api.fgmres_solve(s, h, torch_dev(b), xs, rtol=1e-10, maxit=150)
        outs.append((inf["iters"], host(xs)))
    assert outs[0][0] == outs[1][0], (outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    print(f"lagged hierarchy: {info['iters']} its; rebuilt: {outs[0][0]} its")
