"""The device-side timeout path, driven without a fault or a hang.

Every wait of the patch-apply and class-step kernels is bounded.  The test hook
ib_test_wait_stall makes every wait for data run out after about 2^20 clock cycles (no
barrier is left waiting forever, and the copies already in flight land before the blocks
exit), so the kernels record DEV_TIMEOUT and finish.  Checked here through the C ABI: the
calls that read the status word (cav_sweep, cav_sweep_noalloc, vcycle_apply, fgmres_solve)
return IB_ERR_TIMEOUT, and once the hook is off the same hierarchy sweeps correctly again
(the word was cleared and the device is still usable).
"""
import numpy as np
import pytest

import ib_workloads as W
from tests.gpu_helpers import host, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setups():
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(32, 1e4)
    sysm = api.ib_setup(rec)
    add = api.cav_setup(sysm, nu_pre=1, nu_post=1, alpha=0.85, precision="fp32")
    col = api.cav_setup(sysm, nu_pre=1, nu_post=1, precision="fp32", smoother="coloured")
    return rec, sysm, add, col


def _sweep_ref(api, h, b, w0):
    w = torch_dev(w0)
    api.cav_sweep(h, 0, torch_dev(b), w)
    return host(w)


@pytest.mark.parametrize("which", ["additive", "coloured"])
def test_sweep_reports_timeout_and_recovers(setups, which):
    from paper_2608_14310_b300 import api
    rec, sysm, add, col = setups
    h = add if which == "additive" else col
    b = rec.rhs()
    w0 = np.full(b.size, 1e-3)
    want = _sweep_ref(api, h, b, w0)
    try:
        api.ib_test_wait_stall(True)
        for call in (api.cav_sweep, api.cav_sweep_noalloc):
            w = torch_dev(w0)
            with pytest.raises(api.IBError) as e:
                call(h, 0, torch_dev(b), w)
            assert e.value.status == api.IB_ERR_TIMEOUT, str(e.value)
            assert "wait ran out" in str(e.value)
    finally:
        api.ib_test_wait_stall(False)
    # the status word was cleared and the device still works: the same sweep again
    got = _sweep_ref(api, h, b, w0)
    assert np.array_equal(got, want)


def test_vcycle_and_fgmres_report_timeout(setups):
    from paper_2608_14310_b300 import api
    rec, sysm, add, col = setups
    b = rec.rhs()
    try:
        api.ib_test_wait_stall(True)
        z = torch_dev(np.zeros(b.size))
        with pytest.raises(api.IBError) as e:
            api.vcycle_apply(add, torch_dev(b), z)
        assert e.value.status == api.IB_ERR_TIMEOUT
        x = torch_dev(np.zeros(b.size))
        with pytest.raises(api.IBError) as e:
            api.fgmres_solve(sysm, add, torch_dev(b), x, rtol=1e-10, maxit=3)
        assert e.value.status == api.IB_ERR_TIMEOUT
    finally:
        api.ib_test_wait_stall(False)
    x = torch_dev(np.zeros(b.size))
    info = api.fgmres_solve(sysm, add, torch_dev(b), x, rtol=1e-10, maxit=150)
    assert info["converged"] == 1
    r = torch_dev(np.zeros(b.size))
    api.ib_residual(sysm, torch_dev(b), x, r)
    assert np.linalg.norm(host(r)) <= 2e-10 * np.linalg.norm(b)
