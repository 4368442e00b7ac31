"""The allocation-free sweep entry point (cav_sweep_noalloc) against cav_sweep.

cav_sweep_noalloc exists for callers that cannot let a library call allocate device memory
(code whose device memory is already handed to its own pool or budget, or that cannot take
the implicit synchronisation of cudaMalloc/cudaFree).  It runs the same kernels as
cav_sweep with its scratch in a fixed device array, so on the same inputs it must give the
same result as cav_sweep -- checked here through the C ABI on two calls in a row, the
second continuing from the first's output, so the shared array's leftover contents from
one call cannot leak into the next.  This file is named to be collected last.
"""
import numpy as np
import pytest

import ib_workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the per-sweep relative tolerance of the plain FP64 parity tests


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("precision,smoother", [("fp64", "additive"), ("fp32", "additive"),
                                                ("fp64", "coloured")])
def test_noalloc_sweep_matches_cav_sweep(precision, smoother):
    from paper_2608_14310_b300 import api
    rec = W.membrane_ellipse(32, 1e4)
    sysm = api.ib_setup(rec)
    h = api.cav_setup(sysm, nu_pre=1, nu_post=1, alpha=0.85, precision=precision, smoother=smoother)
    rng = np.random.default_rng(3)
    for level in range(api.cav_num_levels(h) - 1):
        N = api.cav_get_level_info(h, level)["N"]
        n = 3 * N * N
        b = rng.uniform(-1, 1, n)
        w_start = rng.uniform(-1, 1, n) * 1e-2
        for call in range(2):
            w_ref = _dev(w_start)
            api.cav_sweep(h, level, _dev(b), w_ref)
            w_new = _dev(w_start)
            api.cav_sweep_noalloc(h, level, _dev(b), w_new)
            ref, new = _host(w_ref), _host(w_new)
            err = np.linalg.norm(new - ref) / np.linalg.norm(ref)
            assert err <= TOL, (level, call, err)
            w_start = ref


def test_noalloc_sweep_on_levels_without_enlarged_patches():
    # no structure: every patch is a standard Vanka patch, so no packed correction is written
    # or read; the result must still equal cav_sweep's on every level, call after call
    from paper_2608_14310_b300 import api
    rec = W.System(name="empty32", N=32, L=1.0, rho=1.0, mu=0.01, dt=0.01, law=0, closed=True,
                   X=np.zeros((0, 2)), ds=0.1, omega=np.zeros(0))
    sysm = api.ib_setup(rec)
    h = api.cav_setup(sysm, nu_pre=1, nu_post=1, alpha=0.85, precision="fp64")
    rng = np.random.default_rng(4)
    for level in range(api.cav_num_levels(h) - 1):
        info = api.cav_get_level_info(h, level)
        assert info["n_enlarged"] == 0
        n = 3 * info["N"] ** 2
        b = rng.uniform(-1, 1, n)
        w_start = rng.uniform(-1, 1, n) * 1e-2
        for call in range(2):
            w_ref = _dev(w_start)
            api.cav_sweep(h, level, _dev(b), w_ref)
            w_new = _dev(w_start)
            api.cav_sweep_noalloc(h, level, _dev(b), w_new)
            ref, new = _host(w_ref), _host(w_new)
            err = np.linalg.norm(new - ref) / np.linalg.norm(ref)
            assert err <= TOL, (level, call, err)
            w_start = ref


def test_noalloc_sweep_rejects_levels_beyond_its_scratch():
    """The additive branch needs 3 N^2 + enlarged unknowns + partial sums and is rejected at
    N = 1024.  The coloured branch needs only ceil(N^2 / 256) partial sums, which reaches the
    limit (1,048,576) only at N = 16384, the largest grid ib_setup accepts, so no grid the
    library takes can exceed it; both branches share the same size check and message."""
    from paper_2608_14310_b300 import api
    # no structure, N = 1024: the finest level alone needs 3 N^2 = 3,145,728 doubles
    rec = W.System(name="empty1024", N=1024, L=1.0, rho=1.0, mu=0.01, dt=0.01, law=0, closed=True,
                   X=np.zeros((0, 2)), ds=0.1, omega=np.zeros(0))
    sysm = api.ib_setup(rec)
    h = api.cav_setup(sysm, kind="vanka", nu_pre=1, nu_post=1, alpha=0.85, precision="fp64")
    b = _dev(np.zeros(3 * 1024 * 1024))
    w = _dev(np.zeros(3 * 1024 * 1024))
    with pytest.raises(api.IBError) as e:
        api.cav_sweep_noalloc(h, 0, b, w)
    assert e.value.status == api.IB_ERR_INVALID
    assert "static array holds" in str(e.value)
    # a coarser level of the same hierarchy fits (N = 512: 786,432 + 32 doubles)
    b2 = _dev(np.ones(3 * 512 * 512))
    w2 = _dev(np.zeros(3 * 512 * 512))
    api.cav_sweep_noalloc(h, 1, b2, w2)
    assert np.isfinite(_host(w2)).all()
