"""Shared set-up for the GPU parity tests: build the CUDA path and the oracle on the same
seeded workload and move vectors between them."""
import numpy as np
import scipy.sparse as sp


def torch_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def gpu_hierarchy(rec, **kw):
    from paper_2608_14310_b300 import api
    sys_ = api.ib_setup(rec)
    h = api.cav_setup(sys_, **kw)
    return sys_, h


def gpu_ee_csr(h, level):
    from paper_2608_14310_b300 import api
    rowptr, cols, vals = api.cav_ee_export(h, level)
    n = rowptr.size - 1
    return sp.csr_matrix((vals, cols, rowptr), shape=(n, n))


def rel(a, b):
    d = np.linalg.norm(a - b)
    s = max(np.linalg.norm(b), 1e-300)
    return d / s
