"""Thin ctypes binding of include/ib_cav.h: argument marshalling only.

Device vectors are torch CUDA tensors (float64, contiguous) passed by data pointer on the
current torch stream; descriptors are built from plain numbers and host numpy arrays.
Every non-OK status raises IBError carrying the library's message.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcavib.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run `python -m "
                      "paper_2608_14310_b300.build`); there is no fallback implementation")
_lib = C.CDLL(LIB_PATH)

IB_OK, IB_ERR_INVALID, IB_ERR_OOM, IB_ERR_CUDA, IB_ERR_SINGULAR, IB_ERR_NOCONV, IB_ERR_TIMEOUT, \
    IB_ERR_INTERNAL = range(8)
FORCE = {"target": 0, "membrane": 1, "beam": 2}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}
KIND = {"cav": 0, "vanka": 1, "box": 2}
SMOOTHER = {"additive": 0, "coloured": 1}


class IBError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.ib_last_error().decode()
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


BC = {"periodic": 0, "channel": 1}


class ib_grid_desc(C.Structure):
    _fields_ = [("N", C.c_int32), ("L", C.c_double), ("rho", C.c_double), ("mu", C.c_double),
                ("dt", C.c_double), ("bc", C.c_int32)]


class ib_structure_desc(C.Structure):
    _fields_ = [("M", C.c_int32), ("closed", C.c_int32), ("law", C.c_int32),
                ("X", C.POINTER(C.c_double)), ("omega", C.POINTER(C.c_double)), ("ds", C.c_double),
                ("k_target", C.c_double), ("k_stretch", C.c_double), ("k_bend", C.c_double),
                ("X_target", C.POINTER(C.c_double)), ("X_lin", C.POINTER(C.c_double)), ("k_pos", C.c_double),
                ("k_tan", C.c_double), ("clamp_x", C.c_double), ("clamp_y", C.c_double)]


class cav_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("coarsest_N", C.c_int32), ("nu_pre", C.c_int32),
                ("nu_post", C.c_int32), ("alpha", C.c_double), ("precision", C.c_int32),
                ("autotune", C.c_int32), ("krylov_capacity", C.c_int32), ("smoother", C.c_int32),
                ("coloured_levels", C.c_int32), ("nu_additive", C.c_int32), ("box_b", C.c_int32),
                ("box_o", C.c_int32)]


class cav_level_info(C.Structure):
    _fields_ = [("N", C.c_int32), ("n_patches", C.c_int32), ("n_enlarged", C.c_int32),
                ("max_n", C.c_int32), ("sum_n", C.c_int64), ("sum_n2", C.c_int64),
                ("enlarged_sum_n", C.c_int64), ("enlarged_sum_n2", C.c_int64),
                ("inverse_bytes", C.c_int64), ("ee_nnz", C.c_int64), ("ee_rows", C.c_int32),
                ("ee_window", C.c_int32), ("is_coarsest", C.c_int32), ("apply_variant", C.c_int32),
                ("apply_us", C.c_float * 5), ("n_colours", C.c_int32), ("sweep_form", C.c_int32),
                ("sweep_us", C.c_float * 2)]


class fgmres_desc(C.Structure):
    _fields_ = [("rtol", C.c_double), ("maxit", C.c_int32), ("rel_to", C.c_int32),
                ("host_io", C.c_int32), ("loop", C.c_int32)]


LOOP = {"host": 0, "device": 1}


class fgmres_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("relres_est", C.c_double),
                ("relres_true", C.c_double)]


class ibnet_desc(C.Structure):
    _fields_ = [("in_ch", C.c_int32), ("hidden", C.c_int32), ("n_hidden", C.c_int32), ("out_ch", C.c_int32),
                ("seed", C.c_uint64)]


_vp = C.c_void_p
_P = C.POINTER
_sig = {
    "ib_last_error": (C.c_char_p, []),
    "ib_abi_version": (C.c_int, []),
    "ib_launch_count": (C.c_int64, []),
    "cav_profile": (C.c_int, [_vp, C.c_int32]),
    "cav_profile_read": (C.c_int, [_vp, _P(C.c_int32), _P(C.c_double)]),
    "ib_setup": (C.c_int, [_P(ib_grid_desc), _P(ib_structure_desc), _vp, _P(_vp)]),
    "ib_update_structure": (C.c_int, [_vp, _P(ib_structure_desc), _vp]),
    "ib_apply": (C.c_int, [_vp, _vp, _vp, _vp]),
    "ib_residual": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ib_destroy": (None, [_vp]),
    "ib_force": (C.c_int, [_vp, _vp, _vp]),
    "ib_spread": (C.c_int, [_vp, _vp, _vp, _vp]),
    "ib_interp": (C.c_int, [_vp, _vp, _vp, _vp]),
    "ib_step_rhs": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ib_advect": (C.c_int, [_vp, _vp, _vp, _vp]),
    "ib_channel_rhs": (C.c_int, [_vp, _vp, C.c_double, C.c_double, _vp, _vp]),
    "ib_newton_rhs": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ib_residual_norm": (C.c_int, [_vp, _vp, _vp, _vp, _P(C.c_double), _vp]),
    "cav_setup": (C.c_int, [_vp, _P(cav_desc), _vp, _P(_vp)]),
    "cav_num_levels": (C.c_int, [_vp, _P(C.c_int32)]),
    "cav_refactor": (C.c_int, [_vp, _vp, _vp]),
    "cav_get_level_info": (C.c_int, [_vp, C.c_int32, _P(cav_level_info)]),
    "cav_patch_export": (C.c_int, [_vp, C.c_int32, _vp, _vp, _P(C.c_int32), _P(C.c_int64)]),
    "cav_ee_export": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _P(C.c_int64)]),
    "cav_colour_export": (C.c_int, [_vp, C.c_int32, _vp, _P(C.c_int32)]),
    "cav_sweep": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    "cav_sweep_noalloc": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    "cav_residual": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp]),
    "cav_restrict": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    "cav_prolong_add": (C.c_int, [_vp, C.c_int32, _vp, _vp, _vp]),
    "cav_coarse_solve": (C.c_int, [_vp, _vp, _vp, _vp]),
    "vcycle_apply": (C.c_int, [_vp, _vp, _vp, _vp]),
    "cav_destroy": (None, [_vp]),
    "ib_test_wait_stall": (C.c_int, [C.c_int32]),
    "ibnet_create": (C.c_int, [_P(ibnet_desc), _P(_vp)]),
    "ibnet_destroy": (None, [_vp]),
    "ibnet_num_params": (C.c_int64, [_vp]),
    "ibnet_get_params": (C.c_int, [_vp, _vp]),
    "ibnet_set_params": (C.c_int, [_vp, _vp]),
    "ibnet_forward": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, _vp]),
    "ibnet_inner": (C.c_int, [_vp, C.c_int64, _vp, _vp, _P(C.c_double), _vp]),
    "ibnet_gradients": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, _P(C.c_float), _vp, _vp]),
    "ibnet_train_step": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, C.c_float, _P(C.c_float), _vp]),
    "ibnet_pack_input": (C.c_int, [C.c_int32, _P(_vp), _P(_vp), _P(C.c_float), _vp, _vp]),
    "ibnet_pack_history": (C.c_int, [C.c_int32, C.c_int32, _P(_vp), _P(_vp), _P(C.c_float), _vp, _vp]),
    "ibnet_pack_target": (C.c_int, [C.c_int32, _vp, _vp, _vp, _vp, _P(C.c_float), _vp, _vp]),
    "ibnet_apply_delta": (C.c_int, [C.c_int32, _vp, _vp, _vp, _vp, _P(C.c_float), _vp, _vp]),
    "fgmres_solve": (C.c_int, [_vp, _vp, _vp, _vp, _P(fgmres_desc), _P(fgmres_info), _vp, _vp]),
    "fgmres_solve_batched": (C.c_int, [C.c_int32, _P(_vp), _P(_vp), _P(_vp), _P(_vp), _P(fgmres_desc),
                                       _P(fgmres_info), _vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


def _check(st: int, where: str):
    if st != IB_OK:
        raise IBError(st, where)


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def _dev(t):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("device vectors must be contiguous float64 CUDA tensors")
    return _vp(t.data_ptr())


class System:
    """Owns an ib_system handle."""

    def __init__(self, handle, N, rec=None):
        self._h = handle
        self.N = N
        self.rec = rec

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.ib_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """Owns a cav_hierarchy handle (keeps its system alive)."""

    def __init__(self, handle, system: System, desc: dict):
        self._h = handle
        self.system = system
        self.desc = desc

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.cav_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _structure(rec):
    """Descriptor of rec's structure; the fiber law's extra parameters come from rec.meta
    (k_pos, k_tan, X_c and, optionally, the linearisation point X_lin)."""
    X = np.ascontiguousarray(np.asarray(rec.X, dtype=np.float64).reshape(-1))
    om = np.ascontiguousarray(np.asarray(rec.omega, dtype=np.float64))
    Xt = getattr(rec, "X_target", None)
    Xt = None if Xt is None else np.ascontiguousarray(np.asarray(Xt, dtype=np.float64).reshape(-1))
    meta = getattr(rec, "meta", None) or {}
    Xl = meta.get("X_lin")
    Xl = None if Xl is None else np.ascontiguousarray(np.asarray(Xl, dtype=np.float64).reshape(-1))
    Xc = meta.get("X_c", (0.0, 0.0))
    dp = lambda a: a.ctypes.data_as(_P(C.c_double)) if a is not None else None  # noqa: E731
    sd = ib_structure_desc(int(X.size // 2), 1 if rec.closed else 0, int(rec.law), dp(X), dp(om),
                           float(rec.ds), float(rec.k_target), float(rec.k_stretch), float(rec.k_bend),
                           dp(Xt), dp(Xl), float(meta.get("k_pos", 0.0)), float(meta.get("k_tan", 0.0)),
                           float(Xc[0]), float(Xc[1]))
    return sd, (X, om, Xt, Xl)  # keep the arrays alive while the descriptor is used


def ib_update_structure(sys: System, rec, stream=None):
    """Rebuild S, J, E and E_E of `sys` at rec's markers (same grid)."""
    sd, _keep = _structure(rec)
    _check(_lib.ib_update_structure(sys.handle, C.byref(sd), _stream(stream)), "ib_update_structure")
    sys.rec = rec


def ib_setup(rec, stream=None) -> System:
    """rec: an ib_workloads.System (or any object with the same fields)."""
    g = ib_grid_desc(int(rec.N), float(rec.L), float(rec.rho), float(rec.mu), float(rec.dt),
                     BC[getattr(rec, "bc", "periodic")])
    sd, _keep = _structure(rec)
    out = _vp()
    _check(_lib.ib_setup(C.byref(g), C.byref(sd), _stream(stream), C.byref(out)), "ib_setup")
    return System(out, int(rec.N), rec)


def ib_apply(sys: System, x, y, stream=None):
    _check(_lib.ib_apply(sys.handle, _dev(x), _dev(y), _stream(stream)), "ib_apply")


def ib_residual(sys: System, b, x, r, stream=None):
    _check(_lib.ib_residual(sys.handle, _dev(b), _dev(x), _dev(r), _stream(stream)), "ib_residual")


def ib_force(sys: System, F, stream=None):
    _check(_lib.ib_force(sys.handle, _dev(F), _stream(stream)), "ib_force")


def ib_spread(sys: System, F, f, stream=None):
    _check(_lib.ib_spread(sys.handle, _dev(F), _dev(f), _stream(stream)), "ib_spread")


def ib_interp(sys: System, u, U, stream=None):
    _check(_lib.ib_interp(sys.handle, _dev(u), _dev(U), _stream(stream)), "ib_interp")


def ib_step_rhs(sys: System, u_prev, f_body, b, stream=None):
    _check(_lib.ib_step_rhs(sys.handle, _dev(u_prev), _dev(f_body), _dev(b), _stream(stream)), "ib_step_rhs")


def ib_advect(sys: System, u, stream=None) -> np.ndarray:
    M = 0 if sys.rec is None else int(np.asarray(sys.rec.X).shape[0])
    out = np.zeros(2 * M)
    _check(_lib.ib_advect(sys.handle, _dev(u), _vp(out.ctypes.data), _stream(stream)), "ib_advect")
    return out.reshape(M, 2)


def ib_channel_rhs(sys: System, w_n, U_next: float, U_prev: float, b, stream=None):
    _check(_lib.ib_channel_rhs(sys.handle, _dev(w_n), float(U_next), float(U_prev), _dev(b), _stream(stream)),
           "ib_channel_rhs")


def ib_newton_rhs(sys: System, b_base, w, rhs, stream=None):
    _check(_lib.ib_newton_rhs(sys.handle, _dev(b_base), _dev(w), _dev(rhs), _stream(stream)), "ib_newton_rhs")


def ib_residual_norm(sys: System, b, x, r, stream=None) -> float:
    out = C.c_double()
    _check(_lib.ib_residual_norm(sys.handle, _dev(b), _dev(x), _dev(r), C.byref(out), _stream(stream)),
           "ib_residual_norm")
    return out.value


def cav_setup(sys: System, kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, alpha=1.0,
              precision="fp64", autotune=False, krylov_capacity=0, smoother="additive",
              coloured_levels=0, nu_additive=0, box=(4, 2), stream=None) -> Hierarchy:
    """smoother: "additive" on every level, or "coloured" on the `coloured_levels` finest levels
    (0: all) with the additive sweep (nu_additive sweeps per side, 0: nu_pre/nu_post) below.
    kind "box": B(b, o) patches, box = (b, o), with restricted injection (coloured smoother on
    every level)."""
    d = cav_desc(KIND[kind], int(coarsest_N), int(nu_pre), int(nu_post), float(alpha), PRECISION[precision],
                 1 if autotune else 0, int(krylov_capacity), SMOOTHER[smoother], int(coloured_levels),
                 int(nu_additive), int(box[0]), int(box[1]))
    out = _vp()
    _check(_lib.cav_setup(sys.handle, C.byref(d), _stream(stream), C.byref(out)), "cav_setup")
    return Hierarchy(out, sys, dict(kind=kind, coarsest_N=coarsest_N, nu_pre=nu_pre, nu_post=nu_post,
                                    alpha=alpha, precision=precision, autotune=autotune, smoother=smoother,
                                    coloured_levels=coloured_levels, nu_additive=nu_additive, box=tuple(box)))


def cav_refactor(h: Hierarchy, sys: System, stream=None) -> bool:
    """Recompute h's numbers for sys's E_E when its pattern is unchanged (True); False (h
    unchanged) when the pattern differs and a new cav_setup is needed."""
    st = _lib.cav_refactor(h.handle, sys.handle, _stream(stream))
    if st == IB_ERR_INVALID and "pattern changed" in _lib.ib_last_error().decode():
        return False
    _check(st, "cav_refactor")
    h.system = sys
    return True


def cav_num_levels(h: Hierarchy) -> int:
    n = C.c_int32()
    _check(_lib.cav_num_levels(h.handle, C.byref(n)), "cav_num_levels")
    return n.value


def cav_get_level_info(h: Hierarchy, level: int) -> dict:
    info = cav_level_info()
    _check(_lib.cav_get_level_info(h.handle, level, C.byref(info)), "cav_get_level_info")
    out = {f: getattr(info, f) for f, _ in info._fields_}
    out["apply_us"] = list(info.apply_us)
    out["sweep_us"] = list(info.sweep_us)
    return out


def cav_patch_export(h: Hierarchy, level: int):
    n = C.c_int32()
    tot = C.c_int64()
    _check(_lib.cav_patch_export(h.handle, level, None, None, C.byref(n), C.byref(tot)), "cav_patch_export")
    off = np.zeros(n.value + 1, dtype=np.int64)
    dofs = np.zeros(tot.value, dtype=np.int32)
    _check(_lib.cav_patch_export(h.handle, level, _vp(off.ctypes.data), _vp(dofs.ctypes.data),
                                 C.byref(n), C.byref(tot)), "cav_patch_export")
    return off, dofs


def cav_colour_export(h: Hierarchy, level: int) -> np.ndarray:
    """Colour class of every patch of a smoothing level, in patch order (coloured smoother)."""
    info = cav_get_level_info(h, level)
    out = np.zeros(info["n_patches"], dtype=np.int32)
    nc = C.c_int32()
    _check(_lib.cav_colour_export(h.handle, level, _vp(out.ctypes.data), C.byref(nc)), "cav_colour_export")
    return out


def cav_ee_export(h: Hierarchy, level: int):
    """(rowptr, cols, vals) over all 2 N_l^2 velocity rows."""
    info = cav_get_level_info(h, level)
    nnz = C.c_int64()
    _check(_lib.cav_ee_export(h.handle, level, None, None, None, C.byref(nnz)), "cav_ee_export")
    rowptr = np.zeros(2 * info["N"] ** 2 + 1, dtype=np.int64)
    cols = np.zeros(nnz.value, dtype=np.int32)
    vals = np.zeros(nnz.value, dtype=np.float64)
    _check(_lib.cav_ee_export(h.handle, level, _vp(rowptr.ctypes.data), _vp(cols.ctypes.data),
                              _vp(vals.ctypes.data), C.byref(nnz)), "cav_ee_export")
    return rowptr, cols, vals


def cav_sweep(h: Hierarchy, level: int, b, w, stream=None):
    _check(_lib.cav_sweep(h.handle, level, _dev(b), _dev(w), _stream(stream)), "cav_sweep")


def cav_sweep_noalloc(h: Hierarchy, level: int, b, w, stream=None):
    """cav_sweep with its scratch in the library's fixed device array (allocates nothing)."""
    _check(_lib.cav_sweep_noalloc(h.handle, level, _dev(b), _dev(w), _stream(stream)), "cav_sweep_noalloc")


def cav_residual(h: Hierarchy, level: int, b, w, r, stream=None):
    _check(_lib.cav_residual(h.handle, level, _dev(b), _dev(w), _dev(r), _stream(stream)), "cav_residual")


def cav_restrict(h: Hierarchy, level: int, r, bc, stream=None):
    _check(_lib.cav_restrict(h.handle, level, _dev(r), _dev(bc), _stream(stream)), "cav_restrict")


def cav_prolong_add(h: Hierarchy, level: int, xc, w, stream=None):
    _check(_lib.cav_prolong_add(h.handle, level, _dev(xc), _dev(w), _stream(stream)), "cav_prolong_add")


def cav_coarse_solve(h: Hierarchy, r, z, stream=None):
    _check(_lib.cav_coarse_solve(h.handle, _dev(r), _dev(z), _stream(stream)), "cav_coarse_solve")


def vcycle_apply(h: Hierarchy, r, z, stream=None):
    _check(_lib.vcycle_apply(h.handle, _dev(r), _dev(z), _stream(stream)), "vcycle_apply")


def ib_test_wait_stall(enable: bool):
    """Test hook: make the kernels' bounded data waits run out (see include/ib_cav.h)."""
    _check(_lib.ib_test_wait_stall(1 if enable else 0), "ib_test_wait_stall")


def ib_launch_count() -> int:
    return int(_lib.ib_launch_count())


def cav_profile(h: Hierarchy, enable: bool):
    _check(_lib.cav_profile(h.handle, 1 if enable else 0), "cav_profile")


def cav_profile_read(h: Hierarchy):
    n = C.c_int32()
    ms = C.c_double()
    _check(_lib.cav_profile_read(h.handle, C.byref(n), C.byref(ms)), "cav_profile_read")
    return n.value, ms.value


def fgmres_solve(sys: System, h: Hierarchy, b, x, rtol=1e-10, maxit=60, rel_to=0, history=True,
                 stream=None, raise_on_noconv=False, loop="host") -> dict:
    """b, x: CUDA tensors, or host buffers (numpy float64 arrays or CPU torch tensors, e.g.
    pinned) -- then the call copies b and x in and x out inside the call.  loop "device": the
    solve is one CUDA graph launch (device buffers only)."""
    host = isinstance(b, np.ndarray) or (hasattr(b, "is_cuda") and not b.is_cuda)
    d = fgmres_desc(float(rtol), int(maxit), int(rel_to), 1 if host else 0, LOOP[loop])
    info = fgmres_info()
    hist = np.zeros(maxit + 1) if history else None
    if host:
        if isinstance(b, np.ndarray):
            assert isinstance(x, np.ndarray) and b.dtype == np.float64 and x.dtype == np.float64
            bp, xp = _vp(b.ctypes.data), _vp(x.ctypes.data)
        else:
            bp, xp = _vp(b.data_ptr()), _vp(x.data_ptr())
    else:
        bp, xp = _dev(b), _dev(x)
    st = _lib.fgmres_solve(sys.handle, h.handle, bp, xp, C.byref(d), C.byref(info),
                           _vp(hist.ctypes.data) if hist is not None else None, _stream(stream))
    if st not in (IB_OK, IB_ERR_NOCONV) or (st == IB_ERR_NOCONV and raise_on_noconv):
        raise IBError(st, "fgmres_solve")
    out = {f: getattr(info, f) for f, _ in info._fields_}
    if hist is not None:
        out["history"] = hist[:info.iters + 1].copy()
    return out


def fgmres_solve_batched(systems, hierarchies, bs, xs, rtol=1e-10, maxit=60, rel_to=0, stream=None,
                         raise_on_noconv=False, loop="host") -> list:
    """Solve many independent systems together; bs, xs are lists of CUDA tensors.  loop
    "device": the whole batch is one CUDA graph launch."""
    n = len(systems)
    assert n == len(hierarchies) == len(bs) == len(xs) and n >= 1
    arr = _vp * n
    sysa = arr(*[s.handle for s in systems])
    hiera = arr(*[h.handle for h in hierarchies])
    ba = arr(*[_dev(b) for b in bs])
    xa = arr(*[_dev(x) for x in xs])
    infos = (fgmres_info * n)()
    d = fgmres_desc(float(rtol), int(maxit), int(rel_to), 0, LOOP[loop])
    st = _lib.fgmres_solve_batched(n, sysa, hiera, ba, xa, C.byref(d), infos, _stream(stream))
    if st not in (IB_OK, IB_ERR_NOCONV) or (st == IB_ERR_NOCONV and raise_on_noconv):
        raise IBError(st, "fgmres_solve_batched")
    return [{f: getattr(i, f) for f, _ in i._fields_} for i in infos]


def _devf(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("network tensors must be contiguous float32 CUDA tensors")
    return _vp(t.data_ptr())


class IBNet:
    """Owns an ibnet handle (the learned-initial-guess network)."""

    def __init__(self, in_ch=15, hidden=32, n_hidden=3, out_ch=3, seed=1):
        d = ibnet_desc(in_ch, hidden, n_hidden, out_ch, seed)
        h = _vp()
        _check(_lib.ibnet_create(C.byref(d), C.byref(h)), "ibnet_create")
        self._h = h
        self.desc = dict(in_ch=in_ch, hidden=hidden, n_hidden=n_hidden, out_ch=out_ch, seed=seed)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.ibnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self) -> int:
        return int(_lib.ibnet_num_params(self._h))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.num_params(), dtype=np.float32)
        _check(_lib.ibnet_get_params(self._h, _vp(out.ctypes.data)), "ibnet_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(_lib.ibnet_set_params(self._h, _vp(p.ctypes.data)), "ibnet_set_params")

    def inner(self, a, b, stream=None) -> float:
        """<a, b> of two FP32 device tensors, accumulated in FP64."""
        assert a.numel() == b.numel()
        out = C.c_double()
        _check(_lib.ibnet_inner(self._h, a.numel(), _devf(a), _devf(b), C.byref(out), _stream(stream)),
               "ibnet_inner")
        return out.value

    def forward(self, x, out, batch, N, stream=None):
        _check(_lib.ibnet_forward(self._h, _devf(x), _devf(out), batch, N, _stream(stream)), "ibnet_forward")

    def gradients(self, x, target, batch, N, stream=None):
        loss = C.c_float()
        g = np.zeros(self.num_params(), dtype=np.float32)
        _check(_lib.ibnet_gradients(self._h, _devf(x), _devf(target), batch, N, C.byref(loss), _vp(g.ctypes.data),
                                    _stream(stream)), "ibnet_gradients")
        return float(loss.value), g

    def train_step(self, x, target, batch, N, lr, want_loss=False, stream=None):
        loss = C.c_float()
        _check(_lib.ibnet_train_step(self._h, _devf(x), _devf(target), batch, N, float(lr),
                                     C.byref(loss) if want_loss else None, _stream(stream)), "ibnet_train_step")
        return float(loss.value) if want_loss else None


def ibnet_pack_input(N, hist_x, hist_f, in_scale, out, stream=None):
    hx = (_vp * 3)(*[_dev(t) for t in hist_x])
    hf = (_vp * 3)(*[_dev(t) for t in hist_f])
    sc = (C.c_float * 15)(*[float(v) for v in in_scale])
    _check(_lib.ibnet_pack_input(N, hx, hf, sc, _devf(out), _stream(stream)), "ibnet_pack_input")


def ibnet_pack_history(N, hist_x, hist_f, in_scale, out, stream=None):
    K = len(hist_x)
    hx = (_vp * K)(*[_dev(t) for t in hist_x])
    hf = (_vp * K)(*[_dev(t) for t in hist_f])
    sc = (C.c_float * (5 * K))(*[float(v) for v in in_scale])
    _check(_lib.ibnet_pack_history(N, K, hx, hf, sc, _devf(out), _stream(stream)), "ibnet_pack_history")


def ibnet_pack_target(N, x_new, x_prev, out_scale, out, x_prev2=None, x_prev3=None, stream=None):
    sc = (C.c_float * 3)(*[float(v) for v in out_scale])
    _check(_lib.ibnet_pack_target(N, _dev(x_new), _dev(x_prev), _dev(x_prev2), _dev(x_prev3), sc, _devf(out),
                                  _stream(stream)), "ibnet_pack_target")


def ibnet_apply_delta(N, x_prev, delta, out_scale, x_out, x_prev2=None, x_prev3=None, stream=None):
    sc = (C.c_float * 3)(*[float(v) for v in out_scale])
    _check(_lib.ibnet_apply_delta(N, _dev(x_prev), _dev(x_prev2), _dev(x_prev3), None if delta is None else _devf(delta),
                                  sc, _dev(x_out), _stream(stream)), "ibnet_apply_delta")
