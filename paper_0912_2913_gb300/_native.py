"""ctypes binding of librlb (include/rlb.h), one Python function per C entry point.

Argument marshalling only: every function converts torch tensors or numpy
arrays to raw pointers, calls the C function of the same name and raises
``RLBError`` on a non-OK status.  No arithmetic of the scheme happens here.
The library is built in-tree by ``paper_0912_2913_gb300.build``; importing
this module without a CUDA toolkit or loading it without a GPU fails loudly
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

RLB_OK, RLB_ERR_ARG, RLB_ERR_OOM, RLB_ERR_CUDA, RLB_ERR_UNPHYSICAL, RLB_ERR_STATE = range(6)
RLB_FP64, RLB_FP32_DEV = 0, 1
RLB_BC_PERIODIC, RLB_BC_INFLOW_OUTFLOW, RLB_BC_OUTFLOW_BOTH = 0, 1, 2
RLB_HOST, RLB_DEVICE = 0, 1
RLB_EOS_ULTRA, RLB_EOS_GAMMA_LAW = 0, 1
RLB_ZBC_PERIODIC, RLB_ZBC_HALO = 0, 1

# Every symbol include/rlb.h declares.
EXPORTS = (
    "rlb_state_layout", "rlb_workspace_bytes", "rlb_create", "rlb_destroy", "rlb_init_fields", "rlb_step",
    "rlb_step_into", "rlb_step_into_counted", "rlb_state_ptr", "rlb_save_state", "rlb_load_state", "rlb_macro", "rlb_stats",
    "rlb_adjoint_macro", "rlb_adjoint_step", "rlb_adjoint_fields", "rlb_sync", "rlb_status_str", "rlb_last_error",
    "rlb_launch_count", "rlb_selftest_conversions", "rlb_adjoint_step_noalloc", "rlb_debug_bounds_violations",
    "rlb_debug_bounds_selftest", "rlb_halo_exchange",
)


class RLBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [status {status}]")
        self.status = status


class rlb_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("xbc", ctypes.c_int32), ("eos", ctypes.c_int32),
                ("tau", ctypes.c_double), ("c_l", ctypes.c_double),
                ("n_in", ctypes.c_double), ("eps_in", ctypes.c_double), ("beta_in", ctypes.c_double * 3),
                ("n_ref", ctypes.c_double), ("eps_ref", ctypes.c_double),
                ("eos_gamma", ctypes.c_double), ("eos_mass", ctypes.c_double),
                ("zbc", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def _bounds_variant() -> bool:
    """RLB_LIBRARY_VARIANT=bounds loads the bounds-checking debug library."""
    v = os.environ.get("RLB_LIBRARY_VARIANT", "release")
    if v not in ("release", "bounds"):
        raise ValueError(f"RLB_LIBRARY_VARIANT must be 'release' or 'bounds', not {v!r}")
    return v == "bounds"


def library_path() -> str:
    from . import build as _build

    return _build.library_path(bounds=_bounds_variant())


def load(build_if_missing: bool = True):
    """Load librlb (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build

        bounds = _bounds_variant()
        path = _build.library_path(bounds=bounds)
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"librlb is not built ({path}); run __graft_entry__.build()")
            path = _build.build(bounds=bounds)
        L = ctypes.CDLL(path)
        vp, sz, i32, i64, dp = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        P = ctypes.POINTER
        st = ctypes.c_int
        sig = {
            "rlb_state_layout": ([P(rlb_params), P(i64), P(i32), P(sz)], st),
            "rlb_workspace_bytes": ([P(rlb_params), P(sz)], st),
            "rlb_create": ([P(rlb_params), vp, vp, sz, P(vp)], st),
            "rlb_destroy": ([vp], st),
            "rlb_init_fields": ([vp, dp, dp, dp, vp, ctypes.c_int], st),
            "rlb_step": ([vp, i32], st),
            "rlb_step_into": ([vp, vp, vp], st),
            "rlb_step_into_counted": ([vp, vp, vp], st),
            "rlb_state_ptr": ([vp, P(vp)], st),
            "rlb_save_state": ([vp, vp], st),
            "rlb_load_state": ([vp, vp], st),
            "rlb_macro": ([vp, vp, dp, dp, dp, ctypes.c_int], st),
            "rlb_stats": ([vp, P(i64), P(i64), P(i64), P(i64)], st),
            "rlb_adjoint_macro": ([vp, vp, dp, dp, dp, vp], st),
            "rlb_adjoint_step": ([vp, vp, vp, vp, dp, dp], st),
            "rlb_adjoint_step_noalloc": ([vp, vp, vp, vp, dp, dp], st),
            "rlb_adjoint_fields": ([vp, dp, dp, dp, vp, dp, dp, dp, dp], st),
            "rlb_sync": ([vp], st),
            "rlb_status_str": ([ctypes.c_int], ctypes.c_char_p),
            "rlb_last_error": ([vp], ctypes.c_char_p),
            "rlb_launch_count": ([vp], i64),
            "rlb_selftest_conversions": ([vp, vp, i64, vp, vp], st),
            "rlb_debug_bounds_violations": ([P(i64)], st),
            "rlb_debug_bounds_selftest": ([i64, i64, P(i64)], st),
            "rlb_halo_exchange": ([vp, vp], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def _ptr(x) -> int | None:
    """Raw address of a torch tensor or numpy array (None passes through)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to librlb must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays passed to librlb must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} to librlb")


def _dptr(x) -> int | None:
    """Address of a device buffer: a CUDA tensor (a raw int address and None
    pass through).  Host arrays and CPU tensors are refused here, before the
    library could hand a host address to a kernel."""
    if x is None or isinstance(x, int):
        return x
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        return _ptr(x)
    where = "a CPU tensor" if hasattr(x, "data_ptr") else type(x).__name__
    raise ValueError(f"librlb expects a device buffer (a CUDA tensor) here, not {where}")


def _wptr(x, where: int) -> int | None:
    """Address of a buffer on the side that `where` names: RLB_DEVICE a CUDA
    tensor, RLB_HOST a numpy array or a CPU tensor."""
    if where == RLB_DEVICE:
        return _dptr(x)
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        raise ValueError("librlb expects a host buffer here (RLB_HOST), not a CUDA tensor")
    return _ptr(x)


def _check(status: int, ctx=None, allow=()) -> int:
    if status == RLB_OK or status in allow:
        return status
    L = load()
    msg = L.rlb_last_error(ctx).decode(errors="replace")
    raise RLBError(status, f"{L.rlb_status_str(status).decode()}: {msg}")


def make_params(nx, ny, nz, tau, c_l=1.0, prec=RLB_FP64, xbc=RLB_BC_PERIODIC, n_in=1.0, eps_in=1.0,
                beta_in=(0.0, 0.0, 0.0), n_ref=1.0, eps_ref=1.0, eos=RLB_EOS_ULTRA, eos_gamma=4.0 / 3.0,
                eos_mass=0.0, zbc=RLB_ZBC_PERIODIC) -> rlb_params:
    p = rlb_params()
    p.zbc, p.reserved = int(zbc), 0
    p.nx, p.ny, p.nz, p.prec, p.xbc, p.eos = int(nx), int(ny), int(nz), int(prec), int(xbc), int(eos)
    p.eos_gamma, p.eos_mass = float(eos_gamma), float(eos_mass)
    p.tau, p.c_l, p.n_in, p.eps_in = float(tau), float(c_l), float(n_in), float(eps_in)
    for a in range(3):
        p.beta_in[a] = float(beta_in[a])
    p.n_ref, p.eps_ref = float(n_ref), float(eps_ref)
    return p


def rlb_state_layout(p: rlb_params):
    S, e, b = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_size_t()
    _check(load().rlb_state_layout(ctypes.byref(p), ctypes.byref(S), ctypes.byref(e), ctypes.byref(b)))
    return S.value, e.value, b.value


def rlb_workspace_bytes(p: rlb_params) -> int:
    b = ctypes.c_size_t()
    _check(load().rlb_workspace_bytes(ctypes.byref(p), ctypes.byref(b)))
    return b.value


def rlb_create(p: rlb_params, stream: int, workspace, workspace_bytes: int) -> int:
    ctx = ctypes.c_void_p()
    _check(load().rlb_create(ctypes.byref(p), stream, _dptr(workspace), workspace_bytes, ctypes.byref(ctx)))
    return ctx.value


def rlb_destroy(ctx: int) -> None:
    _check(load().rlb_destroy(ctx))


def rlb_init_fields(ctx, n, eps, beta, solid, where) -> None:
    _check(load().rlb_init_fields(ctx, _wptr(n, where), _wptr(eps, where), _wptr(beta, where), _wptr(solid, where),
                                  where), ctx)


def rlb_step(ctx, nsteps: int) -> None:
    _check(load().rlb_step(ctx, int(nsteps)), ctx)


def rlb_step_into(ctx, src, dst) -> None:
    _check(load().rlb_step_into(ctx, _dptr(src), _dptr(dst)), ctx)


def rlb_step_into_counted(ctx, src, dst) -> None:
    _check(load().rlb_step_into_counted(ctx, _dptr(src), _dptr(dst)), ctx)


def rlb_state_ptr(ctx) -> int:
    v = ctypes.c_void_p()
    _check(load().rlb_state_ptr(ctx, ctypes.byref(v)), ctx)
    return v.value


def rlb_save_state(ctx, dst) -> None:
    _check(load().rlb_save_state(ctx, _dptr(dst)), ctx)


def rlb_load_state(ctx, src) -> None:
    _check(load().rlb_load_state(ctx, _dptr(src)), ctx)


def rlb_macro(ctx, state, n, eps, beta, where) -> int:
    """Returns RLB_OK or RLB_ERR_UNPHYSICAL (outputs written in both cases)."""
    return _check(load().rlb_macro(ctx, _dptr(state), _wptr(n, where), _wptr(eps, where), _wptr(beta, where), where),
                  ctx,
                  allow=(RLB_ERR_UNPHYSICAL,))


def rlb_stats(ctx) -> dict:
    a, b, c, d = (ctypes.c_int64() for _ in range(4))
    _check(load().rlb_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), ctx)
    return dict(steps=a.value, n_unphysical=b.value, first_bad=c.value, n_nonpositive_eq=d.value)


def rlb_adjoint_macro(ctx, state, dL_dn, dL_deps, dL_dbeta, lam_out) -> None:
    _check(load().rlb_adjoint_macro(ctx, _dptr(state), _dptr(dL_dn), _dptr(dL_deps), _dptr(dL_dbeta), _dptr(lam_out)),
           ctx)


def rlb_adjoint_step(ctx, state_t, lam_in, lam_out, dL_dtau_accum, dL_dbeta_in_accum) -> None:
    _check(load().rlb_adjoint_step(ctx, _dptr(state_t), _dptr(lam_in), _dptr(lam_out), _dptr(dL_dtau_accum),
                                   _dptr(dL_dbeta_in_accum)), ctx)


def rlb_adjoint_step_noalloc(ctx, state_t, lam_in, lam_out, dL_dtau_accum, dL_dbeta_in_accum) -> None:
    _check(load().rlb_adjoint_step_noalloc(ctx, _dptr(state_t), _dptr(lam_in), _dptr(lam_out), _dptr(dL_dtau_accum),
                                           _dptr(dL_dbeta_in_accum)), ctx)


def rlb_adjoint_fields(ctx, n0, eps0, beta0, lam0, dL_dn0, dL_deps0, dL_dbeta0, dL_dbeta_in_accum) -> None:
    _check(load().rlb_adjoint_fields(ctx, _dptr(n0), _dptr(eps0), _dptr(beta0), _dptr(lam0), _dptr(dL_dn0),
                                     _dptr(dL_deps0), _dptr(dL_dbeta0), _dptr(dL_dbeta_in_accum)), ctx)


def rlb_sync(ctx) -> None:
    _check(load().rlb_sync(ctx), ctx)


def rlb_status_str(status: int) -> str:
    return load().rlb_status_str(status).decode()


def rlb_last_error(ctx=None) -> str:
    return load().rlb_last_error(ctx).decode(errors="replace")


def rlb_selftest_conversions(f_in, d_in, n, f2d_out, d2f_out) -> None:
    _check(load().rlb_selftest_conversions(_dptr(f_in), _dptr(d_in), int(n), _dptr(f2d_out), _dptr(d2f_out)))


def rlb_debug_bounds_violations() -> int:
    """Out-of-range state indices counted by the bounds-checking build."""
    v = ctypes.c_int64()
    _check(load().rlb_debug_bounds_violations(ctypes.byref(v)))
    return v.value


def rlb_debug_bounds_selftest(index: int, n: int) -> int:
    """The bounds build's index check run on one index in a kernel."""
    v = ctypes.c_int64()
    _check(load().rlb_debug_bounds_selftest(index, n, ctypes.byref(v)))
    return v.value


def rlb_launch_count(ctx) -> int:
    return int(load().rlb_launch_count(ctx))


def rlb_halo_exchange(lower, upper) -> None:
    _check(load().rlb_halo_exchange(lower, upper), lower)
