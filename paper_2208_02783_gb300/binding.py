"""ctypes binding of the C ABI in include/transec.h.

Argument marshalling only: every function here converts its arguments to plain
pointers and sizes and calls the entry point of the same name in libtransec.so.
All arithmetic happens in the library's CUDA kernels; there is no fallback, and
loading fails loudly when the library has not been built.

Arrays may be NumPy arrays (host memory) or torch tensors (host or CUDA memory).
A call takes all of its array arguments from one side: either every array is a
CUDA tensor (``on_device`` = 1) or none is.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_native", "libtransec.so")

# status codes (enum transec_status)
OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBREAKDOWN, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
METHOD_AUTO, METHOD_COCG, METHOD_BICG = 0, 1, 2
PREC_FP64, PREC_MIXED, PREC_DF64 = 0, 1, 2


class TransecError(RuntimeError):
    """A library call returned a non-zero status."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class SolverOpts(C.Structure):
    _fields_ = [
        ("method", C.c_int),
        ("precision", C.c_int),
        ("tol", C.c_double),
        ("maxit", C.c_int),
        ("slots", C.c_int),
        ("chunk", C.c_int),
        ("reliable", C.c_double),
        ("tile_y", C.c_int),
        ("slab", C.c_int),
        ("profile", C.c_int),
        ("mixed_maxit", C.c_int),
        ("mixed_decade_its", C.c_int),
        ("host_loop", C.c_int),
        ("df_stall_its", C.c_int),
        ("psym", C.c_int),
        ("sketch_guard", C.c_double),
    ]


_lib = None

_P = C.c_void_p
_SIGS = {
    "transec_version": (C.c_int, []),
    "transec_status_string": (C.c_char_p, [C.c_int]),
    "transec_create": (
        C.c_int,
        [C.POINTER(_P), C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _P],
    ),
    "transec_set_potential": (C.c_int, [_P, _P, C.c_int]),
    "transec_set_abc": (C.c_int, [_P, _P, _P]),
    "transec_set_kmesh": (C.c_int, [_P, C.c_int, _P, _P]),
    "transec_set_solver": (C.c_int, [_P, C.POINTER(SolverOpts)]),
    "transec_get_solver": (C.c_int, [_P, C.POINTER(SolverOpts)]),
    "transec_n_rhs": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "transec_autotune": (C.c_int, [_P, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]),
    "transec_transmission": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P]),
    "transec_column_contributions": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P, C.c_int]),
    "transec_batch_column_contributions": (
        C.c_int, [C.c_int, _P, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P, C.c_int]),
    "transec_apply": (C.c_int, [_P, C.c_double, C.c_int, C.c_int, C.c_int, _P, _P, C.c_int]),
    "transec_apply_noalloc": (C.c_int, [_P, C.c_double, C.c_int, C.c_int, C.c_int, _P, _P]),
    "transec_trace": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int]),
    "transec_stats": (C.c_int, [_P] + [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "transec_stats_reset": (C.c_int, [_P]),
    "transec_unet_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong]),
    "transec_unet_n_params": (C.c_int, [_P, C.POINTER(C.c_longlong)]),
    "transec_unet_set_params": (C.c_int, [_P, _P]),
    "transec_unet_get_params": (C.c_int, [_P, _P]),
    "transec_unet_forward": (C.c_int, [_P, _P, _P, C.c_int]),
    "transec_unet_train_step": (C.c_int, [_P, _P, _P, C.c_float, C.POINTER(C.c_float), _P, C.c_int]),
    "transec_unet_dims": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "transec_unet_last_error": (C.c_char_p, [_P]),
    "transec_unet_train_operator": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_float,
                                             C.c_ulonglong, _P]),
    "transec_fgmres_columns": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, _P, C.c_int, C.c_int, _P, _P, _P,
                                         _P]),
    "transec_shifted_column": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_longlong, _P, _P, _P, _P]),
    "transec_shifted_columns": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, _P, _P, _P, _P, _P]),
    "transec_transmission_sketch": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, C.c_int, C.c_int, C.c_ulonglong,
                                              _P, _P, _P, _P, _P, _P]),
    "transec_sweep_stats": (C.c_int, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                      C.POINTER(C.c_longlong), C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                      C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "transec_unet_destroy": (None, [_P]),
    "transec_unet_set_path": (C.c_int, [_P, C.c_int]),
    "transec_unet_zero_output": (C.c_int, [_P]),
    "transec_eigen_transmission": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int, _P, _P]),
    "transec_eigen_stats": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "transec_unet_conv3d": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P,
                                      C.c_int]),
    "transec_last_error": (C.c_char_p, [_P]),
    "transec_destroy": (None, [_P]),
}

EXPORTED = tuple(_SIGS)


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libtransec.so (built by paper_2208_02783_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_2208_02783_gb300.build` "
            "(the library has no CPU fallback)"
        )
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(ctx, status: int, what: str, allow=()):
    if status == OK or status in allow:
        return status
    lib = load()
    msg = lib.transec_last_error(ctx).decode() if ctx else ""
    if allow and msg.startswith("some "):
        # per-result failures: the status arrays say which results failed
        return status
    raise TransecError(status, f"{what}: {lib.transec_status_string(status).decode()}: {msg}")


class _Arr:
    """Pointer view of a NumPy array or torch tensor with a required dtype."""

    def __init__(self, a, dtype, writable=False):
        self.device = False
        self.keep = None
        try:
            import torch  # noqa: F401

            is_torch = hasattr(a, "data_ptr") and hasattr(a, "is_cuda")
        except ImportError:  # pragma: no cover
            is_torch = False
        if is_torch:
            tdt = {np.float64: "torch.float64", np.int32: "torch.int32", np.int64: "torch.int64",
                   np.float32: "torch.float32"}[dtype]
            if str(a.dtype) != tdt:
                raise TypeError(f"expected {tdt}, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            self.device = bool(a.is_cuda)
            self.keep = a
            self.ptr = C.c_void_p(a.data_ptr())
        else:
            arr = np.asarray(a)
            if writable:
                if arr.dtype != dtype or not arr.flags.c_contiguous:
                    raise TypeError(f"output must be a C-contiguous {np.dtype(dtype)} array")
            else:
                arr = np.ascontiguousarray(arr, dtype=dtype)
            self.keep = arr
            self.ptr = arr.ctypes.data_as(C.c_void_p)


def _side(arrs):
    dev = {x.device for x in arrs if x is not None}
    if len(dev) > 1:
        raise ValueError("mixing host and device arrays in one call")
    return 1 if dev == {True} else 0


def _complex_view(x):
    """complex128 NumPy array -> float64 view; torch complex128 -> view_as_real."""
    if hasattr(x, "is_cuda"):
        import torch

        if x.dtype == torch.complex128:
            return torch.view_as_real(x)
        return x
    x = np.ascontiguousarray(x)
    if x.dtype == np.complex128:
        return x.view(np.float64)
    return x


# ----------------------------------------------------------------------------------
# the entry points, one per C function
# ----------------------------------------------------------------------------------


def transec_version() -> int:
    return load().transec_version()


def transec_status_string(status: int) -> str:
    return load().transec_status_string(status).decode()


def transec_create(nx, ny, nz, hx, hy, hz, fd_order, device=0, stream=None):
    lib = load()
    out = C.c_void_p()
    st = lib.transec_create(C.byref(out), nx, ny, nz, hx, hy, hz, fd_order, device,
                            C.c_void_p(stream) if stream else None)
    if st != OK:
        raise TransecError(st, f"transec_create: {lib.transec_status_string(st).decode()}")
    _NPOINTS[out.value] = int(nx) * int(ny) * int(nz)
    return out


def transec_set_potential(ctx, v_ks):
    a = _Arr(v_ks, np.float64)
    return _check(ctx, load().transec_set_potential(ctx, a.ptr, _side([a])), "transec_set_potential")


def transec_set_abc(ctx, gamma_l, gamma_r):
    a = _Arr(np.asarray(gamma_l, np.float64), np.float64)
    b = _Arr(np.asarray(gamma_r, np.float64), np.float64)
    return _check(ctx, load().transec_set_abc(ctx, a.ptr, b.ptr), "transec_set_abc")


def transec_set_kmesh(ctx, kfrac, weights=None):
    k = _Arr(np.asarray(kfrac, np.float64).reshape(-1, 2), np.float64)
    nk = k.keep.shape[0]
    w = _Arr(np.asarray(weights, np.float64), np.float64) if weights is not None else None
    return _check(ctx, load().transec_set_kmesh(ctx, nk, k.ptr, w.ptr if w else None), "transec_set_kmesh")


def transec_set_solver(ctx, opts: SolverOpts):
    return _check(ctx, load().transec_set_solver(ctx, C.byref(opts)), "transec_set_solver")


def transec_get_solver(ctx) -> SolverOpts:
    o = SolverOpts()
    _check(ctx, load().transec_get_solver(ctx, C.byref(o)), "transec_get_solver")
    return o


def transec_n_rhs(ctx) -> int:
    n = C.c_int64()
    _check(ctx, load().transec_n_rhs(ctx, C.byref(n)), "transec_n_rhs")
    return int(n.value)


def transec_autotune(ctx, energy, ik) -> dict:
    v = [C.c_int(), C.c_int(), C.c_int()]
    _check(ctx, load().transec_autotune(ctx, float(energy), int(ik), *[C.byref(x) for x in v]),
           "transec_autotune")
    return {"tile_y": v[0].value, "slab": v[1].value, "slots": v[2].value}


def transec_transmission(ctx, energies, T_out, T_avg_out=None, status_out=None, iters_out=None):
    e = _Arr(energies, np.float64)
    t = _Arr(T_out, np.float64, writable=True)
    ta = _Arr(T_avg_out, np.float64, writable=True) if T_avg_out is not None else None
    so = _Arr(status_out, np.int32, writable=True) if status_out is not None else None
    io = _Arr(iters_out, np.int32, writable=True) if iters_out is not None else None
    if _side([e, t, ta, so, io]):
        raise ValueError("transec_transmission takes host arrays")
    ne = int(np.asarray(e.keep).size)
    st = load().transec_transmission(
        ctx, ne, e.ptr, t.ptr, ta.ptr if ta else None, so.ptr if so else None, io.ptr if io else None
    )
    return _check(ctx, st, "transec_transmission", allow=(ENOCONV, EBREAKDOWN))


def transec_column_contributions(ctx, energies, ik, cols, t_out, t_minus_out=None, iters_out=None,
                                 status_out=None):
    e = _Arr(energies, np.float64)
    k = _Arr(ik, np.int32)
    c = _Arr(cols, np.int64)
    t = _Arr(t_out, np.float64, writable=True)
    tm = _Arr(t_minus_out, np.float64, writable=True) if t_minus_out is not None else None
    io = _Arr(iters_out, np.int32, writable=True) if iters_out is not None else None
    so = _Arr(status_out, np.int32, writable=True) if status_out is not None else None
    side = _side([e, k, c, t, tm, io, so])
    n = int(e.keep.numel() if hasattr(e.keep, "numel") else np.asarray(e.keep).size)
    st = load().transec_column_contributions(
        ctx, n, e.ptr, k.ptr, c.ptr, t.ptr, tm.ptr if tm else None, io.ptr if io else None,
        so.ptr if so else None, side,
    )
    return _check(ctx, st, "transec_column_contributions", allow=(ENOCONV, EBREAKDOWN))


def transec_batch_column_contributions(ctxs, ictx, energies, ik, cols, t_out, t_minus_out=None,
                                       iters_out=None, status_out=None):
    """Columns of several contexts in one solve; ``ictx`` picks each item's context."""
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    i = _Arr(ictx, np.int32)
    e = _Arr(energies, np.float64)
    k = _Arr(ik, np.int32)
    c = _Arr(cols, np.int64)
    t = _Arr(t_out, np.float64, writable=True)
    tm = _Arr(t_minus_out, np.float64, writable=True) if t_minus_out is not None else None
    io = _Arr(iters_out, np.int32, writable=True) if iters_out is not None else None
    so = _Arr(status_out, np.int32, writable=True) if status_out is not None else None
    side = _side([i, e, k, c, t, tm, io, so])
    n = int(e.keep.numel() if hasattr(e.keep, "numel") else np.asarray(e.keep).size)
    st = load().transec_batch_column_contributions(
        len(ctxs), C.cast(arr, C.c_void_p), n, i.ptr, e.ptr, k.ptr, c.ptr, t.ptr,
        tm.ptr if tm else None, io.ptr if io else None, so.ptr if so else None, side,
    )
    return _check(ctxs[0], st, "transec_batch_column_contributions", allow=(ENOCONV, EBREAKDOWN))


def transec_apply(ctx, energy, ik, x, y, conj_k=False):
    xv = _complex_view(x)
    yv = _complex_view(y)
    a = _Arr(xv, np.float64)
    b = _Arr(yv, np.float64, writable=True)
    side = _side([a, b])
    n_el = int(a.keep.numel() if hasattr(a.keep, "numel") else a.keep.size)
    g = transec_n_points(ctx)
    nvec = n_el // (2 * g)
    st = load().transec_apply(ctx, float(energy), int(ik), 1 if conj_k else 0, nvec, a.ptr, b.ptr, side)
    return _check(ctx, st, "transec_apply")


def transec_apply_noalloc(ctx, energy, ik, x, y, conj_k=False):
    """y = A(E, k) x with no device allocation; x and y must be CUDA tensors."""
    xv = _complex_view(x)
    yv = _complex_view(y)
    a = _Arr(xv, np.float64)
    b = _Arr(yv, np.float64, writable=True)
    if _side([a, b]) != 1:
        raise ValueError("transec_apply_noalloc takes device (CUDA) tensors")
    nvec = int(a.keep.numel()) // (2 * transec_n_points(ctx))
    st = load().transec_apply_noalloc(ctx, float(energy), int(ik), 1 if conj_k else 0, nvec, a.ptr, b.ptr)
    return _check(ctx, st, "transec_apply_noalloc")


def transec_trace(ctx, x, cols, t_out):
    xv = _complex_view(x)
    a = _Arr(xv, np.float64)
    c = _Arr(cols, np.int64)
    t = _Arr(t_out, np.float64, writable=True)
    side = _side([a, c, t])
    nvec = int(c.keep.numel() if hasattr(c.keep, "numel") else np.asarray(c.keep).size)
    st = load().transec_trace(ctx, nvec, a.ptr, c.ptr, t.ptr, side)
    return _check(ctx, st, "transec_trace")


def transec_stats(ctx) -> dict:
    v = [C.c_longlong(), C.c_longlong(), C.c_double(), C.c_longlong(), C.c_double(), C.c_longlong(),
         C.c_longlong(), C.c_longlong(), C.c_double(), C.c_longlong()]
    _check(ctx, load().transec_stats(ctx, *[C.byref(x) for x in v]), "transec_stats")
    keys = ("launches", "point_applies", "stencil_ms", "stencil_launches", "update_ms", "update_launches",
            "fallbacks", "point_applies32", "stencil32_ms", "stencil32_launches")
    return {k: x.value for k, x in zip(keys, v)}


def transec_stats_reset(ctx):
    return _check(ctx, load().transec_stats_reset(ctx), "transec_stats_reset")


def transec_last_error(ctx) -> str:
    return load().transec_last_error(ctx).decode()


def transec_destroy(ctx):
    if ctx:
        _NPOINTS.pop(ctx.value, None)
        load().transec_destroy(ctx)


# grid size bookkeeping for transec_apply (kept on the Python side of the handle)
_NPOINTS: dict[int, int] = {}


def transec_n_points(ctx) -> int:
    return _NPOINTS[ctx.value]


# ----------------------------------------------------------------------------------
# the learned preconditioner's network
# ----------------------------------------------------------------------------------


def _ucheck(u, st, what):
    if st != OK:
        lib = load()
        raise TransecError(st, f"{what}: {lib.transec_status_string(st).decode()}: "
                               f"{lib.transec_unet_last_error(u).decode() if u else ''}")


def transec_unet_create(device, nx, ny, nz, seed=0):
    out = C.c_void_p()
    _ucheck(None, load().transec_unet_create(C.byref(out), device, nx, ny, nz, seed), "transec_unet_create")
    return out


def transec_unet_n_params(u) -> int:
    n = C.c_longlong()
    _ucheck(u, load().transec_unet_n_params(u, C.byref(n)), "transec_unet_n_params")
    return int(n.value)


def transec_unet_set_params(u, params):
    a = _Arr(np.asarray(params, np.float32), np.float32) if params is not None else None
    _ucheck(u, load().transec_unet_set_params(u, a.ptr if a else None), "transec_unet_set_params")


def transec_unet_get_params(u):
    out = np.zeros(transec_unet_n_params(u), np.float32)
    _ucheck(u, load().transec_unet_get_params(u, out.ctypes.data_as(C.c_void_p)), "transec_unet_get_params")
    return out


def transec_eigen_transmission(ctx, lam, v_right, w_left, energies):
    """T(E, k) from p eigenpairs: lam [p] complex, v_right [n_R][p] and w_left [n_L][p]
    complex (rows of the right / left eigenvectors on the right / left CAP supports)."""
    lam = np.ascontiguousarray(lam, np.complex128)
    vr = np.ascontiguousarray(v_right, np.complex128)
    wl = np.ascontiguousarray(w_left, np.complex128)
    e = np.ascontiguousarray(energies, np.float64)
    t = np.zeros(e.size)
    p = lam.size
    if vr.shape[1] != p or wl.shape[1] != p:
        raise ValueError("eigenvector arrays need p columns")
    st = load().transec_eigen_transmission(ctx, p, lam.ctypes.data_as(C.c_void_p), vr.ctypes.data_as(C.c_void_p),
                                           wl.ctypes.data_as(C.c_void_p), e.size, e.ctypes.data_as(C.c_void_p),
                                           t.ctypes.data_as(C.c_void_p))
    _check(ctx, st, "transec_eigen_transmission")
    return t


def transec_eigen_stats(ctx) -> dict:
    a, b = C.c_double(), C.c_double()
    _check(ctx, load().transec_eigen_stats(ctx, C.byref(a), C.byref(b)), "transec_eigen_stats")
    return {"gram_ms": a.value, "sum_ms": b.value}


def transec_unet_zero_output(u):
    _ucheck(u, load().transec_unet_zero_output(u), "transec_unet_zero_output")


def transec_unet_set_path(u, path):
    """0: tcgen05 convolutions where the plane fits (default); 1: mma.sync only."""
    _ucheck(u, load().transec_unet_set_path(u, int(path)), "transec_unet_set_path")


def transec_unet_conv3d(x_bf16, w_bf16, b, path=0, device=0):
    """One convolution alone: x [nz][ny][nx][cin] and w [27][cout][cin] as bfloat16 bit
    patterns (uint16), b [cout] float32 or None; returns y [nz][ny][nx][cout] float32."""
    x = np.ascontiguousarray(x_bf16, np.uint16)
    w = np.ascontiguousarray(w_bf16, np.uint16)
    nz, ny, nx, cin = x.shape
    cout = w.shape[1]
    y = np.zeros((nz, ny, nx, cout), np.float32)
    bb = None if b is None else np.ascontiguousarray(b, np.float32)
    st = load().transec_unet_conv3d(int(device), nx, ny, nz, cin, cout, x.ctypes.data_as(C.c_void_p),
                                    w.ctypes.data_as(C.c_void_p),
                                    bb.ctypes.data_as(C.c_void_p) if bb is not None else None,
                                    y.ctypes.data_as(C.c_void_p), int(path))
    if st != OK:
        raise TransecError(st, "transec_unet_conv3d")
    return y


def transec_unet_forward(u, x, y):
    a = _Arr(x, np.float32)
    b = _Arr(y, np.float32, writable=True)
    _ucheck(u, load().transec_unet_forward(u, a.ptr, b.ptr, _side([a, b])), "transec_unet_forward")


def transec_unet_train_step(u, x, target, lr, want_grads=False):
    a = _Arr(x, np.float32)
    t = _Arr(target, np.float32)
    loss = C.c_float()
    grads = np.zeros(transec_unet_n_params(u), np.float32) if want_grads else None
    st = load().transec_unet_train_step(u, a.ptr, t.ptr, float(lr), C.byref(loss),
                                        grads.ctypes.data_as(C.c_void_p) if want_grads else None,
                                        _side([a, t]))
    _ucheck(u, st, "transec_unet_train_step")
    return float(loss.value), grads


def transec_unet_destroy(u):
    if u:
        load().transec_unet_destroy(u)


def transec_unet_dims(u):
    d = [C.c_int(), C.c_int(), C.c_int()]
    _ucheck(u, load().transec_unet_dims(u, *[C.byref(x) for x in d]), "transec_unet_dims")
    return tuple(x.value for x in d)


def transec_unet_train_operator(ctx, u, steps, e_lo, e_hi, lr, seed=0, source=1):
    """Fit the network to the context's operator family; returns the per-step losses."""
    loss = np.zeros(max(int(steps), 1), np.float32)
    st = load().transec_unet_train_operator(ctx, u, int(source), int(steps), float(e_lo), float(e_hi), float(lr),
                                            int(seed), loss.ctypes.data_as(C.c_void_p))
    _check(ctx, st, "transec_unet_train_operator")
    return loss[: int(steps)]


def transec_fgmres_columns(ctx, u, energies, ik, cols, restart=30, maxit=20000, net_every=2):
    """FGMRES(restart) columns with the network (None: unpreconditioned) as right
    preconditioner on every net_every-th step; returns (t, iters, status, fallback)."""
    e = np.ascontiguousarray(energies, np.float64)
    k = np.ascontiguousarray(ik, np.int32)
    c = np.ascontiguousarray(cols, np.int64)
    n = e.size
    if k.size != n or c.size != n:
        raise ValueError("energies, ik and cols differ in length")
    t = np.zeros(n, np.float64)
    it = np.zeros(n, np.int32)
    so = np.zeros(n, np.int32)
    fb = np.zeros(n, np.int32)
    vp = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    st = load().transec_fgmres_columns(ctx, u if u else None, int(net_every), n, vp(e), vp(k), vp(c),
                                       int(restart), int(maxit),
                                       vp(t), vp(it), vp(so), vp(fb))
    _check(ctx, st, "transec_fgmres_columns", allow=(ENOCONV, EBREAKDOWN))
    return t, it, so, fb


def transec_shifted_column(ctx, energies, ik, col):
    """One column at several energies by the multi-shift transpose BiCG; returns
    (t, t_minus, iters, status) host arrays in the order of ``energies``."""
    e = np.ascontiguousarray(energies, np.float64)
    n = e.size
    t = np.zeros(n)
    tm = np.zeros(n)
    it = np.zeros(n, np.int32)
    so = np.zeros(n, np.int32)
    vp = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    st = load().transec_shifted_column(ctx, n, vp(e), int(ik), int(col), vp(t), vp(tm), vp(it), vp(so))
    _check(ctx, st, "transec_shifted_column", allow=(ENOCONV, EBREAKDOWN))
    return t, tm, it, so


def transec_shifted_columns(ctx, energies, ik, cols):
    """Columns at a window of energies by the multi-shift engine; returns
    (t, t_minus, iters, status) host arrays of shape (nitems, ne)."""
    e = np.ascontiguousarray(energies, np.float64)
    k = np.ascontiguousarray(ik, np.int32)
    c = np.ascontiguousarray(cols, np.int64)
    ne, n = e.size, k.size
    if c.size != n:
        raise ValueError("ik and cols differ in length")
    t = np.zeros((n, ne))
    tm = np.zeros((n, ne))
    it = np.zeros((n, ne), np.int32)
    so = np.zeros((n, ne), np.int32)
    vp = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    st = load().transec_shifted_columns(ctx, ne, vp(e), n, vp(k), vp(c), vp(t), vp(tm), vp(it), vp(so))
    _check(ctx, st, "transec_shifted_columns", allow=(ENOCONV, EBREAKDOWN))
    return t, tm, it, so


def transec_transmission_sketch(ctx, energies, ik, s_left=16, s_right=32, seed=0):
    """Full-trace T(E, k) and T(E, -k) by the two-sided sketch; returns
    (T, T_minus, rank, status, iters, miss) host arrays of shape (len(ik), ne)."""
    e = np.ascontiguousarray(energies, np.float64)
    k = np.ascontiguousarray(ik, np.int32)
    ne, nr = e.size, k.size
    T = np.zeros((nr, ne))
    Tm = np.zeros((nr, ne))
    rk = np.zeros((nr, ne), np.int32)
    so = np.zeros((nr, ne), np.int32)
    it = np.zeros((nr, ne), np.int32)
    ms = np.zeros((nr, ne))
    vp = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    st = load().transec_transmission_sketch(ctx, ne, vp(e), nr, vp(k), int(s_left), int(s_right), int(seed),
                                            vp(T), vp(Tm), vp(rk), vp(so), vp(it), vp(ms))
    _check(ctx, st, "transec_transmission_sketch", allow=(ENOCONV, EBREAKDOWN))
    return T, Tm, rk, so, it, ms


def transec_sweep_stats(ctx) -> dict:
    v = [C.c_longlong(), C.c_longlong(), C.c_double(), C.c_longlong(), C.c_double(), C.c_longlong(),
         C.c_double(), C.c_longlong(), C.c_double(), C.c_longlong(), C.c_double(), C.c_longlong(),
         C.c_longlong()]
    _check(ctx, load().transec_sweep_stats(ctx, *[C.byref(x) for x in v]), "transec_sweep_stats")
    keys = ("iters", "shift_points", "stencil_ms", "stencil_launches", "shift_ms", "shift_launches",
            "stencil_df_ms", "stencil_df_launches", "shift_df_ms", "shift_df_launches", "reduce_ms",
            "fp64_redone", "guard_redone")
    return {k: x.value for k, x in zip(keys, v)}
