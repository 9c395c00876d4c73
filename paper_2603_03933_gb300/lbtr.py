"""Python binding of the C ABI in include/lbtr.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but
check tensor properties, pass device pointers, sizes and the CUDA stream, and
translate the returned status into an exception.  All arithmetic runs in the CUDA
library liblbtr.so; there is no CPU fallback: if the library is missing or cannot
be loaded, every call raises.

Tensors: fields are contiguous CUDA tensors of N = M^d elements (any shape with that
many elements, row-major with x fastest), float64 for LB_FP64 contexts and float32 for
LB_MIXED contexts (lb_imex_tr_solve always takes float64).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

LB_FP64, LB_MIXED = 0, 1
STATUS = {0: "LB_OK", 1: "LB_ERR_INVALID_ARG", 2: "LB_ERR_NOT_ZERO_MEAN", 3: "LB_ERR_NONFINITE",
          4: "LB_ERR_NOCONV", 5: "LB_ERR_TIMEOUT", 6: "LB_ERR_CUDA", 7: "LB_ERR_OOM",
          8: "LB_ERR_UNSUPPORTED"}
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblbtr.so")


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lb_problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("box", ctypes.c_double * 3),
                ("xi", ctypes.c_double), ("tau", ctypes.c_double), ("gamma", ctypes.c_double)]


class lb_sub_opts(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("eps_sub", ctypes.c_double), ("rel_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int)]


class lb_sub_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("residual", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("dnorm", ctypes.c_double), ("model_value", ctypes.c_double),
                ("newton_steps", ctypes.c_longlong), ("rel_residual", ctypes.c_double), ("stalled", ctypes.c_int)]


class lb_eig_opts(ctypes.Structure):
    _fields_ = [("max_steps", ctypes.c_int), ("tol", ctypes.c_double), ("sigma", ctypes.c_double),
                ("check_every", ctypes.c_int), ("seed", ctypes.c_uint64)]


class lb_eig_info(ctypes.Structure):
    _fields_ = [("lambda_min", ctypes.c_double), ("kappa_min", ctypes.c_double), ("residual", ctypes.c_double),
                ("steps", ctypes.c_int), ("converged", ctypes.c_int)]


class lb_tr_opts(ctypes.Structure):
    _fields_ = [("gamma_c", ctypes.c_double), ("gamma_e", ctypes.c_double), ("gamma_lam", ctypes.c_double),
                ("theta", ctypes.c_double), ("mu_lo", ctypes.c_double), ("mu_hi", ctypes.c_double),
                ("mu0", ctypes.c_double), ("r0", ctypes.c_double), ("nu0", ctypes.c_double),
                ("eps", ctypes.c_double), ("max_outer", ctypes.c_int), ("second_order", ctypes.c_int),
                ("tol2", ctypes.c_double), ("sub", lb_sub_opts), ("eig", lb_eig_opts),
                ("pcg_max_iter", ctypes.c_int), ("pcg_rtol", ctypes.c_double), ("hard_tol", ctypes.c_double),
                ("checkpoint_path", ctypes.c_char_p), ("checkpoint_every", ctypes.c_int), ("resume", ctypes.c_int)]


class lb_tr_info(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int), ("inner", ctypes.c_longlong), ("accepted", ctypes.c_int),
                ("contracted", ctypes.c_int), ("shrunk", ctypes.c_int), ("energy", ctypes.c_double),
                ("gmax", ctypes.c_double), ("lambda_min", ctypes.c_double), ("status", ctypes.c_int),
                ("randomized", ctypes.c_int), ("g1_min", ctypes.c_double), ("sub_stalled", ctypes.c_int),
                ("sub_capped", ctypes.c_int), ("sub_worst_rel_res", ctypes.c_double)]


class lb_batch_tuning(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("strategy", ctypes.c_int * 12), ("min_blocks", ctypes.c_int * 12),
                ("ctas_per_sm", ctypes.c_int * 12), ("group", ctypes.c_int * 12),
                ("us", ctypes.c_double * 12), ("chosen", ctypes.c_int)]


class lb_sis_opts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("eps", ctypes.c_double), ("max_steps", ctypes.c_int),
                ("check_every", ctypes.c_int)]


class lb_sis_info(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("energy", ctypes.c_double), ("gmax", ctypes.c_double),
                ("status", ctypes.c_int)]


# (name, restype, argtypes) of every exported entry point declared in include/lbtr.h
_VP, _D, _DP = ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
SIGNATURES = [
    ("lb_create", ctypes.c_int, [ctypes.POINTER(lb_problem), ctypes.c_int, ctypes.POINTER(_VP)]),
    ("lb_destroy", ctypes.c_int, [_VP]),
    ("lb_last_error", ctypes.c_char_p, [_VP]),
    ("lb_workspace_bytes", ctypes.c_size_t, [_VP]),
    ("lb_set_params", ctypes.c_int, [_VP, _D, _D, _D]),
    ("lb_energy_grad", ctypes.c_int, [_VP, _VP, _DP, _VP, _DP, _VP]),
    ("lb_energy_derivs", ctypes.c_int, [_VP, _VP, _DP, _VP, _VP]),
    ("lb_hessvec", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    ("lb_default_sub_opts", None, [ctypes.POINTER(lb_sub_opts)]),
    ("lb_tr_subproblem", ctypes.c_int, [_VP, _VP, _VP, _D, _VP, ctypes.POINTER(lb_sub_opts), _VP,
                                        ctypes.POINTER(lb_sub_info), _VP]),
    ("lb_default_eig_opts", None, [ctypes.POINTER(lb_eig_opts)]),
    ("lb_lambda_min", ctypes.c_int, [_VP, _VP, ctypes.POINTER(lb_eig_opts), _VP,
                                     ctypes.POINTER(lb_eig_info), _VP]),
    ("lb_default_tr_opts", None, [ctypes.POINTER(lb_tr_opts)]),
    ("lb_imex_tr_solve", ctypes.c_int, [_VP, _VP, ctypes.POINTER(lb_tr_opts), ctypes.POINTER(lb_tr_info), _VP]),
    ("lb_default_sis_opts", None, [ctypes.POINTER(lb_sis_opts)]),
    ("lb_sis_solve", ctypes.c_int, [_VP, _VP, ctypes.POINTER(lb_sis_opts), ctypes.POINTER(lb_sis_info), _VP]),
    ("lb_profile_enable", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lb_profile_read", ctypes.c_int, [_VP, ctypes.c_int, _DP, ctypes.POINTER(ctypes.c_longlong), _DP]),
    ("lb_set_barrier_budget", ctypes.c_int, [_VP, ctypes.c_longlong]),
    ("lb_hessvec_host", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    ("lb_set_persistent_subproblem", ctypes.c_int, [_VP, ctypes.c_int]),
    ("lb_persistent_subproblem_available", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    ("lb_measure_fp64_rate", ctypes.c_int, [_DP, _VP]),
    ("lb_hessvec_noalloc", ctypes.c_int, [ctypes.POINTER(lb_problem), ctypes.c_int, _VP, _VP, _VP, _VP]),
    ("lb_batch_create", ctypes.c_int, [ctypes.POINTER(lb_problem), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)]),
    ("lb_batch_destroy", None, [_VP]),
    ("lb_batch_last_error", ctypes.c_char_p, [_VP]),
    ("lb_batch_size", ctypes.c_int, [_VP]),
    ("lb_batch_hessvec", ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    ("lb_batch_set_launch", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("lb_batch_tune", ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int,
                                     ctypes.POINTER(lb_batch_tuning), _VP]),
    ("lb_batch_tr_solve", ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(lb_tr_opts),
                                         ctypes.POINTER(lb_tr_info), ctypes.c_int, _VP]),
]
KERNEL_CLASSES = ["xfwd", "xinv", "xmid", "col_y", "col_inner", "secular", "reduce"]

_lib = None


def load(path: str | None = None):
    """Load liblbtr.so (built in-tree by paper_2603_03933_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -m paper_2603_03933_gb300.build`)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(ctx, status: int, where: str):
    if status != 0:
        msg = load().lb_last_error(ctx.handle if ctx is not None else None)
        raise LBError(status, f"{where}: {msg.decode() if msg else ''}")


@dataclass
class Context:
    """An lb_ctx* with the problem it was created for."""

    handle: ctypes.c_void_p
    dim: int
    n: int
    precision: int

    @property
    def npoints(self) -> int:
        return self.n ** self.dim

    @property
    def dtype(self):
        torch = _torch()
        return torch.float64 if self.precision == LB_FP64 else torch.float32

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.lb_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def _ptr(ctx: Context, t, name: str, dtype=None):
    if t is None:
        return None
    torch = _torch()
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    want = dtype if dtype is not None else ctx.dtype
    if t.dtype != want:
        raise TypeError(f"{name} must be {want}, got {t.dtype}")
    if t.numel() != ctx.npoints:
        raise ValueError(f"{name} must have {ctx.npoints} elements, got {t.numel()}")
    del torch
    return ctypes.c_void_p(t.data_ptr())


def lb_create(dim: int, n: int, box, xi: float, tau: float, gamma: float, precision: int = LB_FP64) -> Context:
    """Create a context (C: lb_create).  box: lengths (L_x, L_y[, L_z])."""
    lib = load()
    box = list(box) + [1.0] * (3 - len(box))
    prob = lb_problem(dim, n, (ctypes.c_double * 3)(*box[:3]), xi, tau, gamma)
    h = ctypes.c_void_p()
    st = lib.lb_create(ctypes.byref(prob), precision, ctypes.byref(h))
    if st != 0:
        raise LBError(st, "lb_create")
    return Context(h, dim, n, precision)


def lb_create_from_array_box(shape, box_per_axis, xi, tau, gamma, precision=LB_FP64) -> Context:
    """Create from a numpy-style shape ([y][x] or [z][y][x]) and box lengths in array axis order."""
    dim = len(shape)
    if len(set(shape)) != 1:
        raise ValueError("grids must have the same number of points on every axis")
    box_xyz = list(box_per_axis)[::-1]
    return lb_create(dim, int(shape[0]), box_xyz, xi, tau, gamma, precision)


def lb_destroy(ctx: Context):
    if ctx.handle:
        load().lb_destroy(ctx.handle)
        ctx.handle = None


def lb_set_params(ctx: Context, xi: float, tau: float, gamma: float):
    _check(ctx, load().lb_set_params(ctx.handle, xi, tau, gamma), "lb_set_params")


def lb_workspace_bytes(ctx: Context) -> int:
    return int(load().lb_workspace_bytes(ctx.handle))


def lb_energy_grad(ctx: Context, phi, grad=None, stream=None):
    """(E, max|g|) with g written into `grad` when given (C: lb_energy_grad)."""
    e = ctypes.c_double()
    gm = ctypes.c_double(float("nan"))
    st = load().lb_energy_grad(ctx.handle, _ptr(ctx, phi, "phi"), ctypes.byref(e), _ptr(ctx, grad, "grad"),
                               ctypes.byref(gm) if grad is not None else None, _stream(stream))
    _check(ctx, st, "lb_energy_grad")
    return e.value, (gm.value if grad is not None else None)


def lb_energy_derivs(ctx: Context, phi, grad=None, stream=None) -> dict:
    """E and dE/dtau, dE/dgamma, dE/dL (x, y, z order) at fixed grid values, g into `grad`
    when given (C: lb_energy_derivs)."""
    out = (ctypes.c_double * 6)()
    st = load().lb_energy_derivs(ctx.handle, _ptr(ctx, phi, "phi"), out, _ptr(ctx, grad, "grad"), _stream(stream))
    _check(ctx, st, "lb_energy_derivs")
    return {"energy": out[0], "dtau": out[1], "dgamma": out[2], "dL_xyz": [out[3], out[4], out[5]][:ctx.dim]}


def lb_hessvec(ctx: Context, phi, v, hv, stream=None):
    """hv = H v (C: lb_hessvec); asynchronous on the stream."""
    st = load().lb_hessvec(ctx.handle, _ptr(ctx, phi, "phi"), _ptr(ctx, v, "v"), _ptr(ctx, hv, "hv"),
                           _stream(stream))
    _check(ctx, st, "lb_hessvec")
    return hv


def _host_ptr(ctx: Context, t, name: str):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a CPU tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype != ctx.dtype:
        raise TypeError(f"{name} must be {ctx.dtype}, got {t.dtype}")
    if t.numel() != ctx.npoints:
        raise ValueError(f"{name} must have {ctx.npoints} elements, got {t.numel()}")
    return t.data_ptr()


def lb_hessvec_host(ctx: Context, phi, vs, hvs, stream=None):
    """hvs[i] = H vs[i] for CPU tensors (C: lb_hessvec_host): the copies in and out overlap the
    products when the tensors are page-locked (tensor.pin_memory()); returns when done."""
    if len(vs) != len(hvs):
        raise ValueError("vs and hvs differ in length")
    n = len(vs)
    pv = (_VP * max(n, 1))(*[_host_ptr(ctx, v, "v") for v in vs])
    ph = (_VP * max(n, 1))(*[_host_ptr(ctx, h, "hv") for h in hvs])
    st = load().lb_hessvec_host(ctx.handle, ctypes.c_void_p(_host_ptr(ctx, phi, "phi")), n, pv, ph, _stream(stream))
    _check(ctx, st, "lb_hessvec_host")
    return hvs


def default_sub_opts() -> lb_sub_opts:
    o = lb_sub_opts()
    load().lb_default_sub_opts(ctypes.byref(o))
    return o


def lb_tr_subproblem(ctx: Context, phi, g, r: float, d, d0=None, opts: lb_sub_opts | None = None,
                     stream=None, raise_on_noconv: bool = True) -> dict:
    """Algorithm 3 (C: lb_tr_subproblem); returns the info struct as a dict."""
    o = opts if opts is not None else default_sub_opts()
    info = lb_sub_info()
    st = load().lb_tr_subproblem(ctx.handle, _ptr(ctx, phi, "phi"), _ptr(ctx, g, "g"), float(r),
                                 _ptr(ctx, d0, "d0"), ctypes.byref(o), _ptr(ctx, d, "d"), ctypes.byref(info),
                                 _stream(stream))
    if not (st == 4 and not raise_on_noconv):
        _check(ctx, st, "lb_tr_subproblem")
    return {"iterations": info.iterations, "converged": bool(info.converged), "residual": info.residual,
            "lambda": info.lambda_, "dnorm": info.dnorm, "model_value": info.model_value,
            "newton_steps": info.newton_steps, "rel_residual": info.rel_residual,
            "stalled": bool(info.stalled), "status": st}


def default_eig_opts() -> lb_eig_opts:
    o = lb_eig_opts()
    load().lb_default_eig_opts(ctypes.byref(o))
    return o


def lb_lambda_min(ctx: Context, phi, vec=None, opts: lb_eig_opts | None = None, stream=None,
                  raise_on_noconv: bool = True) -> dict:
    """Smallest Hessian eigenvalue estimate (C: lb_lambda_min)."""
    o = opts if opts is not None else default_eig_opts()
    info = lb_eig_info()
    st = load().lb_lambda_min(ctx.handle, _ptr(ctx, phi, "phi"), ctypes.byref(o), _ptr(ctx, vec, "vec"),
                              ctypes.byref(info), _stream(stream))
    if not (st == 4 and not raise_on_noconv):
        _check(ctx, st, "lb_lambda_min")
    return {"lambda_min": info.lambda_min, "kappa_min": info.kappa_min, "residual": info.residual,
            "steps": info.steps, "converged": bool(info.converged), "status": st}


def default_tr_opts() -> lb_tr_opts:
    o = lb_tr_opts()
    load().lb_default_tr_opts(ctypes.byref(o))
    return o


def lb_imex_tr_solve(ctx: Context, phi64, opts: lb_tr_opts | None = None, stream=None,
                     raise_on_noconv: bool = True) -> dict:
    """IMEX-TR (C: lb_imex_tr_solve); phi64 (float64 CUDA tensor) is updated in place."""
    torch = _torch()
    o = opts if opts is not None else default_tr_opts()
    info = lb_tr_info()
    st = load().lb_imex_tr_solve(ctx.handle, _ptr(ctx, phi64, "phi", torch.float64), ctypes.byref(o),
                                 ctypes.byref(info), _stream(stream))
    if not (st == 4 and not raise_on_noconv):
        _check(ctx, st, "lb_imex_tr_solve")
    return {"outer": info.outer, "inner": info.inner, "accepted": info.accepted, "contracted": info.contracted,
            "shrunk": info.shrunk, "energy": info.energy, "gmax": info.gmax,
            "lambda_min": info.lambda_min if not math.isnan(info.lambda_min) else None, "status": st,
            "randomized": info.randomized, "g1_min": info.g1_min if not math.isnan(info.g1_min) else None,
            "sub_stalled": info.sub_stalled, "sub_capped": info.sub_capped,
            "sub_worst_rel_res": info.sub_worst_rel_res}


def default_sis_opts() -> lb_sis_opts:
    o = lb_sis_opts()
    load().lb_default_sis_opts(ctypes.byref(o))
    return o


def lb_sis_solve(ctx: Context, phi64, opts: lb_sis_opts | None = None, stream=None,
                 raise_on_noconv: bool = True) -> dict:
    """Semi-implicit gradient flow (C: lb_sis_solve); phi64 (float64 CUDA tensor) is updated in place."""
    torch = _torch()
    o = opts if opts is not None else default_sis_opts()
    info = lb_sis_info()
    st = load().lb_sis_solve(ctx.handle, _ptr(ctx, phi64, "phi", torch.float64), ctypes.byref(o),
                             ctypes.byref(info), _stream(stream))
    if not (st == 4 and not raise_on_noconv):
        _check(ctx, st, "lb_sis_solve")
    return {"steps": info.steps, "energy": info.energy, "gmax": info.gmax, "status": st}


def lb_set_barrier_budget(ctx: Context, cycles: int):
    _check(ctx, load().lb_set_barrier_budget(ctx.handle, int(cycles)), "lb_set_barrier_budget")


def lb_set_persistent_subproblem(ctx: Context, enable: bool):
    """One-launch inner loop of the subproblem on 128^3 mixed grids (default on)."""
    _check(ctx, load().lb_set_persistent_subproblem(ctx.handle, 1 if enable else 0), "lb_set_persistent_subproblem")


def lb_persistent_subproblem_available(ctx: Context) -> bool:
    out = ctypes.c_int()
    _check(ctx, load().lb_persistent_subproblem_available(ctx.handle, ctypes.byref(out)),
           "lb_persistent_subproblem_available")
    return bool(out.value)


def lb_measure_fp64_rate(stream=None) -> float:
    """FP64 FMA throughput of the current device in TFLOP/s (C: lb_measure_fp64_rate)."""
    out = ctypes.c_double()
    st = load().lb_measure_fp64_rate(ctypes.byref(out), _stream(stream))
    if st != 0:
        raise LBError(st, "lb_measure_fp64_rate")
    return out.value


def lb_profile_enable(ctx: Context, enable: bool = True):
    """Start (and reset) or stop per-kernel-class event timing (C: lb_profile_enable)."""
    _check(ctx, load().lb_profile_enable(ctx.handle, 1 if enable else 0), "lb_profile_enable")


def lb_profile_read(ctx: Context) -> dict:
    """{class: (total_ms, launches, algorithmic_bytes)} for every kernel class (C: lb_profile_read)."""
    out = {}
    for k, name in enumerate(KERNEL_CLASSES):
        ms, n, b = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        _check(ctx, load().lb_profile_read(ctx.handle, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)),
               "lb_profile_read")
        out[name] = (ms.value, n.value, b.value)
    return out


def lb_hessvec_noalloc(dim: int, n: int, box, xi: float, tau: float, gamma: float, precision: int,
                       phi, v, hv, stream=None):
    """hv = H v without a context or any device allocation (C: lb_hessvec_noalloc).

    For callers that cannot allocate device memory.  box: (L_x, L_y[, L_z]).  Scratch is a
    fixed array inside the library (N <= 2^18 points); concurrent calls race."""
    torch = _torch()
    want = torch.float64 if precision == LB_FP64 else torch.float32
    npts = n ** dim
    for name, t in (("phi", phi), ("v", v), ("hv", hv)):
        if not t.is_cuda or not t.is_contiguous() or t.dtype != want or t.numel() != npts:
            raise ValueError(f"{name} must be a contiguous CUDA {want} tensor of {npts} elements")
    box = list(box) + [1.0] * (3 - len(box))
    prob = lb_problem(dim, n, (ctypes.c_double * 3)(*box[:3]), xi, tau, gamma)
    st = load().lb_hessvec_noalloc(ctypes.byref(prob), precision, ctypes.c_void_p(phi.data_ptr()),
                                   ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(hv.data_ptr()), _stream(stream))
    if st != 0:
        raise LBError(st, "lb_hessvec_noalloc")
    return hv


class Batch:
    """An lb_batch* (independent problems whose products run as one CUDA graph)."""

    def __init__(self, handle, contexts_meta, precision):
        self.handle = handle
        self.meta = contexts_meta          # (dim, n) per problem
        self.precision = precision

    def __len__(self):
        return len(self.meta)

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.lb_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def lb_batch_create(problems, precision: int = LB_FP64) -> Batch:
    """problems: sequence of (dim, n, box_xyz, xi, tau, gamma) (C: lb_batch_create)."""
    lib = load()
    arr = (lb_problem * len(problems))()
    meta = []
    for i, (dim, n, box, xi, tau, gamma) in enumerate(problems):
        box = list(box) + [1.0] * (3 - len(box))
        arr[i] = lb_problem(dim, n, (ctypes.c_double * 3)(*box[:3]), xi, tau, gamma)
        meta.append((dim, n))
    h = ctypes.c_void_p()
    st = lib.lb_batch_create(arr, len(problems), precision, ctypes.byref(h))
    if st != 0:
        raise LBError(st, "lb_batch_create")
    return Batch(h, meta, precision)


def _batch_ptrs(batch: Batch, phis, vs, hvs):
    torch = _torch()
    want = torch.float64 if batch.precision == LB_FP64 else torch.float32
    n = len(batch)
    if not (len(phis) == len(vs) == len(hvs) == n):
        raise ValueError("one phi, v and hv per problem")
    ptrs = []
    for group in (phis, vs, hvs):
        arr = (_VP * n)()
        for i, t in enumerate(group):
            dim, m = batch.meta[i]
            if t.dtype != want or not t.is_cuda or not t.is_contiguous() or t.numel() != m ** dim:
                raise ValueError(f"field {i}: need a contiguous {want} CUDA tensor of {m ** dim} values")
            arr[i] = t.data_ptr()
        ptrs.append(arr)
    return ptrs


class BatchFields:
    """The device pointers of a batch call, marshalled once (phis, vs, hvs keep their
    tensors alive); pass it to lb_batch_hessvec in place of the three lists."""

    def __init__(self, batch: Batch, phis, vs, hvs):
        self.tensors = (list(phis), list(vs), list(hvs))
        self.ptrs = _batch_ptrs(batch, phis, vs, hvs)


def lb_batch_tune(batch: Batch, phis, vs, hvs, replays: int = 10, stream=None) -> dict:
    """Time the persistent sweep launch's candidate configurations and keep the fastest
    (C: lb_batch_tune); returns the table with its measurements."""
    ptrs = _batch_ptrs(batch, phis, vs, hvs)
    t = lb_batch_tuning()
    st = load().lb_batch_tune(batch.handle, ptrs[0], ptrs[1], ptrs[2], int(replays), ctypes.byref(t), _stream(stream))
    if st != 0:
        msg = load().lb_batch_last_error(batch.handle)
        raise LBError(st, "lb_batch_tune: " + (msg.decode() if msg else ""))
    return {"candidates": [{"strategy": "persistent" if t.strategy[k] else "grouped", "min_blocks": t.min_blocks[k],
                            "ctas_per_sm": t.ctas_per_sm[k], "row_blocks_per_task": t.group[k], "us": t.us[k]}
                           for k in range(t.count)], "chosen": t.chosen}


def lb_batch_set_launch(batch: Batch, persistent: bool, min_blocks: int = 4, ctas_per_sm: int = 0, group: int = 1):
    """Choose the batch's launch strategy for its 2D problems (C: lb_batch_set_launch)."""
    st = load().lb_batch_set_launch(batch.handle, 1 if persistent else 0, int(min_blocks), int(ctas_per_sm), int(group))
    if st != 0:
        msg = load().lb_batch_last_error(batch.handle)
        raise LBError(st, "lb_batch_set_launch: " + (msg.decode() if msg else ""))


def lb_batch_hessvec(batch: Batch, phis, vs=None, hvs=None, stream=None):
    """hvs[i] = H_i vs[i] for every problem, as one CUDA graph (C: lb_batch_hessvec).
    `phis` may be a BatchFields (then vs and hvs are omitted): no per-call marshalling."""
    if isinstance(phis, BatchFields):
        ptrs = phis.ptrs
        hvs = phis.tensors[2]
    else:
        ptrs = _batch_ptrs(batch, phis, vs, hvs)
    st = load().lb_batch_hessvec(batch.handle, ptrs[0], ptrs[1], ptrs[2], _stream(stream))
    if st != 0:
        msg = load().lb_batch_last_error(batch.handle)
        raise LBError(st, "lb_batch_hessvec: " + (msg.decode() if msg else ""))
    return hvs


def _tr_info_dict(info: lb_tr_info) -> dict:
    return {"outer": info.outer, "inner": info.inner, "accepted": info.accepted, "contracted": info.contracted,
            "shrunk": info.shrunk, "energy": info.energy, "gmax": info.gmax,
            "lambda_min": info.lambda_min if not math.isnan(info.lambda_min) else None, "status": info.status,
            "randomized": info.randomized, "g1_min": info.g1_min if not math.isnan(info.g1_min) else None,
            "sub_stalled": info.sub_stalled, "sub_capped": info.sub_capped,
            "sub_worst_rel_res": info.sub_worst_rel_res}


def lb_batch_tr_solve(batch: Batch, phis, opts: lb_tr_opts | None = None, nthreads: int = 0, stream=None,
                      raise_on_error: bool = True) -> list:
    """IMEX-TR for every problem on a pool of host threads (C: lb_batch_tr_solve); each
    phis[i] (float64 CUDA tensor) is updated in place.  Returns one info dict per problem."""
    torch = _torch()
    n = len(batch)
    if len(phis) != n:
        raise ValueError("one phi per problem")
    arr = (_VP * n)()
    for i, t in enumerate(phis):
        dim, m = batch.meta[i]
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != m ** dim:
            raise ValueError(f"field {i}: need a contiguous float64 CUDA tensor of {m ** dim} values")
        arr[i] = t.data_ptr()
    o = opts if opts is not None else default_tr_opts()
    infos = (lb_tr_info * n)()
    st = load().lb_batch_tr_solve(batch.handle, arr, ctypes.byref(o), infos, int(nthreads), _stream(stream))
    if st != 0 and raise_on_error:
        msg = load().lb_batch_last_error(batch.handle)
        raise LBError(st, "lb_batch_tr_solve: " + (msg.decode() if msg else ""))
    return [_tr_info_dict(infos[i]) for i in range(n)]

