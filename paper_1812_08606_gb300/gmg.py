"""Thin ctypes binding of libgmg (include/gmg.h), same names as the C ABI.

Only argument marshalling lives here: tensors are passed as raw device
pointers and the CUDA stream as a ``cudaStream_t``; every step of the solve
runs in the library's CUDA kernels.  PyTorch supplies device memory and
streams.  If libgmg.so is missing or cannot be loaded, every call raises:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

GMG_MAX_HISTORY = 256

GMG_OK = 0
GMG_ERR_ARG = 1
GMG_ERR_CUDA = 2
GMG_ERR_ALLOC = 3
GMG_ERR_NOT_CONVERGED = 4
GMG_ERR_BREAKDOWN = 5
GMG_ERR_NONFINITE = 6

GMG_PREC_FP64 = 0
GMG_PREC_MIXED = 1
GMG_PROLONG_TRILINEAR = 0
GMG_PROLONG_CONSTANT = 1
GMG_PROLONG_OPDEP = 2
GMG_COARSEN_MEAN = 0
GMG_COARSEN_SERIES = 1
GMG_PC_SGS = 0
GMG_PC_JACOBI = 1
GMG_PC_IDENTITY = 2
GMG_ORTH_CGS2 = 0
GMG_ORTH_MGS = 1
GMG_OUTER_FP64 = 0
GMG_OUTER_DOUBLE_FLOAT = 1
GMG_CYCLE_V = 0
GMG_CYCLE_FMG = 1
GMG_CYCLE_AUTO = 2
GMG_KRYLOV_FGMRES = 0
GMG_KRYLOV_GMRES = 1
GMG_KRYLOV_CG = 2
GMG_KRYLOV_FCG = 3
GMG_KRYLOV_CGS = 4
GMG_KRYLOV_BICGSTAB = 5
KRYLOV_NAMES = {"fgmres": 0, "gmres": 1, "cg": 2, "fcg": 3, "cgs": 4, "bicgstab": 5}

# e / eps0 in V cm (densities in cm^-3, mobilities in cm^2/(V s), lengths in cm)
E_OVER_EPS0_CM = 1.602176634e-19 / 8.8541878128e-14


class gmg_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("phi_bottom", ctypes.c_double), ("phi_top", ctypes.c_double),
        ("coarse_min", ctypes.c_int), ("cheb_steps", ctypes.c_int), ("restart", ctypes.c_int),
        ("max_iters", ctypes.c_int), ("rtol", ctypes.c_double), ("eig_steps", ctypes.c_int),
        ("eig_hi", ctypes.c_double), ("eig_lo", ctypes.c_double), ("precision", ctypes.c_int),
        ("prolongation", ctypes.c_int), ("smoother_pc", ctypes.c_int), ("orthogonalization", ctypes.c_int),
        ("outer_arith", ctypes.c_int), ("smoother_kernel", ctypes.c_int), ("cycle", ctypes.c_int),
        ("coarsening", ctypes.c_int),
    ]


class gmg_solve_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
        ("true_rel_residual", ctypes.c_double), ("bnorm", ctypes.c_double), ("n_history", ctypes.c_int),
        ("res_history", ctypes.c_double * GMG_MAX_HISTORY), ("setup_ms", ctypes.c_float),
        ("solve_ms", ctypes.c_float), ("fmg", ctypes.c_int), ("precond_calls", ctypes.c_int),
    ]

    @property
    def history(self):
        return [self.res_history[i] for i in range(self.n_history)]


class gmg_density_coef(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double), ("mu_e", ctypes.c_double), ("mu_p", ctypes.c_double),
        ("diff_x", ctypes.c_double), ("diff_y", ctypes.c_double), ("diff_z", ctypes.c_double),
        ("e_over_eps0", ctypes.c_double),
    ]


class gmg_transport_coef(ctypes.Structure):
    _fields_ = [
        ("mu_e", ctypes.c_double), ("mu_p", ctypes.c_double), ("diff_x", ctypes.c_double),
        ("diff_y", ctypes.c_double), ("diff_z", ctypes.c_double), ("ion_a", ctypes.c_double),
        ("ion_b", ctypes.c_double), ("pressure", ctypes.c_double),
    ]


class GMGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_LIB = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "gmg_default_params": (None, [ctypes.POINTER(gmg_params), ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "gmg_setup": (ctypes.c_int, [ctypes.POINTER(gmg_params), _P, _P, ctypes.POINTER(_P)]),
    "gmg_update_coefficient": (ctypes.c_int, [_P, _P]),
    "fgmres_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(gmg_solve_info)]),
    "gmg_krylov_solve": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.POINTER(gmg_solve_info)]),
    "apply_operator": (ctypes.c_int, [_P, _P, _P]),
    "assemble_rhs": (ctypes.c_int, [_P, _P, _P]),
    "field_from_potential": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "adjoint_coefficient_grad": (ctypes.c_int, [_P, _P, _P, _P]),
    "gmg_solve_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int,
                                      ctypes.POINTER(gmg_solve_info)]),
    "gmg_solve_host_async": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int,
                                            ctypes.POINTER(gmg_solve_info)]),
    "gmg_host_wait": (ctypes.c_int, [_P]),
    "gmg_set_stream": (ctypes.c_int, [_P, _P]),
    "gmg_destroy": (None, [_P]),
    "gmg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gmg_num_levels": (ctypes.c_int, [_P]),
    "gmg_level_faces": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    "gmg_level_set_bounds": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "gmg_level_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
    "gmg_level_coefficient": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "gmg_apply_preconditioner": (ctypes.c_int, [_P, _P, _P]),
    "gmg_apply_outer": (ctypes.c_int, [_P, _P, _P]),
    "gmg_level_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "gmg_level_smooth": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int]),
    "gmg_level_smoother_pc": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "gmg_level_residual_restrict": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "gmg_level_prolong_add": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "gmg_coarse_solve": (ctypes.c_int, [_P, _P, _P]),
    "gmg_hessenberg_max_real_eig": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "gmg_test_fail_allocation_after": (None, [ctypes.c_int]),
    "gmg_coarse_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(gmg_params), _P, _P, _P, _P]),
    "assemble_coefficient_rhs": (ctypes.c_int, [ctypes.POINTER(gmg_params), _P, _P, ctypes.POINTER(gmg_density_coef),
                                                _P, _P, _P]),
    "transport_stage": (ctypes.c_int, [ctypes.POINTER(gmg_params), _P, _P, _P, _P, _P,
                                       ctypes.POINTER(gmg_transport_coef), ctypes.c_double, _P, _P, _P]),
    "gmg_round_to_f32": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "transport_step": (ctypes.c_int, [ctypes.POINTER(gmg_params), _P, _P, _P, ctypes.POINTER(gmg_transport_coef),
                                      ctypes.c_double, _P, _P, _P, _P, _P, _P]),
    "gmg_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "gmg_profile_reset": (ctypes.c_int, [_P]),
    "gmg_profile_min_bytes": (ctypes.c_int, [_P, ctypes.c_double]),
    "gmg_profile_num_kernels": (ctypes.c_int, []),
    "gmg_profile_get": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
}


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load libgmg.so (building it first if asked).  Raises if unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libgmg.so not built at {path}; run paper_1812_08606_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def gmg_status_string(status: int) -> str:
    return load().gmg_status_string(int(status)).decode()


status_string = gmg_status_string


def _check(status: int, where: str, allow=(GMG_OK,)):
    if status not in allow:
        raise GMGError(status, where)
    return status


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype=torch.float64, numel=None, name="tensor") -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _host(t: torch.Tensor, dtype=torch.float64, numel=None, name="tensor") -> int:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} host tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements")
    return t.data_ptr()


def gmg_default_params(nx: int, ny: int, nz: int, **overrides) -> gmg_params:
    p = gmg_params()
    load().gmg_default_params(ctypes.byref(p), int(nx), int(ny), int(nz))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Context:
    """Owner of one gmg_ctx*; freed by close() or garbage collection."""

    def __init__(self, handle: int, params: gmg_params, stream):
        self.handle = ctypes.c_void_p(handle)
        self.params = params
        self.stream = stream
        self.n = params.nx * params.ny * params.nz
        self.shape = (params.nz, params.ny, params.nx)

    def close(self):
        if self.handle is not None and self.handle.value:
            load().gmg_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def level_dtype(self):
        return torch.float32 if self.params.precision == GMG_PREC_MIXED else torch.float64


def gmg_setup(params: gmg_params, a: torch.Tensor, stream=None) -> Context:
    n = params.nx * params.ny * params.nz
    out = ctypes.c_void_p()
    st = load().gmg_setup(ctypes.byref(params), _dev(a, numel=n, name="a"), _stream_ptr(stream), ctypes.byref(out))
    _check(st, "gmg_setup")
    return Context(out.value, params, stream)


def gmg_update_coefficient(ctx: Context, a: torch.Tensor):
    _check(load().gmg_update_coefficient(ctx.handle, _dev(a, numel=ctx.n, name="a")), "gmg_update_coefficient")


def fgmres_solve(ctx: Context, f: torch.Tensor, phi: torch.Tensor, homogeneous_bc: bool = False) -> gmg_solve_info:
    """Solve in place into phi (initial guess on entry).  Returns the info;
    a solve that hit max_iters returns info.converged == 0 without raising."""
    info = gmg_solve_info()
    st = load().fgmres_solve(ctx.handle, _dev(f, numel=ctx.n, name="f"), _dev(phi, numel=ctx.n, name="phi"),
                             int(bool(homogeneous_bc)), ctypes.byref(info))
    _check(st, "fgmres_solve", allow=(GMG_OK, GMG_ERR_NOT_CONVERGED))
    return info


def gmg_krylov_solve(ctx: Context, method, f: torch.Tensor, phi: torch.Tensor,
                     homogeneous_bc: bool = False) -> gmg_solve_info:
    """Like fgmres_solve with the Krylov method ``method`` (a GMG_KRYLOV_*
    value or one of "fgmres", "gmres", "cg", "fcg", "cgs", "bicgstab")."""
    m = KRYLOV_NAMES[method] if isinstance(method, str) else int(method)
    info = gmg_solve_info()
    st = load().gmg_krylov_solve(ctx.handle, m, _dev(f, numel=ctx.n, name="f"), _dev(phi, numel=ctx.n, name="phi"),
                                 int(bool(homogeneous_bc)), ctypes.byref(info))
    _check(st, "gmg_krylov_solve", allow=(GMG_OK, GMG_ERR_NOT_CONVERGED))
    return info


def apply_operator(ctx: Context, x: torch.Tensor, y: torch.Tensor):
    _check(load().apply_operator(ctx.handle, _dev(x, numel=ctx.n, name="x"), _dev(y, numel=ctx.n, name="y")),
           "apply_operator")


def assemble_rhs(ctx: Context, f: torch.Tensor, b: torch.Tensor):
    _check(load().assemble_rhs(ctx.handle, _dev(f, numel=ctx.n, name="f"), _dev(b, numel=ctx.n, name="b")),
           "assemble_rhs")


def field_from_potential(ctx: Context, phi: torch.Tensor, ex: torch.Tensor, ey: torch.Tensor, ez: torch.Tensor):
    dt = ex.dtype
    if dt not in (torch.float32, torch.float64) or ey.dtype != dt or ez.dtype != dt:
        raise ValueError("ex, ey, ez must all be float32 or all float64")
    _check(load().field_from_potential(ctx.handle, _dev(phi, numel=ctx.n, name="phi"),
                                       _dev(ex, dt, ctx.n, "ex"), _dev(ey, dt, ctx.n, "ey"),
                                       _dev(ez, dt, ctx.n, "ez"), int(dt == torch.float32)),
           "field_from_potential")


def adjoint_coefficient_grad(ctx: Context, phi: torch.Tensor, lam: torch.Tensor, dlda: torch.Tensor):
    _check(load().adjoint_coefficient_grad(ctx.handle, _dev(phi, numel=ctx.n, name="phi"),
                                           _dev(lam, numel=ctx.n, name="lambda"),
                                           _dev(dlda, numel=ctx.n, name="dlda")), "adjoint_coefficient_grad")


def _solve_host(fn: str, ctx: Context, a_host, f_host, phi_host, phi0_host, ex_host, ey_host, ez_host):
    info = gmg_solve_info()
    a_ptr = _host(a_host, numel=ctx.n, name="a") if a_host is not None else None
    x0_ptr = _host(phi0_host, numel=ctx.n, name="phi0") if phi0_host is not None else None
    fp32 = 0
    eptrs = [None, None, None]
    if ex_host is not None:
        fp32 = int(ex_host.dtype == torch.float32)
        dt = torch.float32 if fp32 else torch.float64
        eptrs = [_host(t, dt, ctx.n, nm) for t, nm in ((ex_host, "ex"), (ey_host, "ey"), (ez_host, "ez"))]
    st = getattr(load(), fn)(ctx.handle, a_ptr, _host(f_host, numel=ctx.n, name="f"), x0_ptr,
                             _host(phi_host, numel=ctx.n, name="phi"), eptrs[0], eptrs[1], eptrs[2], fp32,
                             ctypes.byref(info))
    _check(st, fn, allow=(GMG_OK, GMG_ERR_NOT_CONVERGED))
    return info


def gmg_solve_host(ctx: Context, a_host, f_host, phi_host, phi0_host=None, ex_host=None, ey_host=None,
                   ez_host=None):
    """End-to-end solve on host tensors (pinned for full bandwidth): the
    result lands in phi_host; phi0_host=None means a zero initial guess."""
    return _solve_host("gmg_solve_host", ctx, a_host, f_host, phi_host, phi0_host, ex_host, ey_host, ez_host)


def gmg_solve_host_async(ctx: Context, a_host, f_host, phi_host, phi0_host=None, ex_host=None, ey_host=None,
                         ez_host=None):
    """gmg_solve_host, pipelined: returns once the solve is done, with the
    copy-out of phi (and E) held back for the next host-array call (after its
    upload of a) or for gmg_host_wait(ctx), which completes it before the host
    arrays are read."""
    return _solve_host("gmg_solve_host_async", ctx, a_host, f_host, phi_host, phi0_host, ex_host, ey_host, ez_host)


def gmg_host_wait(ctx: Context):
    """Waits for every copy and kernel of the context's host-array solves."""
    _check(load().gmg_host_wait(ctx.handle), "gmg_host_wait")


def gmg_set_stream(ctx: Context, stream):
    _check(load().gmg_set_stream(ctx.handle, _stream_ptr(stream)), "gmg_set_stream")
    ctx.stream = stream


def gmg_destroy(ctx: Context):
    ctx.close()


def gmg_num_levels(ctx: Context) -> int:
    return load().gmg_num_levels(ctx.handle)


def gmg_level_info(ctx: Context, level: int):
    nx, ny, nz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lmax, lmin = ctypes.c_double(), ctypes.c_double()
    _check(load().gmg_level_info(ctx.handle, int(level), ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nz),
                                 ctypes.byref(lmax), ctypes.byref(lmin)), "gmg_level_info")
    return {"shape": (nz.value, ny.value, nx.value), "lam_max": lmax.value, "lam_min": lmin.value}


def gmg_level_faces(ctx: Context, level: int):
    """(kx, ky, kz, ktop) FP64 device tensors: the level's face matrix entries."""
    shape = gmg_level_info(ctx, level)["shape"]
    dev = torch.device("cuda", torch.cuda.current_device())
    kx, ky, kz = (torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(3))
    ktop = torch.empty(shape[1:], dtype=torch.float64, device=dev)
    _check(load().gmg_level_faces(ctx.handle, int(level), kx.data_ptr(), ky.data_ptr(), kz.data_ptr(),
                                  ktop.data_ptr()), "gmg_level_faces")
    return kx, ky, kz, ktop


def gmg_level_set_bounds(ctx: Context, level: int, lam_max: float, lam_min: float):
    _check(load().gmg_level_set_bounds(ctx.handle, int(level), float(lam_max), float(lam_min)),
           "gmg_level_set_bounds")


def _level_n(ctx, level):
    s = gmg_level_info(ctx, level)["shape"]
    return s[0] * s[1] * s[2]


def gmg_level_coefficient(ctx: Context, level: int, out: torch.Tensor):
    _check(load().gmg_level_coefficient(ctx.handle, int(level), _dev(out, numel=_level_n(ctx, level), name="out")),
           "gmg_level_coefficient")


def gmg_apply_preconditioner(ctx: Context, v: torch.Tensor, z: torch.Tensor):
    _check(load().gmg_apply_preconditioner(ctx.handle, _dev(v, numel=ctx.n, name="v"),
                                           _dev(z, numel=ctx.n, name="z")), "gmg_apply_preconditioner")


def gmg_apply_outer(ctx: Context, z: torch.Tensor, w: torch.Tensor):
    _check(load().gmg_apply_outer(ctx.handle, _dev(z, torch.float32, ctx.n, "z"), _dev(w, numel=ctx.n, name="w")),
           "gmg_apply_outer")


def gmg_level_apply(ctx: Context, level: int, x: torch.Tensor, y: torch.Tensor):
    n, dt = _level_n(ctx, level), ctx.level_dtype
    _check(load().gmg_level_apply(ctx.handle, int(level), _dev(x, dt, n, "x"), _dev(y, dt, n, "y")),
           "gmg_level_apply")


def gmg_level_smooth(ctx: Context, level: int, b: torch.Tensor, x: torch.Tensor, x_is_zero: bool):
    n, dt = _level_n(ctx, level), ctx.level_dtype
    _check(load().gmg_level_smooth(ctx.handle, int(level), _dev(b, dt, n, "b"), _dev(x, dt, n, "x"),
                                   int(bool(x_is_zero))), "gmg_level_smooth")


def gmg_level_smoother_pc(ctx: Context, level: int, r: torch.Tensor, z: torch.Tensor):
    n, dt = _level_n(ctx, level), ctx.level_dtype
    _check(load().gmg_level_smoother_pc(ctx.handle, int(level), _dev(r, dt, n, "r"), _dev(z, dt, n, "z")),
           "gmg_level_smoother_pc")


def gmg_level_residual_restrict(ctx: Context, level: int, b: torch.Tensor, x: torch.Tensor, coarse: torch.Tensor):
    n, nc, dt = _level_n(ctx, level), _level_n(ctx, level - 1), ctx.level_dtype
    _check(load().gmg_level_residual_restrict(ctx.handle, int(level), _dev(b, dt, n, "b"), _dev(x, dt, n, "x"),
                                              _dev(coarse, dt, nc, "coarse")), "gmg_level_residual_restrict")


def gmg_level_prolong_add(ctx: Context, level: int, e: torch.Tensor, x: torch.Tensor):
    n, nc, dt = _level_n(ctx, level), _level_n(ctx, level - 1), ctx.level_dtype
    _check(load().gmg_level_prolong_add(ctx.handle, int(level), _dev(e, dt, nc, "e"), _dev(x, dt, n, "x")),
           "gmg_level_prolong_add")


def gmg_coarse_solve(ctx: Context, b: torch.Tensor, x: torch.Tensor):
    n, dt = _level_n(ctx, 0), ctx.level_dtype
    _check(load().gmg_coarse_solve(ctx.handle, _dev(b, dt, n, "b"), _dev(x, dt, n, "x")), "gmg_coarse_solve")


def gmg_hessenberg_max_real_eig(h) -> float:
    """Largest real part of the eigenvalues of a square upper Hessenberg
    matrix (host computation inside the library; needs no GPU)."""
    import numpy as np
    h = np.ascontiguousarray(h, dtype=np.float64)
    m = h.shape[0]
    out = ctypes.c_double()
    _check(load().gmg_hessenberg_max_real_eig(h.ctypes.data_as(ctypes.c_void_p), int(m), ctypes.byref(out)),
           "gmg_hessenberg_max_real_eig")
    return out.value


def gmg_test_fail_allocation_after(n: int):
    load().gmg_test_fail_allocation_after(int(n))


def gmg_profile_enable(ctx: Context, on: bool = True):
    _check(load().gmg_profile_enable(ctx.handle, int(bool(on))), "gmg_profile_enable")


def gmg_profile_min_bytes(ctx: Context, min_bytes: float):
    _check(load().gmg_profile_min_bytes(ctx.handle, float(min_bytes)), "gmg_profile_min_bytes")


def gmg_profile_reset(ctx: Context):
    _check(load().gmg_profile_reset(ctx.handle), "gmg_profile_reset")


def gmg_profile_num_kernels() -> int:
    return load().gmg_profile_num_kernels()


def gmg_profile_get(ctx: Context, k: int) -> dict:
    name = ctypes.c_char_p()
    launches, timed = ctypes.c_longlong(), ctypes.c_longlong()
    ms, nbytes = ctypes.c_double(), ctypes.c_double()
    _check(load().gmg_profile_get(ctx.handle, int(k), ctypes.byref(name), ctypes.byref(launches), ctypes.byref(timed),
                                  ctypes.byref(ms), ctypes.byref(nbytes)), "gmg_profile_get")
    return {"name": name.value.decode(), "launches": launches.value, "timed": timed.value, "ms": ms.value,
            "bytes": nbytes.value}


def profile(ctx: Context) -> list:
    """All kernel classes with at least one launch, sorted by time."""
    rows = [gmg_profile_get(ctx, k) for k in range(gmg_profile_num_kernels())]
    return sorted((r for r in rows if r["launches"]), key=lambda r: -r["ms"])


GMG_NOALLOC_MAX_UNKNOWNS = 512


def gmg_coarse_solve_noalloc(params: gmg_params, a: torch.Tensor, b: torch.Tensor, x: torch.Tensor, stream=None):
    """Dense direct solve A(a) x = b on a small grid (<= 512 cells) with no
    device allocation: the scratch lives in a fixed array inside libgmg."""
    n = params.nx * params.ny * params.nz
    _check(load().gmg_coarse_solve_noalloc(ctypes.byref(params), _dev(a, numel=n, name="a"),
                                           _dev(b, numel=n, name="b"), _dev(x, numel=n, name="x"),
                                           _stream_ptr(stream)), "gmg_coarse_solve_noalloc")


def assemble_coefficient_rhs(params: gmg_params, n_e: torch.Tensor, n_p: torch.Tensor, a: torch.Tensor,
                             f: torch.Tensor, tau: float, mu_e: float, mu_p: float, diffusion=(0.0, 0.0, 0.0),
                             e_over_eps0: float = E_OVER_EPS0_CM, stream=None):
    """a and f of the elliptic step (eqs. (semi2), (e18)) from the densities,
    on the grid of ``params``; all tensors FP64 on the device."""
    n = params.nx * params.ny * params.nz
    dc = gmg_density_coef(float(tau), float(mu_e), float(mu_p), float(diffusion[0]), float(diffusion[1]),
                          float(diffusion[2]), float(e_over_eps0))
    _check(load().assemble_coefficient_rhs(ctypes.byref(params), _dev(n_e, numel=n, name="n_e"),
                                           _dev(n_p, numel=n, name="n_p"), ctypes.byref(dc),
                                           _dev(a, numel=n, name="a"), _dev(f, numel=n, name="f"),
                                           _stream_ptr(stream)), "assemble_coefficient_rhs")


def transport_stage(params: gmg_params, base_e: torch.Tensor, base_p: torch.Tensor, eval_e: torch.Tensor,
                    eval_p: torch.Tensor, phi: torch.Tensor, c: float, out_e: torch.Tensor, out_p: torch.Tensor,
                    mu_e: float, mu_p: float, diffusion=(0.0, 0.0, 0.0), ion_a: float = 5.7, ion_b: float = 260.0,
                    pressure: float = 760.0, stream=None):
    """One explicit transport stage out = base + c R(eval) (eqs. (e1)-(e2)); FP64 device tensors."""
    n = params.nx * params.ny * params.nz
    tc = gmg_transport_coef(float(mu_e), float(mu_p), float(diffusion[0]), float(diffusion[1]), float(diffusion[2]),
                            float(ion_a), float(ion_b), float(pressure))
    _check(load().transport_stage(ctypes.byref(params), _dev(base_e, numel=n, name="base_e"),
                                  _dev(base_p, numel=n, name="base_p"), _dev(eval_e, numel=n, name="eval_e"),
                                  _dev(eval_p, numel=n, name="eval_p"), _dev(phi, numel=n, name="phi"),
                                  ctypes.byref(tc), float(c), _dev(out_e, numel=n, name="out_e"),
                                  _dev(out_p, numel=n, name="out_p"), _stream_ptr(stream)), "transport_stage")


def gmg_round_to_f32(src: torch.Tensor, dst: torch.Tensor, stream=None):
    """dst = src rounded to FP32 (nearest even); FP64 / FP32 device tensors of one size."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("gmg_round_to_f32: src and dst sizes differ")
    _check(load().gmg_round_to_f32(_dev(src, numel=n, name="src"), _dev(dst, numel=n, name="dst", dtype=torch.float32),
                                   ctypes.c_size_t(n), _stream_ptr(stream)), "gmg_round_to_f32")


def transport_step(params: gmg_params, n_e: torch.Tensor, n_p: torch.Tensor, phi: torch.Tensor, tau: float,
                   half_e: torch.Tensor, half_p: torch.Tensor, out_e: torch.Tensor, out_p: torch.Tensor,
                   rate: torch.Tensor, mu_e: float, mu_p: float, diffusion=(0.0, 0.0, 0.0), ion_a: float = 5.7,
                   ion_b: float = 260.0, pressure: float = 760.0, stream=None):
    """Predictor and corrector of eqs. (e1)-(e2) in the field of phi: half = n + (tau/2) R(n),
    out = n + tau R(half); half_*, rate are scratch; FP64 device tensors; out may be n."""
    n = params.nx * params.ny * params.nz
    tc = gmg_transport_coef(float(mu_e), float(mu_p), float(diffusion[0]), float(diffusion[1]), float(diffusion[2]),
                            float(ion_a), float(ion_b), float(pressure))
    _check(load().transport_step(ctypes.byref(params), _dev(n_e, numel=n, name="n_e"), _dev(n_p, numel=n, name="n_p"),
                                 _dev(phi, numel=n, name="phi"), ctypes.byref(tc), float(tau),
                                 _dev(half_e, numel=n, name="half_e"), _dev(half_p, numel=n, name="half_p"),
                                 _dev(out_e, numel=n, name="out_e"), _dev(out_p, numel=n, name="out_p"),
                                 _dev(rate, numel=n, name="rate"), _stream_ptr(stream)), "transport_step")

