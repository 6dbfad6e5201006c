"""ctypes binding of libhelm.so (include/helm.h): argument marshalling only.

Every computation runs in the library's sm_103a kernels; this module converts torch
tensors to raw pointers and the current CUDA stream, and turns status codes into
exceptions.  It raises ``HelmError`` if the library is missing instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhelm.so")

HELM_OK = 0
HELM_EINVAL = -1
HELM_ENOMEM = -2
HELM_ENOCONV = -3
HELM_ENUMERIC = -4
HELM_ETIMEOUT = -5
HELM_ECUDA = -6
HELM_EAGAIN = -7
HELM_C64 = 1
HELM_C128 = 2
HELM_CAUTO = 3
HELM_AUTO_C128_POINTS = 16384   # include/helm.h: HELM_CAUTO picks complex128 up to this many unknowns
_PRECISIONS = {"c64": HELM_C64, "c128": HELM_C128, "auto": HELM_CAUTO}


def _precision_code(precision: str) -> int:
    if precision not in _PRECISIONS:
        raise ValueError("precision must be 'c64', 'c128' or 'auto'")
    return _PRECISIONS[precision]

_STATUS = {0: "HELM_OK", -1: "HELM_EINVAL", -2: "HELM_ENOMEM", -3: "HELM_ENOCONV", -4: "HELM_ENUMERIC",
           -5: "HELM_ETIMEOUT", -6: "HELM_ECUDA", -7: "HELM_EAGAIN"}

# names declared in include/helm.h (checked by the CPU test suite)
EXPORTS = ("helm_setup", "helm_destroy", "helm_precond_apply", "helm_apply_operator", "helm_solve",
           "helm_solve_host", "helm_batch_solve", "helm_workspace_bytes", "helm_levels", "helm_precond_precision",
           "helm_poly_smoother",
           "helm_axis_coefficients",
           "helm_last_error",
           "helm_launch_count", "helm_profile_begin", "helm_profile_end", "helm_precond_apply_noalloc",
           "helm_batch_solve_host", "helm_serve_start", "helm_serve_submit", "helm_serve_poll", "helm_serve_wait",
           "helm_serve_stats", "helm_serve_stop", "helm_autotune", "helm_tuning_load", "helm_tuning_get",
           "helm_set_barrier_timeout", "helm_multidot")


class helm_serve_opts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int), ("precond_prec", ctypes.c_int),
                ("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("s", ctypes.c_int), ("ecs_frac", ctypes.c_double), ("theta_gamma", ctypes.c_double)]


class helm_serve_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("rejected", ctypes.c_longlong),
                ("queued", ctypes.c_int), ("active", ctypes.c_int), ("peak_active", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("handles_created", ctypes.c_int), ("handles_reused", ctypes.c_int),
                ("group_builds", ctypes.c_longlong), ("graph_builds", ctypes.c_longlong), ("build_s", ctypes.c_double)]


class HelmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class helm_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("ecs_frac", ctypes.c_double),
                ("theta_gamma", ctypes.c_double), ("ecs_sides", ctypes.c_int)]


HELM_ECS_BOTH, HELM_ECS_HIGH = 0, 1
_ECS_SIDES = {"both": HELM_ECS_BOTH, "high": HELM_ECS_HIGH}


class helm_opts(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("s", ctypes.c_int), ("coarsest_n", ctypes.c_int),
                ("precond_prec", ctypes.c_int), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("csl_eps", ctypes.c_double), ("smoother", ctypes.c_int), ("outer_basis", ctypes.c_int)]


HELM_BASIS_AUTO, HELM_BASIS_F64, HELM_BASIS_DF = 0, 1, 2
HELM_BASIS_DF_MIN_TOL = 1e-9
_BASES = {"auto": HELM_BASIS_AUTO, "f64": HELM_BASIS_F64, "df": HELM_BASIS_DF}


def _basis_code(basis: str) -> int:
    if basis not in _BASES:
        raise ValueError("basis must be 'auto', 'f64' or 'df'")
    return _BASES[basis]


class helm_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("rel_res_est", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("status", ctypes.c_int), ("basis", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhelm.so (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise HelmError(HELM_ECUDA, f"{path} is missing: build it with `python -m paper_1012_5379_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.helm_setup.argtypes = [ctypes.POINTER(helm_grid), vp, dp, dp, ctypes.POINTER(helm_opts), vp,
                               ctypes.POINTER(vp)]
    lib.helm_setup.restype = ip
    lib.helm_destroy.argtypes = [vp]
    lib.helm_destroy.restype = None
    lib.helm_precond_apply.argtypes = [vp, vp, vp, ip, vp]
    lib.helm_precond_apply.restype = ip
    lib.helm_apply_operator.argtypes = [vp, ip, vp, vp, ip, vp]
    lib.helm_apply_operator.restype = ip
    lib.helm_solve.argtypes = [vp, vp, vp, dp, ctypes.POINTER(helm_info), vp]
    lib.helm_solve.restype = ip
    lib.helm_solve_host.argtypes = [vp, vp, vp, dp, ctypes.POINTER(helm_info), vp]
    lib.helm_solve_host.restype = ip
    lib.helm_batch_solve.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(vp), dp,
                                     ctypes.POINTER(helm_info), vp]
    lib.helm_batch_solve.restype = ip
    lib.helm_batch_solve_host.argtypes = lib.helm_batch_solve.argtypes
    lib.helm_batch_solve_host.restype = ip
    lib.helm_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.helm_workspace_bytes.restype = ip
    lib.helm_levels.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip), ip]
    lib.helm_levels.restype = ip
    lib.helm_autotune.argtypes = [ctypes.POINTER(helm_grid), vp, dp, dp, ctypes.POINTER(helm_opts), ip,
                                  ctypes.c_char_p, ctypes.POINTER(dp), ctypes.POINTER(dp), vp]
    lib.helm_autotune.restype = ip
    lib.helm_multidot.argtypes = [ip, vp, ip, ctypes.c_size_t, vp, ctypes.POINTER(dp), vp]
    lib.helm_multidot.restype = ip
    lib.helm_set_barrier_timeout.argtypes = [dp]
    lib.helm_set_barrier_timeout.restype = ip
    lib.helm_tuning_load.argtypes = [ctypes.c_char_p]
    lib.helm_tuning_load.restype = ip
    lib.helm_tuning_get.argtypes = [ctypes.c_char_p, ip, ip, ip, ip, ctypes.POINTER(ip)]
    lib.helm_tuning_get.restype = ip
    lib.helm_precond_precision.argtypes = [vp, ctypes.POINTER(ip)]
    lib.helm_precond_precision.restype = ip
    dptr = ctypes.POINTER(ctypes.c_double)
    lib.helm_poly_smoother.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ip, dptr,
                                       dptr]
    lib.helm_poly_smoother.restype = ip
    lib.helm_axis_coefficients.argtypes = [ip, ctypes.c_double, ip, ctypes.c_double, ctypes.c_double, dptr, dptr,
                                           dptr]
    lib.helm_axis_coefficients.restype = ip
    lib.helm_last_error.argtypes = []
    lib.helm_last_error.restype = ctypes.c_char_p
    lib.helm_precond_apply_noalloc.argtypes = [ctypes.POINTER(helm_grid), dp, dp, ctypes.POINTER(helm_opts), vp, vp,
                                               ip, vp]
    lib.helm_precond_apply_noalloc.restype = ip
    lib.helm_serve_start.argtypes = [ctypes.POINTER(helm_serve_opts), ctypes.POINTER(vp)]
    lib.helm_serve_start.restype = ip
    lib.helm_serve_submit.argtypes = [vp, ip, ip, dp, dp, vp, vp, dp, ctypes.POINTER(ctypes.c_longlong)]
    lib.helm_serve_submit.restype = ip
    lib.helm_serve_poll.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(helm_info), ctypes.POINTER(dp)]
    lib.helm_serve_poll.restype = ip
    lib.helm_serve_wait.argtypes = [vp, ctypes.c_longlong, dp, ctypes.POINTER(helm_info), ctypes.POINTER(dp)]
    lib.helm_serve_wait.restype = ip
    lib.helm_serve_stats.argtypes = [vp, ctypes.POINTER(helm_serve_counters)]
    lib.helm_serve_stats.restype = ip
    lib.helm_serve_stop.argtypes = [vp]
    lib.helm_serve_stop.restype = ip
    lib.helm_launch_count.argtypes = []
    lib.helm_launch_count.restype = ctypes.c_ulonglong
    lib.helm_profile_begin.argtypes = [ctypes.c_char_p]
    lib.helm_profile_begin.restype = ip
    lib.helm_profile_end.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.helm_profile_end.restype = ip
    _lib = lib
    return lib


def _check(code: int, allow=(HELM_OK,)) -> int:
    if code not in allow:
        raise HelmError(code, load().helm_last_error().decode())
    return code


def _stream(stream) -> int:
    if stream is not None:
        return int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ptr(t) -> int:
    return t if isinstance(t, int) else t.data_ptr()


_DTYPES = {"c64": "torch.complex64", "c128": "torch.complex128"}


def _require_vec(name: str, t, shape, dtype: Optional[str] = None) -> None:
    """Reject a tensor the kernels would read or write out of bounds: wrong dtype
    (complex64 / complex128), shape, strides or device.  Raw integer pointers are
    passed through unchecked (the caller vouches for them)."""
    if isinstance(t, int):
        return
    if dtype is not None and str(t.dtype) != _DTYPES[dtype]:
        raise ValueError(f"{name} must be {_DTYPES[dtype]}, got {t.dtype}")
    if str(t.dtype) not in _DTYPES.values():
        raise ValueError(f"{name} must be complex64 or complex128, got {t.dtype}")
    if tuple(t.shape) != tuple(shape) and t.numel() != _numel(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _require_device(name: str, t) -> None:
    """A tensor must live on the current CUDA device (raw pointers pass unchecked)."""
    if isinstance(t, int):
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    import torch
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, the current device is cuda:{torch.cuda.current_device()}")


def _require_pair(names, a, b, shape, dtype: Optional[str] = None) -> None:
    """Two vectors of one call: the same complex precision (or `dtype`), `shape` and
    layout, both on the current device."""
    _require_vec(names[0], a, shape, dtype)
    _require_vec(names[1], b, shape, dtype if (dtype or isinstance(a, int)) else _dtype_name(a))
    _require_device(names[0], a)
    _require_device(names[1], b)


def _numel(shape) -> int:
    out = 1
    for s in shape:
        out *= s
    return out


def _dtype_name(t) -> str:
    return "c128" if str(t.dtype).endswith("complex128") else "c64"


def _prec_of(t) -> int:
    return HELM_C128 if str(t.dtype).endswith("complex128") else HELM_C64


@dataclass
class Info:
    iters: int
    restarts: int
    rel_res_est: float
    rel_res_true: float
    status: int
    basis: str = "f64"  # the Krylov basis arithmetic the solve ran in ('f64' or 'df')

    @staticmethod
    def of(ci: helm_info) -> "Info":
        return Info(ci.iters, ci.restarts, ci.rel_res_est, ci.rel_res_true, ci.status,
                    "df" if ci.basis == HELM_BASIS_DF else "f64")


class Handle:
    """One Helmholtz problem: grid, wavenumber, CSG angle, hierarchy and workspace
    (helm_setup / helm_destroy)."""

    def __init__(self, dim: int, n: int, theta_beta: float, k: Optional[float] = None, phi=None,
                 theta_gamma: float = 0.5, ecs_frac: float = 0.125, nu1: int = 1, nu2: int = 1, s: int = 3,
                 coarsest_n: int = 3, precision: str = "c64", restart: int = 0, maxit: int = 400, stream=None,
                 csl_eps: float = 0.0, smoother: str = "gmres", ecs_sides: str = "both", basis: str = "auto"):
        lib = load()
        self.dim, self.n = dim, n
        self.precision = precision
        if ecs_sides not in _ECS_SIDES:
            raise ValueError("ecs_sides must be 'both' or 'high'")
        g = helm_grid(dim, n, ecs_frac, theta_gamma, _ECS_SIDES[ecs_sides])
        if smoother not in ("gmres", "poly"):
            raise ValueError("smoother must be 'gmres' or 'poly'")
        o = helm_opts(nu1, nu2, s, coarsest_n, _precision_code(precision), restart, maxit,
                      float(csl_eps), 1 if smoother == "poly" else 0, _basis_code(basis))
        h = ctypes.c_void_p()
        phi_ptr = None if phi is None else _ptr(phi)
        self._phi = phi  # keep the caller's field alive during setup
        _check(lib.helm_setup(ctypes.byref(g), phi_ptr, float(k if k is not None else 0.0), float(theta_beta),
                              ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        self._h = h

    @property
    def ptr(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().helm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def resolved_precision(self) -> str:
        """The preconditioner precision of the handle ('c64' or 'c128'; what 'auto'
        resolved to)."""
        p = ctypes.c_int()
        _check(load().helm_precond_precision(self._h, ctypes.byref(p)))
        return "c128" if p.value == HELM_C128 else "c64"

    def levels(self) -> list:
        n = ctypes.c_int()
        sizes = (ctypes.c_int * 32)()
        _check(load().helm_levels(self._h, ctypes.byref(n), sizes, 32))
        return list(sizes[: n.value])

    def workspace_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(load().helm_workspace_bytes(self._h, ctypes.byref(b)))
        return b.value

    def _vec_shape(self):
        return (self.n,) * self.dim

    def precond_apply(self, r, z, stream=None):
        """z ~ (M^CSG)^{-1} r by one V-cycle (torch complex64/complex128 CUDA tensors of
        the same dtype, n^dim elements)."""
        _require_pair(("r", "z"), r, z, self._vec_shape())
        prec = _prec_of(r)
        _check(load().helm_precond_apply(self._h, _ptr(r), _ptr(z), prec, _stream(stream)))
        return z

    def apply_operator(self, v, w, which: str = "M", stream=None):
        _require_pair(("v", "w"), v, w, self._vec_shape())
        prec = _prec_of(v)
        _check(load().helm_apply_operator(self._h, 1 if which == "H" else 0, _ptr(v), _ptr(w), prec,
                                          _stream(stream)))
        return w

    def solve(self, b, x, tol: float, stream=None) -> Info:
        """FGMRES solve of H x = b (complex128 CUDA tensors; x holds the initial guess)."""
        _require_pair(("b", "x"), b, x, self._vec_shape(), "c128")
        ci = helm_info()
        _check(load().helm_solve(self._h, _ptr(b), _ptr(x), float(tol), ctypes.byref(ci), _stream(stream)),
               allow=(HELM_OK, HELM_ENOCONV, HELM_ENUMERIC))
        return Info.of(ci)

    def solve_host(self, b_host, x_host, tol: float, stream=None) -> Info:
        """As solve, with host arrays (numpy complex128 or pinned torch tensors)."""
        ci = helm_info()
        bp = b_host.ctypes.data if hasattr(b_host, "ctypes") else _ptr(b_host)
        xp = x_host.ctypes.data if hasattr(x_host, "ctypes") else _ptr(x_host)
        _check(load().helm_solve_host(self._h, bp, xp, float(tol), ctypes.byref(ci), _stream(stream)),
               allow=(HELM_OK, HELM_ENOCONV, HELM_ENUMERIC))
        return Info.of(ci)


def precond_apply_noalloc(dim: int, n: int, theta_beta: float, k: float, r, z, theta_gamma: float = 0.5,
                          ecs_frac: float = 0.125, nu1: int = 1, nu2: int = 1, s: int = 3, precision: str = "c64",
                          coarsest_n: int = 3, stream=None):
    """One V-cycle on a small grid through helm_precond_apply_noalloc: the library
    allocates no device memory for it (its working memory is a fixed array inside the
    library).  r, z: torch CUDA tensors of shape (n,)*dim, both complex64 or both
    complex128, contiguous, on the current device (ValueError otherwise: the C entry
    point takes one precision for both and cannot see a tensor's size)."""
    if isinstance(r, int) or isinstance(z, int):
        raise ValueError("r and z must be torch tensors")
    if tuple(r.shape) != (n,) * dim or tuple(z.shape) != (n,) * dim:
        raise ValueError(f"r and z must have shape {(n,) * dim}, got {tuple(r.shape)} and {tuple(z.shape)}")
    _require_pair(("r", "z"), r, z, (n,) * dim)
    g = helm_grid(dim, n, ecs_frac, theta_gamma, HELM_ECS_BOTH)
    o = helm_opts(nu1, nu2, s, coarsest_n, HELM_C128 if precision == "c128" else HELM_C64, 0, 0, 0.0, 0)
    prec = _prec_of(r)
    _check(load().helm_precond_apply_noalloc(ctypes.byref(g), float(k), float(theta_beta), ctypes.byref(o),
                                             _ptr(r), _ptr(z), prec, _stream(stream)))
    return z


def autotune(dim: int, n: int, theta_beta: float, k: Optional[float] = None, phi=None, precision: str = "c64",
             theta_gamma: float = 0.5, ecs_frac: float = 0.125, reps: int = 10, path: Optional[str] = None,
             stream=None):
    """helm_autotune: tune the V-cycle's launch choices for this problem's levels on the
    current device; returns (default, tuned) milliseconds per V-cycle.  With `path` the
    process's whole table is written there as JSON."""
    g = helm_grid(dim, n, ecs_frac, theta_gamma, HELM_ECS_BOTH)
    o = helm_opts(1, 1, 3, 3, _precision_code(precision), 0, 1, 0.0, 0)
    d0, d1 = ctypes.c_double(), ctypes.c_double()
    _check(load().helm_autotune(ctypes.byref(g), None if phi is None else _ptr(phi),
                                float(k if k is not None else 0.0), float(theta_beta), ctypes.byref(o), int(reps),
                                None if path is None else path.encode(), ctypes.byref(d0), ctypes.byref(d1),
                                _stream(stream)))
    return d0.value, d1.value


def set_barrier_timeout(seconds: float) -> None:
    """helm_set_barrier_timeout: spin limit of the persistent V-cycle segments' grid
    barrier (seconds, default 1)."""
    _check(load().helm_set_barrier_timeout(float(seconds)))


def tuning_load(path: Optional[str] = None) -> None:
    """helm_tuning_load: replace the process's tuned launch choices with a JSON table."""
    _check(load().helm_tuning_load(None if path is None else path.encode()))


def tuning_get(pass_name: str, dim: int, P: int, precision: str = "c64", J: int = 0):
    """helm_tuning_get: the table's 4 integers for a key, or None (built-in default)."""
    v = (ctypes.c_int * 4)()
    rc = load().helm_tuning_get(pass_name.encode(), int(dim), int(P), _precision_code(precision), int(J), v)
    if rc < 0:
        _check(rc)
    return list(v) if rc == 1 else None


def multidot(V, w, basis: str = "df", stream=None):
    """h_i = <V[i], w> through the outer multi-dot pass (helm_multidot): V a contiguous
    complex128 CUDA tensor of shape (nvec, npts), w one of shape (npts,).  Returns a
    complex128 numpy array of nvec values."""
    import numpy as np
    if basis not in ("f64", "df"):
        raise ValueError("basis must be 'f64' or 'df'")
    if V.dim() != 2 or w.dim() != 1 or V.shape[1] != w.shape[0]:
        raise ValueError("V must be (nvec, npts) and w (npts,)")
    nvec, npts = int(V.shape[0]), int(V.shape[1])
    _require_vec("V", V, (nvec, npts), "c128")
    _require_vec("w", w, (npts,), "c128")
    _require_device("V", V)
    _require_device("w", w)
    out = (ctypes.c_double * (2 * max(nvec, 1)))()
    _check(load().helm_multidot(_basis_code(basis), _ptr(V), nvec, npts, _ptr(w), out, _stream(stream)))
    a = np.frombuffer(out, dtype=np.float64)[:2 * nvec]
    return a[0::2] + 1j * a[1::2]


def poly_smoother(k: float, h: float, theta_beta: float, theta_gamma: float, dim: int):
    """The third-degree polynomial smoother of a level (Sec. 4): (phi, [w1, w2, w3])."""
    phi = ctypes.c_double()
    w = (ctypes.c_double * 6)()
    _check(load().helm_poly_smoother(float(k), float(h), float(theta_beta), float(theta_gamma), int(dim),
                                     ctypes.byref(phi), w))
    return phi.value, [complex(w[2 * j], w[2 * j + 1]) for j in range(3)]


def axis_coefficients(n: int, ecs_frac: float, theta_gamma: float, theta_beta: float, ecs_sides: str = "both"):
    """The setup's stencil coefficients (a, d, c) of one axis (Sec. 2), computed on the
    host by helm_axis_coefficients: three complex128 numpy arrays of length n."""
    import numpy as np
    if ecs_sides not in _ECS_SIDES:
        raise ValueError("ecs_sides must be 'both' or 'high'")
    out = [np.zeros(2 * n, dtype=np.float64) for _ in range(3)]
    dptr = ctypes.POINTER(ctypes.c_double)
    _check(load().helm_axis_coefficients(int(n), float(ecs_frac), _ECS_SIDES[ecs_sides], float(theta_gamma),
                                         float(theta_beta), *[o.ctypes.data_as(dptr) for o in out]))
    return tuple(o[0::2] + 1j * o[1::2] for o in out)


def launch_count() -> int:
    """Kernels launched by libhelm.so so far in this process."""
    return int(load().helm_launch_count())


def profile_begin(prefix: str = "") -> None:
    _check(load().helm_profile_begin(prefix.encode()))


def profile_end() -> dict:
    """Per-class launches, total CUDA-event milliseconds, algorithmic bytes, flops."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().helm_profile_end(buf, len(buf)))
    return json.loads(buf.value.decode())


def batch_solve(handles: Sequence[Handle], bs, xs, tol: float, stream=None):
    """helm_batch_solve over several handles; returns a list of Info."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.ptr for h in handles])
    bp = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
    xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    infos = (helm_info * n)()
    _check(load().helm_batch_solve(hs, n, bp, xp, float(tol), infos, _stream(stream)),
           allow=(HELM_OK, HELM_ENOCONV, HELM_ENUMERIC))
    return [Info.of(infos[i]) for i in range(n)]


def batch_solve_host(handles: Sequence[Handle], bs, xs, tol: float, stream=None):
    """helm_batch_solve_host: host arrays (numpy complex128 or pinned tensors)."""
    n = len(handles)
    hp = (ctypes.c_void_p * n)(*[h.ptr for h in handles])
    addr = lambda a: a.ctypes.data if hasattr(a, "ctypes") else _ptr(a)
    bp = (ctypes.c_void_p * n)(*[addr(b) for b in bs])
    xp = (ctypes.c_void_p * n)(*[addr(x) for x in xs])
    infos = (helm_info * n)()
    _check(load().helm_batch_solve_host(hp, n, bp, xp, float(tol), infos, _stream(stream)),
           allow=(HELM_OK, HELM_ENOCONV, HELM_ENUMERIC))
    return [Info.of(infos[i]) for i in range(n)]


def _host_ptr(a) -> int:
    return a.ctypes.data if hasattr(a, "ctypes") else a.data_ptr()


class Server:
    """Continuous-batching solve server (helm_serve_*).  submit() borrows the source
    and solution arrays (numpy complex128, or pinned torch tensors for overlapped
    copies) until the ticket completes; this object keeps references to them."""

    def __init__(self, budget_bytes: int = 120 << 30, max_active: int = 0, precision: str = "c64",
                 restart: int = 40, maxit: int = 400, theta_gamma: float = 0.5, ecs_frac: float = 0.125):
        o = helm_serve_opts(budget_bytes, max_active, HELM_C128 if precision == "c128" else HELM_C64, restart,
                            maxit, 1, 1, 3, ecs_frac, theta_gamma)
        s = ctypes.c_void_p()
        _check(load().helm_serve_start(ctypes.byref(o), ctypes.byref(s)))
        self._s = s
        self._borrowed = {}

    def submit(self, dim: int, n: int, k: float, theta_beta: float, b_host, x_host, tol: float) -> int:
        t = ctypes.c_longlong()
        _check(load().helm_serve_submit(self._s, dim, n, float(k), float(theta_beta), _host_ptr(b_host),
                                        _host_ptr(x_host), float(tol), ctypes.byref(t)))
        self._borrowed[t.value] = (b_host, x_host)
        return t.value

    def poll(self, ticket: int):
        """(Info, latency seconds, status) once finished, else None."""
        ci, lat = helm_info(), ctypes.c_double()
        rc = load().helm_serve_poll(self._s, ticket, ctypes.byref(ci), ctypes.byref(lat))
        if rc == HELM_EAGAIN:
            return None
        self._borrowed.pop(ticket, None)
        _check(rc, allow=(HELM_OK, HELM_ENOCONV, HELM_ENUMERIC, HELM_ENOMEM))
        return Info.of(ci), lat.value, rc

    def wait(self, ticket: int, timeout: float = 600.0):
        ci, lat = helm_info(), ctypes.c_double()
        rc = load().helm_serve_wait(self._s, ticket, float(timeout), ctypes.byref(ci), ctypes.byref(lat))
        if rc != HELM_ETIMEOUT:
            self._borrowed.pop(ticket, None)
        _check(rc, allow=(HELM_OK, HELM_ENOCONV, HELM_ENUMERIC, HELM_ENOMEM))
        return Info.of(ci), lat.value, rc

    def stats(self) -> dict:
        st = helm_serve_counters()
        _check(load().helm_serve_stats(self._s, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in helm_serve_counters._fields_}

    def stop(self):
        """Finish every request, stop the worker, free the device memory."""
        if self._s is not None and self._s.value:
            s, self._s = self._s, ctypes.c_void_p()
            _check(load().helm_serve_stop(s))
        self._borrowed.clear()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
