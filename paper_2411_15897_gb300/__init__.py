"""Python binding of libbah, the GB300 block-acoustic elastic Helmholtz solver.

Argument marshalling only: every step of the solve runs in the CUDA kernels
behind the C ABI of include/bah.h.  The functions keep the C names
(bah_create, bah_apply_operator, ...) and take torch tensors for device
buffers; ``Solver`` wraps one context.

The library must have been built (``python -m paper_2411_15897_gb300._build``
or ``__graft_entry__.build()``); importing works without it, but every call
raises ``RuntimeError`` if libbah.so cannot be loaded -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbah.so")

BAH_OK = 0
BAH_ERR_ARG = -1
BAH_ERR_OOM = -2
BAH_ERR_CUDA = -3
BAH_ERR_NOT_CONVERGED = -4
BAH_ERR_NONFINITE = -5
BAH_ERR_UNSUPPORTED = -6
BAH_FP64 = 0
BAH_MIXED = 1
BAH_CYCLE_V = 0
BAH_CYCLE_W = 1
BAH_INTERGRID_BILINEAR = 0
BAH_INTERGRID_MIXED = 1
BAH_KRYLOV_FP64 = 0
BAH_KRYLOV_DF = 1

# every symbol include/bah.h declares
EXPORTS = ("bah_default_opts", "bah_create", "bah_destroy", "bah_sizes", "bah_get_info", "bah_spectral_radius",
           "bah_spectral_radius_z",
           "bah_apply_operator",
           "bah_apply_preconditioner", "bah_solve", "bah_block_cycle", "bah_level_stencil",
           "bah_status_string", "bah_last_error", "bah_profile_control", "bah_profile_read",
           "bah_residual_norm_static", "bah_solve_adjoint", "bah_misfit", "bah_gradient")
BAH_STATIC_MAX_RHS = 64


class bah_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3)]


class bah_medium(C.Structure):
    _fields_ = [("lambda_", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
                ("rho", C.POINTER(C.c_double)), ("gamma", C.POINTER(C.c_double)), ("omega", C.c_double)]


class bah_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("levels", C.c_int), ("max_coarse_cells", C.c_int), ("cycle", C.c_int),
                ("nu_pre", C.c_int), ("nu_post", C.c_int), ("jacobi_w", C.c_double * 8), ("n_jacobi_w", C.c_int),
                ("shift_alpha", C.c_double), ("intergrid", C.c_int), ("restart", C.c_int), ("maxit", C.c_int),
                ("rhs_block", C.c_int), ("krylov_arith", C.c_int), ("block_rtol", C.c_double),
                ("block_maxit", C.c_int), ("block_alpha", C.c_double), ("block_krylov", C.c_int)]


class bah_info(C.Structure):
    _fields_ = [("levels", C.c_int), ("shift_alpha", C.c_double), ("coarse_points", C.c_int),
                ("cluster_level", C.c_int), ("cluster_ctas", C.c_int), ("cluster_smem_bytes", C.c_longlong),
                ("block_iters", C.c_longlong), ("block_failures", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bah_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("relres_true", C.c_double),
                ("relres_est", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BahError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({last_error()})")


_lib = None


def lib():
    """The loaded libbah (ctypes.CDLL); raises RuntimeError if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbah.so not found at {LIB_PATH}: build it with "
                               "`python -m paper_2411_15897_gb300._build` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.bah_default_opts.argtypes = [C.POINTER(bah_opts)]
        L.bah_default_opts.restype = None
        L.bah_create.argtypes = [C.POINTER(bah_grid), C.POINTER(bah_medium), C.POINTER(bah_opts), C.POINTER(vp)]
        L.bah_create.restype = C.c_int
        L.bah_destroy.argtypes = [vp]
        L.bah_destroy.restype = None
        L.bah_sizes.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
        L.bah_sizes.restype = C.c_int
        L.bah_get_info.argtypes = [vp, C.POINTER(bah_info)]
        L.bah_get_info.restype = C.c_int
        L.bah_spectral_radius.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.bah_spectral_radius.restype = C.c_int
        L.bah_spectral_radius_z.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.bah_spectral_radius_z.restype = C.c_int
        L.bah_apply_operator.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp]
        L.bah_apply_operator.restype = C.c_int
        L.bah_apply_preconditioner.argtypes = [vp, vp, vp, C.c_int, vp]
        L.bah_apply_preconditioner.restype = C.c_int
        L.bah_solve.argtypes = [vp, vp, vp, C.c_int, C.c_double, C.POINTER(bah_stats), vp]
        L.bah_solve.restype = C.c_int
        L.bah_block_cycle.argtypes = [vp, C.c_int, vp, vp, vp]
        L.bah_block_cycle.restype = C.c_int
        ip = C.POINTER(C.c_int)
        L.bah_level_stencil.argtypes = [vp, C.c_int, C.c_int, vp, ip, ip, ip, ip]
        L.bah_level_stencil.restype = C.c_int
        L.bah_profile_control.argtypes = [vp, C.c_uint, C.c_int]
        L.bah_profile_control.restype = C.c_int
        L.bah_profile_read.argtypes = [vp, vp]
        L.bah_profile_read.restype = C.c_int
        L.bah_solve_adjoint.argtypes = [vp, vp, vp, C.c_int, C.c_double, C.POINTER(bah_stats), vp]
        L.bah_solve_adjoint.restype = C.c_int
        L.bah_misfit.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, vp, vp, vp]
        L.bah_misfit.restype = C.c_int
        L.bah_gradient.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp, vp]
        L.bah_gradient.restype = C.c_int
        L.bah_residual_norm_static.argtypes = [vp, vp, vp, C.c_int, vp, vp]
        L.bah_residual_norm_static.restype = C.c_int
        L.bah_status_string.argtypes = [C.c_int]
        L.bah_status_string.restype = C.c_char_p
        L.bah_last_error.argtypes = []
        L.bah_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def status_string(s):
    return lib().bah_status_string(int(s)).decode()


def last_error():
    return lib().bah_last_error().decode()


def _check(s, what):
    if s != BAH_OK:
        raise BahError(s, what)
    return s


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------
def bah_default_opts(**kw) -> bah_opts:
    o = bah_opts()
    lib().bah_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "jacobi_w":
            for i, w in enumerate(v):
                o.jacobi_w[i] = float(w)
            o.n_jacobi_w = len(v)
        else:
            setattr(o, k, v)
    return o


def bah_create(n, h, lam, mu, rho, gamma, omega, opts: bah_opts | None = None):
    """Create a context; medium arrays are host numpy arrays (cells, x_1 fastest)."""
    g = bah_grid()
    g.dim = len(n)
    for i, v in enumerate(n):
        g.n[i] = int(v)
    for i, v in enumerate(h):
        g.h[i] = float(v)
    arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (lam, mu, rho, gamma)]
    P = C.POINTER(C.c_double)
    m = bah_medium(*(a.ctypes.data_as(P) for a in arrs), float(omega))
    ctx = C.c_void_p()
    _check(lib().bah_create(C.byref(g), C.byref(m), C.byref(opts) if opts is not None else None, C.byref(ctx)),
           "bah_create")
    return ctx


def bah_destroy(ctx):
    lib().bah_destroy(ctx)


def bah_get_info(ctx):
    out = bah_info()
    _check(lib().bah_get_info(ctx, C.byref(out)), "bah_get_info")
    return out.as_dict()


def bah_spectral_radius(ctx, x0, iters, stream=None):
    """(rho, history) of the power method on T = I - P^{-1} D H from device vector x0."""
    hist = (C.c_double * int(iters))()
    rho = C.c_double()
    _check(lib().bah_spectral_radius(ctx, _ptr(x0), int(iters), hist, C.byref(rho), _stream(stream)),
           "bah_spectral_radius")
    return rho.value, np.array(hist[:])


def bah_spectral_radius_z(ctx, x0, iters, stream=None):
    """(rho, history) of the power method on Z = Xi A_s^{-1} B^T H_p,s^{-1} (Theorem 1)
    from the device pressure-lattice vector x0 (needs a context with block_rtol > 0)."""
    hist = (C.c_double * int(iters))()
    rho = C.c_double()
    _check(lib().bah_spectral_radius_z(ctx, _ptr(x0), int(iters), hist, C.byref(rho), _stream(stream)),
           "bah_spectral_radius_z")
    return rho.value, np.array(hist[:])


def bah_sizes(ctx):
    n = C.c_longlong()
    L = C.c_int()
    _check(lib().bah_sizes(ctx, C.byref(n), C.byref(L)), "bah_sizes")
    return n.value, L.value


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if hasattr(t, "data_ptr") else C.c_void_p(t.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def bah_apply_operator(ctx, x, y, nrhs=1, conj_transpose=0, stream=None):
    return _check(lib().bah_apply_operator(ctx, _ptr(x), _ptr(y), int(nrhs), int(conj_transpose), _stream(stream)),
                  "bah_apply_operator")


def bah_apply_preconditioner(ctx, r, z, nrhs=1, stream=None):
    return _check(lib().bah_apply_preconditioner(ctx, _ptr(r), _ptr(z), int(nrhs), _stream(stream)),
                  "bah_apply_preconditioner")


def bah_block_cycle(ctx, block, b, x, stream=None):
    return _check(lib().bah_block_cycle(ctx, int(block), _ptr(b), _ptr(x), _stream(stream)), "bah_block_cycle")


def bah_level_stencil(ctx, block, level):
    """FP64 stencil of one block and level: (array (slots, n2, n1) complex128, rx, rz)."""
    rx, rz, n1, n2 = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(lib().bah_level_stencil(ctx, int(block), int(level), None, C.byref(rx), C.byref(rz), C.byref(n1),
                                   C.byref(n2)), "bah_level_stencil")
    out = np.zeros(((2 * rx.value + 1) * (2 * rz.value + 1), n2.value, n1.value), dtype=np.complex128)
    _check(lib().bah_level_stencil(ctx, int(block), int(level), C.c_void_p(out.ctypes.data), None, None, None, None),
           "bah_level_stencil")
    return out, rx.value, rz.value


def bah_solve(ctx, b, x, nrhs=1, rtol=1e-6, stream=None):
    """Returns (status, [stats dict per rhs]).  b, x: both torch CUDA tensors or
    both host arrays (numpy / pinned torch CPU tensors)."""
    st = (bah_stats * max(1, nrhs))()
    s = lib().bah_solve(ctx, _ptr(b), _ptr(x), int(nrhs), float(rtol), st, _stream(stream))
    if s not in (BAH_OK, BAH_ERR_NOT_CONVERGED, BAH_ERR_NONFINITE):
        raise BahError(s, "bah_solve")
    return s, [st[k].as_dict() for k in range(nrhs)]


BAH_K_NAMES = ("operator", "distrib", "urhs", "jacobi", "residual", "restrict", "prolong", "coarse", "dot",
               "axpy", "norm", "update", "small", "unused13", "cluster", "unused15")


class bah_profile(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("class_launches", C.c_longlong * 16), ("class_calls", C.c_longlong * 16),
                ("class_ms", C.c_double * 16), ("class_bytes", C.c_double * 16)]

    def as_dict(self):
        return {"launches": self.launches,
                "classes": {nm: {"launches": self.class_launches[k], "calls": self.class_calls[k],
                                 "ms": self.class_ms[k], "bytes": self.class_bytes[k]}
                            for k, nm in enumerate(BAH_K_NAMES)}}


def bah_profile_control(ctx, timing_mask=0, reset=True):
    return _check(lib().bah_profile_control(ctx, C.c_uint(timing_mask), int(reset)), "bah_profile_control")


def bah_profile_read(ctx):
    p = bah_profile()
    _check(lib().bah_profile_read(ctx, C.byref(p)), "bah_profile_read")
    return p.as_dict()


def bah_solve_adjoint(ctx, b, y, nrhs=1, rtol=1e-6, stream=None):
    """Solve H^H y = b; returns (status, [stats dict per rhs])."""
    st = (bah_stats * max(1, nrhs))()
    s = lib().bah_solve_adjoint(ctx, _ptr(b), _ptr(y), int(nrhs), float(rtol), st, _stream(stream))
    if s not in (BAH_OK, BAH_ERR_NOT_CONVERGED, BAH_ERR_NONFINITE):
        raise BahError(s, "bah_solve_adjoint")
    return s, [st[k].as_dict() for k in range(nrhs)]


def bah_misfit(ctx, x, d, rec, nrec, nrhs, adj, misfit, stream=None):
    return _check(lib().bah_misfit(ctx, _ptr(x), _ptr(d), _ptr(rec), int(nrec), int(nrhs), _ptr(adj), _ptr(misfit),
                                   _stream(stream)), "bah_misfit")


def bah_gradient(ctx, x, y, nrhs, g_lambda, g_mu, g_rho, stream=None):
    return _check(lib().bah_gradient(ctx, _ptr(x), _ptr(y), int(nrhs), _ptr(g_lambda), _ptr(g_mu), _ptr(g_rho),
                                     _stream(stream)), "bah_gradient")


def bah_residual_norm_static(ctx, b, x, nrhs, relres, stream=None):
    """relres (device, nrhs doubles) = ||b - H x|| / ||b|| per right-hand side,
    computed without allocating (static device scratch); see include/bah.h."""
    return _check(lib().bah_residual_norm_static(ctx, _ptr(b), _ptr(x), int(nrhs), _ptr(relres), _stream(stream)),
                  "bah_residual_norm_static")


# ---------------------------------------------------------------------------
# convenience object
# ---------------------------------------------------------------------------
class Solver:
    """One solver context for a grid, medium and frequency."""

    def __init__(self, n, h, lam, mu, rho, gamma, omega, **opts):
        self.n = tuple(int(v) for v in n)
        self.opts = bah_default_opts(**opts)
        self.ctx = bah_create(self.n, h, lam, mu, rho, gamma, omega, self.opts)
        self.vector_len, self.levels = bah_sizes(self.ctx)
        self.info = bah_get_info(self.ctx)
        self.alpha = self.info["shift_alpha"]

    @classmethod
    def from_problem(cls, prob, **opts):
        return cls(prob.n, prob.h, prob.lam, prob.mu, prob.rho, prob.gamma, prob.omega, **opts)

    @property
    def shape(self):
        return (len(self.n) + 1,) + tuple(reversed(self.n))

    def close(self):
        if self.ctx is not None:
            bah_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _new(self, like, nrhs=1):
        import torch
        return torch.empty((nrhs,) + self.shape if nrhs > 1 else self.shape, dtype=torch.complex128,
                           device=like.device if hasattr(like, "device") else "cuda")

    def apply_operator(self, x, conj_transpose=False):
        nrhs = x.numel() // self.vector_len
        y = self._new(x, nrhs).reshape(x.shape)
        bah_apply_operator(self.ctx, x.contiguous(), y, nrhs, int(conj_transpose))
        return y

    def apply_preconditioner(self, r):
        nrhs = r.numel() // self.vector_len
        z = self._new(r, nrhs).reshape(r.shape)
        bah_apply_preconditioner(self.ctx, r.contiguous(), z, nrhs)
        return z

    def block_cycle(self, block, b):
        import torch
        x = torch.empty_like(b)
        bah_block_cycle(self.ctx, block, b.contiguous(), x)
        return x

    def solve(self, b, rtol=1e-6):
        import torch
        nrhs = (b.size if isinstance(b, np.ndarray) else b.numel()) // self.vector_len
        if isinstance(b, np.ndarray):
            b = np.ascontiguousarray(b, dtype=np.complex128)
            x = np.zeros_like(b)
        else:
            b = b.contiguous()
            x = torch.zeros_like(b)
        status, stats = bah_solve(self.ctx, b, x, nrhs, rtol)
        return x, status, stats
