"""Thin Python binding of libbse (include/bse.h): argument marshalling only.

Every function here forwards to the CUDA library; there is no CPU fallback.
If libbse.so has not been built, `load_library` raises.

Low-level names mirror the C ABI (bse_create, bse_solve, ...).  The `Solver`
class and `bse_eigenvalues` (torch.autograd) wrap them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbse.so")

# ---------------------------------------------------------------- constants
BSE_OK, BSE_EINVAL, BSE_ENOMEM, BSE_ENOTPD, BSE_ENOCONV, BSE_ETIMEOUT, BSE_ECUDA, BSE_ESTATE, \
    BSE_ENOTFINITE = range(9)
BSE_TDA, BSE_PH = 0, 1
BSE_C64, BSE_C128, BSE_C64_MIXED, BSE_C128_DF = 0, 1, 2, 3
BSE_HOST, BSE_DEVICE = 0, 1
BSE_LOWEST = 0
BSE_OP_A, BSE_OP_MPLUS, BSE_OP_MMINUS, BSE_OP_H = 0, 1, 2, 3

EXPORTED = ["bse_strerror", "bse_create", "bse_create_batched", "bse_solve", "bse_solve_ex",
            "bse_solve_batched", "bse_backward", "bse_apply", "bse_get_stats", "bse_destroy",
            "bse_apply_noalloc", "bse_backward_ex", "bse_haydock", "bse_selftest_bounded_wait",
            "bse_get_residuals", "bse_apply_mixed", "bse_measure_fp64_peak", "bse_solve_dense"]
BSE_IMPL_AUTO, BSE_IMPL_CUDA_CORES, BSE_IMPL_TENSOR_CORES = 0, 1, 2
BSE_VARIANT_SHAO, BSE_VARIANT_GRUNING, BSE_VARIANT_PROJECTED = 0, 1, 2
BSE_NOALLOC_MAX_N = 4096


class bse_solve_opts(ctypes.Structure):
    _fields_ = [("ncv", ctypes.c_int), ("maxit", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("v0", ctypes.c_void_p), ("lock_tol", ctypes.c_double),
                ("stream_launches", ctypes.c_int), ("tile_tau", ctypes.c_double),
                ("variant", ctypes.c_int)]


class bse_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("passes", ctypes.c_int64), ("restarts", ctypes.c_int64),
                ("nconv", ctypes.c_int), ("max_residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_product", ctypes.c_double),
                ("launches", ctypes.c_int64), ("shape_ctas_per_sm", ctypes.c_int),
                ("shape_strided", ctypes.c_int), ("tuned", ctypes.c_int),
                ("tiles_fine", ctypes.c_int64), ("tiles_coarse", ctypes.c_int64),
                ("retried_exact", ctypes.c_int)]


class BSEError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {bse_strerror(status)} (status {status})")


_LIB = None


def load_library(path: str | None = None):
    """Load libbse.so (raises if it is missing: there is no fallback path)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build(); "
                           "the BSE solver has no CPU fallback")
    lib = ctypes.CDLL(path)
    c_int, c_i64, c_dbl, c_vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    H = ctypes.c_void_p
    lib.bse_strerror.argtypes = [c_int]
    lib.bse_strerror.restype = ctypes.c_char_p
    lib.bse_create.argtypes = [c_i64, c_vp, c_vp, c_int, c_int, c_int, c_vp, ctypes.POINTER(H)]
    lib.bse_create_batched.argtypes = [c_int, ctypes.POINTER(c_i64), ctypes.POINTER(c_vp),
                                       ctypes.POINTER(c_vp), c_int, c_int, c_int, c_vp, ctypes.POINTER(H)]
    lib.bse_solve.argtypes = [H, c_int, c_dbl, c_int, ctypes.POINTER(c_dbl), c_vp, ctypes.POINTER(c_int)]
    lib.bse_solve_ex.argtypes = [H, c_int, c_dbl, c_int, ctypes.POINTER(bse_solve_opts),
                                 ctypes.POINTER(c_dbl), c_vp, ctypes.POINTER(c_int)]
    lib.bse_solve_batched.argtypes = [H, c_int, c_dbl, c_int, ctypes.POINTER(bse_solve_opts),
                                      ctypes.POINTER(c_dbl), ctypes.POINTER(c_vp), ctypes.POINTER(c_int)]
    lib.bse_backward.argtypes = [H, ctypes.POINTER(c_dbl), c_int, c_vp, c_vp]
    lib.bse_apply.argtypes = [H, c_int, c_int, c_vp, c_vp]
    lib.bse_get_stats.argtypes = [H, ctypes.POINTER(bse_stats)]
    lib.bse_get_residuals.argtypes = [H, c_int, ctypes.POINTER(c_dbl), c_int]
    lib.bse_apply_mixed.argtypes = [H, c_int, c_dbl, c_vp, c_vp]
    lib.bse_solve_dense.argtypes = [H, c_int, c_dbl, ctypes.POINTER(c_dbl), c_vp, ctypes.POINTER(c_int)]
    lib.bse_measure_fp64_peak.argtypes = [c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl)]
    lib.bse_destroy.argtypes = [H]
    lib.bse_apply_noalloc.argtypes = [c_i64, c_vp, c_vp, c_int, c_int, c_vp, c_vp, c_vp]
    lib.bse_backward_ex.argtypes = [H, ctypes.POINTER(c_dbl), c_int, c_vp, c_vp, c_int]
    lib.bse_selftest_bounded_wait.argtypes = [c_int, ctypes.POINTER(c_int)]
    PD = ctypes.POINTER(c_dbl)
    lib.bse_haydock.argtypes = [H, c_vp, c_int, c_int, c_int, c_int, PD, c_dbl, PD, PD, PD,
                                ctypes.POINTER(c_int)]
    for name in EXPORTED:
        if name != "bse_strerror":
            getattr(lib, name).restype = c_int
    _LIB = lib
    return lib


# ---------------------------------------------------------------- C-ABI names
def bse_strerror(status: int) -> str:
    return load_library().bse_strerror(int(status)).decode()


def _check(rc, where, ok=(BSE_OK,)):
    if rc not in ok:
        raise BSEError(rc, where)
    return rc


def bse_create(N, A_ptr, B_ptr, form, dtype, where, stream=0):
    h = ctypes.c_void_p()
    rc = load_library().bse_create(int(N), A_ptr, B_ptr, form, dtype, where, stream, ctypes.byref(h))
    _check(rc, "bse_create")
    return h


def bse_create_batched(Ns, A_ptrs, B_ptrs, form, dtype, where, stream=0):
    count = len(Ns)
    n_arr = (ctypes.c_int64 * count)(*[int(n) for n in Ns])
    a_arr = (ctypes.c_void_p * count)(*A_ptrs)
    b_arr = (ctypes.c_void_p * count)(*B_ptrs) if B_ptrs is not None else None
    h = ctypes.c_void_p()
    rc = load_library().bse_create_batched(count, n_arr, a_arr, b_arr, form, dtype, where, stream,
                                           ctypes.byref(h))
    _check(rc, "bse_create_batched")
    return h


def bse_solve_ex(h, nev, tol, which=BSE_LOWEST, opts=None, evec_ptr=None):
    ev = (ctypes.c_double * nev)()
    nconv = ctypes.c_int(0)
    o = ctypes.byref(opts) if opts is not None else None
    rc = load_library().bse_solve_ex(h, nev, float(tol), which, o, ev, evec_ptr, ctypes.byref(nconv))
    return rc, np.array(ev[:], dtype=np.float64), nconv.value


def bse_solve(h, nev, tol, which=BSE_LOWEST, evec_ptr=None):
    return bse_solve_ex(h, nev, tol, which, None, evec_ptr)


def bse_solve_batched(h, count, nev, tol, which=BSE_LOWEST, opts=None, evec_ptrs=None):
    ev = (ctypes.c_double * (count * nev))()
    nconv = (ctypes.c_int * count)()
    o = ctypes.byref(opts) if opts is not None else None
    ptrs = (ctypes.c_void_p * count)(*evec_ptrs) if evec_ptrs is not None else None
    rc = load_library().bse_solve_batched(h, nev, float(tol), which, o, ev, ptrs, nconv)
    return rc, np.array(ev[:], dtype=np.float64).reshape(count, nev), np.array(nconv[:])


def bse_backward(h, g_ptr, where, dA_ptr, dB_ptr):
    return load_library().bse_backward(h, ctypes.cast(g_ptr, ctypes.POINTER(ctypes.c_double)), where,
                                       dA_ptr, dB_ptr)


def bse_backward_ex(h, g_ptr, where, dA_ptr, dB_ptr, impl=BSE_IMPL_AUTO):
    return load_library().bse_backward_ex(h, ctypes.cast(g_ptr, ctypes.POINTER(ctypes.c_double)), where,
                                          dA_ptr, dB_ptr, impl)


def bse_haydock(h, d_ptr, where, m, sign, omega, eta, want_coefs=True):
    """Returns (status, spectrum, response (complex), coefficients, steps)."""
    omega = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
    nw = omega.shape[0]
    spec = np.zeros(nw)
    resp = np.zeros(2 * nw)
    coef = np.zeros(2 * m + 1) if want_coefs else None
    steps = ctypes.c_int(0)
    P = ctypes.POINTER(ctypes.c_double)
    rc = load_library().bse_haydock(h, d_ptr, where, m, sign, nw, omega.ctypes.data_as(P), eta,
                                    spec.ctypes.data_as(P), resp.ctypes.data_as(P),
                                    coef.ctypes.data_as(P) if coef is not None else None, ctypes.byref(steps))
    return rc, spec, resp[0::2] + 1j * resp[1::2], coef, steps.value


def bse_selftest_bounded_wait(arrive):
    """Returns (status, expired) of one bounded device wait (see bse.h)."""
    e = ctypes.c_int(-1)
    rc = load_library().bse_selftest_bounded_wait(int(arrive), ctypes.byref(e))
    return rc, e.value


def bse_apply(h, op, k, X_ptr, Y_ptr):
    return load_library().bse_apply(h, op, k, X_ptr, Y_ptr)


def bse_solve_dense(h, nev, tol, evec_ptr=None):
    """Dense structure-preserving diagonalisation (see bse.h): (status, eigenvalues, nconv)."""
    ev = (ctypes.c_double * nev)()
    nconv = ctypes.c_int(0)
    rc = load_library().bse_solve_dense(h, nev, float(tol), ev, evec_ptr, ctypes.byref(nconv))
    return rc, np.array(ev[:], dtype=np.float64), nconv.value


def bse_apply_mixed(h, op, tile_tau, x_ptr, y_ptr):
    """The mixed path's product on one complex128 device vector (see bse.h)."""
    return load_library().bse_apply_mixed(h, op, float(tile_tau), x_ptr, y_ptr)


def bse_apply_noalloc(N, A_ptr, B_ptr, dtype, op, x_ptr, y_ptr, stream=0):
    """Allocation-free product from full device matrices (N <= BSE_NOALLOC_MAX_N)."""
    return load_library().bse_apply_noalloc(int(N), A_ptr, B_ptr, dtype, op, x_ptr, y_ptr, stream)


def bse_get_stats(h) -> dict:
    s = bse_stats()
    _check(load_library().bse_get_stats(h, ctypes.byref(s)), "bse_get_stats")
    return {f: getattr(s, f) for f, _ in bse_stats._fields_}


def bse_get_residuals(h, n, problem=0):
    """FP64 relative residuals of the pairs the last solve returned (output order)."""
    r = (ctypes.c_double * max(n, 1))()
    _check(load_library().bse_get_residuals(h, int(problem), r, int(n)), "bse_get_residuals")
    return np.array(r[:n], dtype=np.float64)


def bse_measure_fp64_peak(iters=1 << 16):
    """Measured FP64 FMA rate of the current device (TFLOP/s, ms of the timed launch)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load_library().bse_measure_fp64_peak(int(iters), ctypes.byref(tf), ctypes.byref(ms)),
           "bse_measure_fp64_peak")
    return tf.value, ms.value


def bse_destroy(h):
    if h:
        return load_library().bse_destroy(h)
    return BSE_OK


# ---------------------------------------------------------------- torch-facing wrapper
def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.complex128:
        return BSE_C128
    if t.dtype == torch.complex64:
        return BSE_C64
    raise TypeError("A and B must be complex64 or complex128")


class Solver:
    """One BSE problem (or a batch) held on the GPU by libbse.

    A, B: torch tensors (complex64 / complex128, row-major N x N) on a CUDA
    device or numpy arrays on the host.  Only their upper triangles are read.
    """

    def __init__(self, A, B=None, form=None, stream=None, df=False, mixed=False):
        """df=True (complex128 input only): Lanczos products in double-FP32
        arithmetic (dtype BSE_C128_DF); everything else stays FP64.
        mixed=True (complex64 input only): dtype BSE_C64_MIXED (complex64
        storage, FP64 basis, double-FP32 products)."""
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("libbse needs a CUDA device")
        load_library()
        self.form = (BSE_PH if B is not None else BSE_TDA) if form is None else form
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if isinstance(A, np.ndarray):
            A = np.ascontiguousarray(A)
            self.dtype = BSE_C128 if A.dtype == np.complex128 else BSE_C64
            if A.dtype not in (np.complex64, np.complex128):
                raise TypeError("A must be complex64 or complex128")
            Bc = np.ascontiguousarray(B, dtype=A.dtype) if B is not None else None
            where = BSE_HOST
            aptr = A.ctypes.data
            bptr = Bc.ctypes.data if Bc is not None else None
            self.device = torch.device("cuda", torch.cuda.current_device())
        else:
            A = A.contiguous()
            self.dtype = _dtype_code(A)
            Bc = B.contiguous().to(A.dtype) if B is not None else None
            where = BSE_DEVICE if A.is_cuda else BSE_HOST
            if where == BSE_HOST:
                A = A.numpy()
                Bc = Bc.numpy() if Bc is not None else None
                aptr, bptr = A.ctypes.data, (Bc.ctypes.data if Bc is not None else None)
                self.device = torch.device("cuda", torch.cuda.current_device())
            else:
                aptr, bptr = A.data_ptr(), (Bc.data_ptr() if Bc is not None else None)
                self.device = A.device
        self.N = int(A.shape[0])
        self.cdtype = torch.complex128 if self.dtype == BSE_C128 else torch.complex64
        if df:
            if self.dtype != BSE_C128:
                raise TypeError("df products need complex128 A and B")
            self.dtype = BSE_C128_DF
        if mixed:
            if self.dtype != BSE_C64:
                raise TypeError("the mixed path needs complex64 A and B")
            self.dtype = BSE_C64_MIXED
        with torch.cuda.device(self.device):
            self.h = bse_create(self.N, aptr, bptr, self.form, self.dtype, where, self.stream.cuda_stream)
        self.nev = 0

    def solve(self, nev, tol=None, ncv=0, maxit=0, seed=0, vectors=True, lock_tol=0.0, check=True,
              graphs=True, v0=None, tile_tau=0.0, variant=BSE_VARIANT_SHAO, persistent=True):
        torch = _torch()
        if tol is None:
            tol = 1e-12 if self.dtype == BSE_C128 else 1e-6
        rows = 2 * self.N if self.form == BSE_PH else self.N
        ev = torch.empty((nev, rows), dtype=self.cdtype, device=self.device) if vectors else None
        v0t = None
        if v0 is not None:     # start vector in the Krylov-basis precision, on the device
            torch = _torch()
            bdt = torch.complex64 if self.dtype == BSE_C64 else torch.complex128
            v0t = torch.as_tensor(v0).to(device=self.device, dtype=bdt).contiguous()
        opts = bse_solve_opts(ncv=ncv, maxit=maxit, seed=seed, v0=v0t.data_ptr() if v0t is not None else None,
                              lock_tol=lock_tol, stream_launches=(0 if persistent else 2) if graphs else 1,
                              tile_tau=tile_tau, variant=variant)
        rc, vals, nconv = bse_solve_ex(self.h, nev, tol, BSE_LOWEST, opts,
                                       ev.data_ptr() if ev is not None else None)
        if check:
            _check(rc, "bse_solve")
        self.nev = nev
        self.status = rc
        vecs = ev.T if ev is not None else None   # (rows, nev) column-major view
        return vals, vecs, nconv

    def solve_dense(self, nev, tol=1e-10, vectors=True, check=True):
        """Dense structure-preserving diagonalisation (bse_solve_dense), PH handles only."""
        torch = _torch()
        ev = torch.empty((nev, 2 * self.N), dtype=self.cdtype, device=self.device) if vectors else None
        rc, vals, nconv = bse_solve_dense(self.h, nev, tol, ev.data_ptr() if ev is not None else None)
        if check:
            _check(rc, "bse_solve_dense")
        self.nev = nev
        self.status = rc
        return vals, (ev.T if ev is not None else None), nconv

    def apply(self, op, X):
        """Y = op(X) for a device block X (rows x k, any layout; k columns)."""
        torch = _torch()
        X2 = X.reshape(X.shape[0], -1)
        k = X2.shape[1]
        Xc = X2.T.contiguous().to(self.cdtype)       # column-major storage
        Y = torch.empty_like(Xc)
        _check(bse_apply(self.h, op, k, Xc.data_ptr(), Y.data_ptr()), "bse_apply")
        out = Y.T
        return out.reshape(X.shape) if X.dim() == 1 else out

    def backward(self, g, impl=BSE_IMPL_AUTO):
        torch = _torch()
        g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
        dA = torch.empty((self.N, self.N), dtype=self.cdtype, device=self.device)
        dB = torch.empty_like(dA) if self.form == BSE_PH else None
        rc = bse_backward_ex(self.h, g.ctypes.data, BSE_HOST, dA.data_ptr(),
                             dB.data_ptr() if dB is not None else None, impl)
        _check(rc, "bse_backward")
        return dA, dB

    def haydock(self, d, m, omega, eta, sign=-1):
        """Lanczos-Haydock absorption spectrum (bse_haydock): returns
        (spectrum, response F, {"alpha", "beta", "norm2"}, steps)."""
        torch = _torch()
        dt = torch.as_tensor(d).to(device=self.device, dtype=torch.complex128).contiguous()
        rc, spec, resp, coef, steps = bse_haydock(self.h, dt.data_ptr(), BSE_DEVICE, int(m), int(sign), omega, eta)
        _check(rc, "bse_haydock")
        coefs = {"alpha": coef[:m][:steps], "beta": coef[m:2 * m][:max(steps - 1, 0)], "norm2": coef[2 * m]}
        return spec, resp, coefs, steps

    def stats(self):
        return bse_get_stats(self.h)

    def residuals(self):
        """FP64 relative residual of every pair the last solve returned."""
        return bse_get_residuals(self.h, self.nev)

    def close(self):
        if getattr(self, "h", None):
            bse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedSolver:
    """Many independent PH problems of uneven N solved in lock-step launches."""

    def __init__(self, As, Bs, stream=None, mixed=False):
        """mixed=True (complex64 input only): dtype BSE_C64_MIXED for every
        problem (complex64 storage, FP64 basis, double-FP32 products)."""
        torch = _torch()
        load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.As = [a.contiguous() for a in As]
        self.Bs = [b.contiguous() for b in Bs]
        self.dtype = _dtype_code(self.As[0])
        if mixed:
            if self.dtype != BSE_C64:
                raise TypeError("the mixed path needs complex64 A and B")
            self.dtype = BSE_C64_MIXED
        self.cdtype = self.As[0].dtype
        self.Ns = [int(a.shape[0]) for a in self.As]
        self.device = self.As[0].device
        self.h = bse_create_batched(self.Ns, [a.data_ptr() for a in self.As], [b.data_ptr() for b in self.Bs],
                                    BSE_PH, self.dtype, BSE_DEVICE, self.stream.cuda_stream)
        self.As = self.Bs = None      # the library holds its own packed copies

    def solve(self, nev, tol=1e-6, ncv=0, maxit=0, vectors=False, check=True, graphs=True, tile_tau=0.0,
              variant=BSE_VARIANT_SHAO):
        torch = _torch()
        vecs = [torch.empty((nev, 2 * n), dtype=self.cdtype, device=self.device) for n in self.Ns] \
            if vectors else None
        opts = bse_solve_opts(ncv=ncv, maxit=maxit, seed=0, v0=None, lock_tol=0.0,
                              stream_launches=0 if graphs else 1, tile_tau=tile_tau, variant=variant)
        rc, vals, nconv = bse_solve_batched(self.h, len(self.Ns), nev, tol, BSE_LOWEST, opts,
                                            [v.data_ptr() for v in vecs] if vecs else None)
        if check:
            _check(rc, "bse_solve_batched")
        self.nev = nev
        return vals, ([v.T for v in vecs] if vecs else None), nconv

    def stats(self):
        return bse_get_stats(self.h)

    def residuals(self, problem):
        """FP64 relative residuals of the pairs the last solve returned for `problem`."""
        return bse_get_residuals(self.h, self.nev, problem)

    def close(self):
        if getattr(self, "h", None):
            bse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bse_eigenvalues(A, B, nev, tol=None, **kw):
    """Differentiable lowest eigenvalues (torch.autograd; the backward pass
    is the library's Hellmann-Feynman adjoint kernel).

    The solver handle (packed A, B and the eigenvectors) lives as long as the
    autograd graph that holds it: backward may run more than once
    (retain_graph=True), and the handle is released when the graph is freed.
    If neither input requires a gradient the handle is released at once."""
    torch = _torch()

    class _Eig(torch.autograd.Function):
        @staticmethod
        def forward(ctx, A_, B_):
            s = Solver(A_.detach(), None if B_ is None else B_.detach())
            vals, _, _ = s.solve(nev, tol=tol, **kw)
            if any(ctx.needs_input_grad):
                ctx.solver = s
            else:
                s.close()
            ctx.has_b = B_ is not None
            return torch.from_numpy(vals).to(A_.device)

        @staticmethod
        def backward(ctx, gout):
            s = getattr(ctx, "solver", None)
            if s is None or s.h is None:
                raise RuntimeError("bse_eigenvalues: the solver of this graph was released")
            dA, dB = s.backward(gout.detach().double().cpu().numpy())
            return dA, (dB if ctx.has_b else None)

    return _Eig.apply(A, B)
