"""Thin ctypes binding of libsurvgpu.so (include/survgpu.h).

Argument marshalling only: arrays (torch tensors on the GPU or the CPU, or
numpy arrays) are passed to the C ABI as raw pointers; every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback:
if the library is missing or no CUDA device is present, the calls raise.

Names follow the C ABI: ``cox_fit``, ``fg_fit``, ``loglik_grad_hess``,
``surv_sort_desc``, plus ``SurvData`` to describe a cohort and
``Workspace`` for a reusable device workspace.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsurvgpu.so")

SURV_OK = 0
SURV_W_NOT_CONVERGED = 1
SURV_E_INVALID = -1
SURV_E_UNSORTED = -2
SURV_E_STATUS = -3
SURV_E_NONFINITE = -4
SURV_E_NO_EVENTS = -5
SURV_E_CUDA = -6
SURV_E_DEVICE_TIMEOUT = -7
SURV_E_NOMEM = -8
SURV_E_INDEX = -9

SURV_CSC, SURV_DENSE = 0, 1
SURV_F32, SURV_F64, SURV_BF16 = 0, 1, 2
SURV_COX, SURV_FG = 0, 1
SURV_PEN = {"none": 0, "l1": 1, "l2": 2}
SURV_PREC = {"f32c": 0, "f64": 1}
SURV_FLAG_TEST_STALL = 1
SURV_FLAG_PERSISTENT = 2
SURV_FLAG_CV_TUNE = 4
SURV_FLAG_SPARSE_NUMERATOR = 8
SURV_FLAG_ONE_COORDINATE = 16
SURV_FLAG_SPEC_B8 = 32
SURV_FLAG_NO_PDL = 64
SURV_FLAG_CV_TILE1 = 256
SURV_FLAG_CV_TILE2 = 512

# exported symbols, in the order the header declares them
EXPORTS = ["surv_opts_default", "surv_workspace_create", "surv_workspace_destroy", "surv_sort_desc",
           "cox_fit", "fg_fit", "loglik_grad_hess", "surv_groups", "loglik_grad_hess_noalloc",
           "cox_nll_forward", "cox_nll_backward", "cox_lambda_max", "cox_cv_path", "surv_strerror",
           "surv_last_error", "surv_version"]


class surv_data(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int64), ("time", C.c_void_p), ("status", C.c_void_p),
                ("layout", C.c_int32), ("dtype", C.c_int32), ("col_ptr", C.c_void_p), ("row_idx", C.c_void_p),
                ("values", C.c_void_p)]


class surv_nll_data(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int32), ("ncols", C.c_int32), ("time", C.c_void_p),
                ("status", C.c_void_p), ("X", C.c_void_p)]


class surv_opts(C.Structure):
    _fields_ = [("penalty", C.c_int32), ("precision", C.c_int32), ("lambda_", C.c_double),
                ("penalty_factor", C.c_void_p), ("tol", C.c_double), ("max_sweeps", C.c_int32),
                ("flags", C.c_int32), ("wait_limit_s", C.c_double), ("stream", C.c_void_p),
                ("workspace", C.c_void_p)]


class surv_fit_info(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("converged", C.c_int32), ("nnz_beta", C.c_int32),
                ("device_error", C.c_int32), ("loglik", C.c_double), ("objective", C.c_double),
                ("objective_prev", C.c_double), ("n_groups", C.c_int64), ("coordinate_passes", C.c_int64),
                ("eta_updates", C.c_int64), ("kernel_launches", C.c_int64), ("ccd_kernel_ms", C.c_double),
                ("phase_ms", C.c_double * 16), ("row_passes", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_ms"] = list(self.phase_ms)
        return d


class surv_cv_info(C.Structure):
    _fields_ = [("nfits", C.c_int32), ("best_lambda", C.c_int32), ("max_sweeps_used", C.c_int32),
                ("fits_converged", C.c_int32), ("graph_replays", C.c_int32), ("ctas_per_fit", C.c_int32),
                ("row_pass_form", C.c_int32), ("tile_form", C.c_int32), ("kernel_launches", C.c_int64), ("n_groups", C.c_int64), ("coordinate_passes", C.c_int64),
                ("eta_updates", C.c_int64), ("ccd_kernel_ms", C.c_double), ("heldout_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libsurvgpu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsurvgpu.so not found at %s: run paper_2204_08183_gb300.build.build()" % path)
    lib = C.CDLL(path)
    lib.surv_opts_default.argtypes = [C.POINTER(surv_opts)]
    lib.surv_opts_default.restype = None
    lib.surv_workspace_create.argtypes = [C.POINTER(C.c_void_p)]
    lib.surv_workspace_destroy.argtypes = [C.c_void_p]
    lib.surv_sort_desc.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    for f in (lib.cox_fit, lib.fg_fit):
        f.argtypes = [C.POINTER(surv_data), C.POINTER(surv_opts), C.c_void_p, C.POINTER(surv_fit_info)]
        f.restype = C.c_int
    lib.loglik_grad_hess.argtypes = [C.POINTER(surv_data), C.c_int32, C.c_void_p, C.c_int32,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(surv_opts)]
    lib.surv_groups.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.c_int64), C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p]
    lib.loglik_grad_hess_noalloc.argtypes = [C.POINTER(surv_data), C.c_int32, C.c_void_p, C.c_int32,
                                             C.POINTER(C.c_double), C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.c_int32, C.c_void_p]
    for f in (lib.cox_nll_forward, lib.cox_nll_backward):
        f.argtypes = [C.POINTER(surv_nll_data), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        f.restype = C.c_int
    lib.cox_lambda_max.argtypes = [C.POINTER(surv_data), C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    lib.cox_lambda_max.restype = C.c_int
    lib.cox_cv_path.argtypes = [C.POINTER(surv_data), C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                C.POINTER(surv_opts), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.POINTER(surv_cv_info)]
    lib.cox_cv_path.restype = C.c_int
    lib.surv_strerror.argtypes = [C.c_int]
    lib.surv_strerror.restype = C.c_char_p
    lib.surv_last_error.restype = C.c_char_p
    _lib = lib
    return lib


class SurvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (load().surv_strerror(code).decode(), code, msg))
        self.code = code


def _check(rc, allow=(SURV_OK,)):
    if rc not in allow:
        raise SurvError(rc, load().surv_last_error().decode())
    return rc


def _ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not (a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"]):
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    raise TypeError("expected a torch tensor or a numpy array, got %r" % type(a))


def _dtype_code(a):
    name = str(a.dtype)
    if name.endswith("float32"):
        return SURV_F32
    if name.endswith("float64"):
        return SURV_F64
    if name.endswith("bfloat16"):
        return SURV_BF16
    raise TypeError("values must be float32, float64 or bfloat16 (dense X), got %s" % name)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return stream


class SurvData:
    """A cohort in the library's layout (subjects in decreasing time order).

    Dense X: a column-major (n, p) array -- a Fortran-ordered numpy array, or
    a torch tensor holding X^T contiguously (shape (p, n)), passed as ``X``
    (float32, float64 or bfloat16).  CSC: ``col_ptr``
    (int64, p+1), ``row_idx`` (int32), ``values`` (float32/float64 or None
    for indicators).  Arrays may live on
    the host or on the GPU; references are kept alive by this object.
    """

    def __init__(self, time, status, *, X=None, col_ptr=None, row_idx=None, values=None, n=None, p=None):
        self._keep = [time, status, X, col_ptr, row_idx, values]
        self.time, self.status = time, status
        n = int(time.shape[0]) if n is None else int(n)
        s = surv_data()
        s.n = n
        s.time = _ptr(time)
        s.status = _ptr(status)
        if X is not None:
            if isinstance(X, np.ndarray):
                if X.ndim != 2 or X.shape[0] != n or not X.flags["F_CONTIGUOUS"]:
                    raise ValueError("dense X must be a Fortran-ordered (n, p) array")
                p = X.shape[1]
            else:  # torch: expect the (p, n) row-major transpose
                if X.dim() != 2 or X.shape[1] != n:
                    raise ValueError("dense torch X must have shape (p, n) (column-major X)")
                p = X.shape[0]
            s.layout = SURV_DENSE
            s.dtype = _dtype_code(X)
            s.values = _ptr(X)
        else:
            p = int(col_ptr.shape[0]) - 1 if p is None else int(p)
            s.layout = SURV_CSC
            s.dtype = _dtype_code(values) if values is not None else SURV_F32
            s.col_ptr = _ptr(col_ptr)
            s.row_idx = _ptr(row_idx)
            s.values = _ptr(values)
        s.p = int(p)
        self.n, self.p = n, int(p)
        self.c = s


class Workspace:
    """Reusable device workspace (surv_workspace)."""

    def __init__(self):
        h = C.c_void_p()
        _check(load().surv_workspace_create(C.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            load().surv_workspace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_opts(penalty="none", lam=0.0, penalty_factor=None, tol=1e-8, max_sweeps=1000, precision="f32c",
              stream=None, workspace=None, flags=0, wait_limit_s=0.0):
    o = surv_opts()
    load().surv_opts_default(C.byref(o))
    o.penalty = SURV_PEN[penalty]
    o.precision = SURV_PREC[precision]
    o.lambda_ = float(lam)
    o.penalty_factor = _ptr(penalty_factor)
    o.tol = float(tol)
    o.max_sweeps = int(max_sweeps)
    o.flags = int(flags)
    o.wait_limit_s = float(wait_limit_s)
    o.stream = _stream(stream)
    o.workspace = workspace.handle if workspace is not None else None
    return o


def _fit(fn, data, beta, allow_not_converged, **kw):
    opts = make_opts(**kw)
    if beta is None:
        beta = np.zeros(data.p, dtype=np.float64)
    info = surv_fit_info()
    rc = fn(C.byref(data.c), C.byref(opts), C.c_void_p(_ptr(beta)), C.byref(info))
    allow = (SURV_OK, SURV_W_NOT_CONVERGED) if allow_not_converged else (SURV_OK,)
    _check(rc, allow)
    return beta, info.as_dict(), rc


def cox_fit(data: SurvData, beta=None, allow_not_converged=True, **kw):
    """Penalised Cox CCD fit.  ``beta`` (float64, host or device) is the warm
    start and receives the estimate.  Returns (beta, info dict, return code)."""
    return _fit(load().cox_fit, data, beta, allow_not_converged, **kw)


def fg_fit(data: SurvData, beta=None, allow_not_converged=True, **kw):
    """Penalised Fine-Gray CCD fit; same contract as cox_fit."""
    return _fit(load().fg_fit, data, beta, allow_not_converged, **kw)


def loglik_grad_hess(data: SurvData, model: str, beta, j: int, **kw):
    """(l, dl/dbeta_j, d2l/dbeta_j^2) at beta, computed on the GPU."""
    opts = make_opts(**kw)
    l, g, h = C.c_double(), C.c_double(), C.c_double()
    m = {"cox": SURV_COX, "fg": SURV_FG}[model]
    rc = load().loglik_grad_hess(C.byref(data.c), m, C.c_void_p(_ptr(beta)), int(j), C.byref(l), C.byref(g),
                                 C.byref(h), C.byref(opts))
    _check(rc)
    return l.value, g.value, h.value


def loglik_grad_hess_noalloc(data: SurvData, model: str, beta, j: int, precision="f32c", stream=None):
    """Same as loglik_grad_hess through the allocation-free entry point: the
    library uses its fixed device scratch array and allocates nothing (the
    cohort must already be on the GPU)."""
    l, g, h = C.c_double(), C.c_double(), C.c_double()
    m = {"cox": SURV_COX, "fg": SURV_FG}[model]
    rc = load().loglik_grad_hess_noalloc(C.byref(data.c), m, C.c_void_p(_ptr(beta)), int(j), C.byref(l),
                                         C.byref(g), C.byref(h), SURV_PREC[precision], _stream(stream))
    _check(rc)
    return l.value, g.value, h.value


def cox_lambda_max(data: SurvData, penalty_factor=None, stream=None):
    """Smallest L1 strength whose Cox optimum is beta = 0 (computed on the GPU)."""
    v = C.c_double()
    _check(load().cox_lambda_max(C.byref(data.c), C.c_void_p(_ptr(penalty_factor)), C.byref(v), _stream(stream)))
    return v.value


def cox_cv_path(data: SurvData, fold_id, nfolds: int, lambdas, penalty="l1", ctas_per_fit=0,
                allow_not_converged=True, **kw):
    """Cross-validated Cox penalty path: nlambda x nfolds fits in one batched
    schedule.  ``fold_id`` int8 [n] (host or device) in data order,
    ``lambdas`` float64 (host).  Returns a dict with beta [nlambda, nfolds, p],
    heldout [nlambda, nfolds], cv_mean [nlambda], sweeps [nlambda, nfolds]
    (numpy), info and the return code."""
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    L = int(lam.shape[0])
    F = L * int(nfolds)
    opts = make_opts(penalty=penalty, **kw)
    beta = np.empty((L, int(nfolds), data.p), np.float64)
    held = np.empty((L, int(nfolds)), np.float64)
    mean = np.empty(L, np.float64)
    sweeps = np.empty((L, int(nfolds)), np.int32)
    info = surv_cv_info()
    rc = load().cox_cv_path(C.byref(data.c), C.c_void_p(_ptr(fold_id)), int(nfolds), C.c_void_p(_ptr(lam)), L,
                            C.byref(opts), int(ctas_per_fit), C.c_void_p(_ptr(beta)), C.c_void_p(_ptr(held)),
                            C.c_void_p(_ptr(mean)), C.c_void_p(_ptr(sweeps)), C.byref(info))
    _check(rc, (SURV_OK, SURV_W_NOT_CONVERGED) if allow_not_converged else (SURV_OK,))
    assert F == info.nfits
    return {"beta": beta, "heldout": held, "cv_mean": mean, "sweeps": sweeps, "info": info.as_dict(), "rc": rc}


def surv_sort_desc(time, perm=None, stream=None):
    """Stable decreasing-time order of ``time`` (int32); returns ``perm``."""
    n = int(time.shape[0])
    if perm is None:
        if hasattr(time, "data_ptr"):
            import torch
            perm = torch.empty(n, dtype=torch.int32, device=time.device)
        else:
            perm = np.empty(n, dtype=np.int32)
    rc = load().surv_sort_desc(C.c_void_p(_ptr(time)), n, C.c_void_p(_ptr(perm)), _stream(stream))
    _check(rc)
    return perm


def surv_groups(time, status, stream=None):
    """Tie-group table of sorted data: (gend int32[K], dk int32[K], Gk float64[K]) as numpy arrays."""
    n = int(time.shape[0])
    K = C.c_int64()
    lib = load()
    st = _stream(stream)
    _check(lib.surv_groups(C.c_void_p(_ptr(time)), C.c_void_p(_ptr(status)), n, 0, C.byref(K), None, None, None, st))
    k = K.value
    gend = np.empty(k, np.int32)
    dk = np.empty(k, np.int32)
    Gk = np.empty(k, np.float64)
    if k:
        _check(lib.surv_groups(C.c_void_p(_ptr(time)), C.c_void_p(_ptr(status)), n, k, C.byref(K),
                               C.c_void_p(gend.ctypes.data), C.c_void_p(dk.ctypes.data),
                               C.c_void_p(Gk.ctypes.data), st))
    return gend, dk, Gk


def strerror(code: int) -> str:
    return load().surv_strerror(code).decode()


# ----------------------------------------------------------- differentiable form
def _nll_data(X, time, status, ncols):
    n, p = int(X.shape[0]), int(X.shape[1])
    return surv_nll_data(n, p, int(ncols), C.c_void_p(_ptr(time)), C.c_void_p(_ptr(status)), C.c_void_p(_ptr(X)))


def cox_nll_forward(X, time, status, B, workspace, stream=None):
    """NLL per column of B (float64, device) through cox_nll_forward.  X:
    bfloat16 (n, p) row-major; B: float32 (p, C); time int32, status int8,
    all CUDA tensors."""
    import torch
    nll = torch.empty(int(B.shape[1]), dtype=torch.float64, device=B.device)
    d = _nll_data(X, time, status, B.shape[1])
    _check(load().cox_nll_forward(C.byref(d), C.c_void_p(_ptr(B)), C.c_void_p(_ptr(nll)), _stream(stream),
                                  workspace.handle))
    return nll


def cox_nll_backward(X, time, status, grad_nll, ncols, workspace, stream=None):
    """dNLL/dB weighted by grad_nll (float64 [C], device) at the B of the
    last cox_nll_forward on `workspace`; float32 (p, C)."""
    import torch
    gB = torch.empty((int(X.shape[1]), int(ncols)), dtype=torch.float32, device=grad_nll.device)
    d = _nll_data(X, time, status, ncols)
    _check(load().cox_nll_backward(C.byref(d), C.c_void_p(_ptr(grad_nll)), C.c_void_p(_ptr(gB)), _stream(stream),
                                   workspace.handle))
    return gB


# Idle workspaces of the autograd function, per (device, stream): a forward
# leases one and keeps it (eta and the risk-set sums live there) until its
# autograd node is freed, which returns it for the next forward on the same
# stream.  Reuse is ordered by the stream, and a training loop allocates
# device memory only while the pool grows (once per graph alive at a time).
_WS_POOL = {}


class _WorkspaceLease:
    def __init__(self, key):
        idle = _WS_POOL.setdefault(key, [])
        self.key = key
        self.ws = idle.pop() if idle else Workspace()

    def __del__(self):
        ws, self.ws = getattr(self, "ws", None), None
        if ws is not None:
            try:
                _WS_POOL.setdefault(self.key, []).append(ws)
            except Exception:
                pass


def _cox_nll_function():
    import torch

    class CoxNLL(torch.autograd.Function):
        """NLL_b(eta = X B) per column b as a differentiable function of B
        (X bfloat16 (n, p), time int32 and status int8 sorted by decreasing
        time, all on the GPU).  Forward and backward run in libsurvgpu; each
        forward holds a pooled workspace for its backward (see
        _WorkspaceLease), so steady-state training steps allocate nothing."""

        @staticmethod
        def forward(ctx, B, X, time, status):
            B = B.contiguous()
            lease = _WorkspaceLease((B.device.index, torch.cuda.current_stream(B.device).cuda_stream))
            nll = cox_nll_forward(X, time, status, B, lease.ws)
            ctx.lease, ctx.X, ctx.time, ctx.status, ctx.ncols = lease, X, time, status, int(B.shape[1])
            return nll

        @staticmethod
        def backward(ctx, grad_out):
            g = grad_out.detach().to(torch.float64).contiguous()
            gB = cox_nll_backward(ctx.X, ctx.time, ctx.status, g, ctx.ncols, ctx.lease.ws)
            return gB, None, None, None

    return CoxNLL


_COX_NLL = None


def cox_nll(B, X, time, status):
    """Differentiable Cox NLL per column of B (autograd; see CoxNLL)."""
    global _COX_NLL
    if _COX_NLL is None:
        _COX_NLL = _cox_nll_function()
    return _COX_NLL.apply(B, X, time, status)
