"""Python binding of libtqr (include/tqr.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Matrices are
torch tensors on the GPU holding FP64 data in column-major order, i.e. a
tensor ``A`` of shape (m, n) with ``A.stride() == (1, m)`` (see
:func:`colmajor`).  Device work is enqueued on the current torch stream unless
a stream is given.  Errors raise :class:`TqrError`; the library must be built
(``paper_1104_4475_gb300.build.build()``) -- there is no fallback.
"""

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

GEQRT, UNMQR, TTQRT, TTMQR, TSQRT, TSMQR = range(6)
FLAT_TS, FLAT_TT, SAMEH_KUCK, BINARY, FIBONACCI, GREEDY, PLASMA, ASAP, GRASAP, PLASMA_TS = range(10)
TREES = {"flat_ts": FLAT_TS, "flat_tt": FLAT_TT, "sameh_kuck": SAMEH_KUCK, "binary": BINARY,
         "fibonacci": FIBONACCI, "greedy": GREEDY, "plasma": PLASMA, "asap": ASAP, "grasap": GRASAP,
         "plasma_ts": PLASMA_TS}

TQR_ERR_INVALID_LIST = -100
TQR_ERR_TIMEOUT = -101
TQR_ERR_NONFINITE = -102
TQR_ERR_CUDA = -103
TQR_ERR_NOMEM = -104
TQR_ERR_CAPACITY = -105
TQR_ERR_INTERNAL = -106
TQR_ERR_UNSUPPORTED = -107
TQR_ERR_TOO_LARGE = -108


class TqrError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, tqr_strerror(code), code))


TQR_FP64, TQR_SPLIT_TF32, TQR_TF32 = 0, 1, 2


class tqr_lstsq_info(ctypes.Structure):
    _fields_ = [("refine_iterations", ctypes.c_int32), ("cgls_iterations", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("status", ctypes.c_int32), ("backward_error", ctypes.c_double),
                ("residual_norm", ctypes.c_double), ("factor_seconds", ctypes.c_double),
                ("solve_seconds", ctypes.c_double)]


class tqr_batch_info(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("strip", ctypes.c_int32), ("n_tasks", ctypes.c_int64),
                ("n_edges", ctypes.c_int64), ("max_critical_path", ctypes.c_int64), ("flops", ctypes.c_double),
                ("n_fused", ctypes.c_int32), ("f32", ctypes.c_int32)]


class tqr_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nb", ctypes.c_int32), ("ib", ctypes.c_int32),
                ("p", ctypes.c_int32), ("q", ctypes.c_int32), ("tree", ctypes.c_int32), ("BS", ctypes.c_int32),
                ("ts", ctypes.c_int32), ("strip", ctypes.c_int32), ("n_elims", ctypes.c_int64),
                ("n_tile_tasks", ctypes.c_int64), ("n_device_tasks", ctypes.c_int64),
                ("n_edges", ctypes.c_int64), ("critical_path", ctypes.c_int64), ("flops", ctypes.c_double)]


_lib = None


def lib():
    """The loaded libtqr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("libtqr.so is not built (run paper_1104_4475_gb300.build.build())")
        L = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        pi32, pi64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
        sig = {
            "tqr_factor": [vp, i64, i64, i32, i32, i32, i32, vp, ctypes.POINTER(vp)],
            "tqr_factor_list": [vp, i64, i64, i32, i32, pi32, i64, i32, vp, ctypes.POINTER(vp)],
            "tqr_factor_ex": [vp, i64, i64, i32, i32, i32, i32, i32, vp, ctypes.POINTER(vp)],
            "tqr_lstsq": [vp, i64, i64, vp, vp, i32, i32, i32, i32, i32, ctypes.c_double, i32, vp,
                          ctypes.POINTER(tqr_lstsq_info)],
            "tqr_apply_qt": [vp, vp, i64, i64, vp],
            "tqr_apply_q": [vp, vp, i64, i64, vp],
            "tqr_form_t": [vp, vp, vp, vp],
            "tqr_sync": [vp],
            "tqr_get_info": [vp, ctypes.POINTER(tqr_info)],
            "tqr_factor_host": [vp, i64, i64, i32, i32, i32, i32, vp, i64, vp, ctypes.POINTER(vp)],
            "tqr_factor_host_async": [vp, i64, i64, i32, i32, i32, i32, vp, i64, vp, ctypes.POINTER(vp)],
            "tqr_elimination_list": [i32, i32, i32, i32, pi32, i64, pi64],
            "tqr_validate_list": [i32, i32, pi32, i64],
            "tqr_critical_path": [i32, i32, i32, i32, pi64, pi32],
            "tqr_tasks": [i32, i32, i32, i32, pi32, pi64, i64, pi64],
            "tqr_device_graph": [i64, i64, i32, i32, i32, i32, i32, pi32, i64, pi64, pi32, pi32, i64, pi64],
            "tqr_peak_probe": [i32, i64, vp, ctypes.POINTER(ctypes.c_double)],
            "tqr_noalloc_graph": [i64, i64, i32, i32, pi32, i64, i32, i32, pi32, i64, pi64, pi32, pi32, i64, pi64],
            "tqr_set_trace": [vp, i32],
            "tqr_factor_batched": [i32, ctypes.POINTER(vp), pi64, pi64, pi32, pi32, pi32, pi32, vp,
                                   ctypes.POINTER(vp)],
            "tqr_batch_sync": [vp],
            "tqr_factor_batched_f32": [i32, ctypes.POINTER(vp), pi64, pi64, pi32, vp, ctypes.POINTER(vp)],
            "tqr_ts1_plan": [i32, pi64, pi64, pi32, i32, pi32, pi32, pi32],
            "tqr_batch_tau": [vp, i32, vp, vp],
            "tqr_get_edges": [vp, pi32, pi32, i64, pi64],
            "tqr_poison_workspace": [vp],
            "tqr_mlp_param_count": [i32],
            "tqr_mlp_forward": [vp, i32, vp, i32, vp, vp],
            "tqr_mlp_loss_grad": [vp, i32, vp, vp, i32, vp, vp, vp, vp],
            "tqr_mlp_adam_step": [vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, i32, vp],
            "tqr_batch_get_info": [vp, ctypes.POINTER(tqr_batch_info)],
            "tqr_get_trace": [vp, pi64, i64, pi64],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.tqr_set_timeout_ms.argtypes = [ctypes.c_double]
        L.tqr_set_timeout_ms.restype = ctypes.c_int
        L.tqr_inject_fault.argtypes = [ctypes.c_int]
        L.tqr_inject_fault.restype = ctypes.c_int
        L.tqr_factor_noalloc.argtypes = [vp, i64, i64, i32, i32, pi32, i64, i32, vp, vp, vp, vp]
        L.tqr_factor_noalloc.restype = ctypes.c_int
        L.tqr_batch_free.argtypes = [vp]
        L.tqr_batch_free.restype = None
        L.tqr_free.argtypes = [vp]
        L.tqr_free.restype = None
        L.tqr_release_plans.argtypes = []
        L.tqr_release_plans.restype = ctypes.c_int
        L.tqr_strerror.argtypes = [ctypes.c_int]
        L.tqr_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc, where):
    if rc != 0:
        raise TqrError(rc, where)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _colmajor_ptr(t, what, dtype=None):
    import torch
    dtype = torch.float64 if dtype is None else dtype
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or t.dim() != 2:
        raise TypeError("%s must be a 2-D %s CUDA tensor" % (what, str(dtype).replace("torch.", "")))
    m = t.shape[0]
    if t.stride(0) != 1 or (t.shape[1] > 1 and t.stride(1) < m):
        raise ValueError("%s must be column-major (stride (1, ld) with ld >= rows)" % what)
    return ctypes.c_void_p(t.data_ptr()), (t.stride(1) if t.shape[1] > 1 else max(1, m))


def colmajor(x, device="cuda"):
    """A column-major float64 CUDA tensor holding the 2-D array ``x``."""
    import torch
    a = np.asarray(x, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device).t()


def to_numpy(t):
    """A numpy copy of a (column-major) tensor."""
    return t.detach().cpu().numpy().copy()


class Factors:
    """A tqr_factors handle (owns the library-side state of one factorization)."""

    def __init__(self, ptr, A):
        self.ptr = ptr
        self.A = A

    def info(self):
        return tqr_get_info(self)

    def free(self):
        if self.ptr:
            lib().tqr_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ------------------------------------------------------------------- device
def tqr_factor(A, nb, ib, tree, BS=1, stream=None, reuse=None):
    """QR of the column-major CUDA tensor A in place (R and V); returns a
    Factors handle.  ``reuse`` (a Factors of the same shape and parameters)
    makes the call allocate nothing."""
    ptr, ld = _colmajor_ptr(A, "A")
    m, n = A.shape
    if ld != m:
        raise ValueError("A must have leading dimension m")
    h = ctypes.c_void_p(reuse.ptr if reuse is not None else None)
    _check(lib().tqr_factor(ptr, m, n, nb, ib, int(tree), BS, _stream(stream), ctypes.byref(h)), "tqr_factor")
    if reuse is not None and h.value == reuse.ptr:
        reuse.A = A
        return reuse
    return Factors(h.value, A)


def tqr_factor_ex(A, nb, ib, tree, BS=1, precision=TQR_FP64, stream=None, reuse=None):
    """tqr_factor with a choice of update arithmetic (TQR_FP64, TQR_SPLIT_TF32, TQR_TF32)."""
    ptr, ld = _colmajor_ptr(A, "A")
    m, n = A.shape
    if ld != m:
        raise ValueError("A must have leading dimension m")
    h = ctypes.c_void_p(reuse.ptr if reuse is not None else None)
    _check(lib().tqr_factor_ex(ptr, m, n, nb, ib, int(tree), BS, int(precision), _stream(stream),
                               ctypes.byref(h)), "tqr_factor_ex")
    if reuse is not None and h.value == reuse.ptr:
        reuse.A = A
        return reuse
    return Factors(h.value, A)


def tqr_lstsq(A, b, x, nb, ib, tree, BS=1, precision=TQR_FP64, tol=0.0, maxit=50, stream=None):
    """min ||A x - b||: A (m x n column-major CUDA tensor, unchanged), b (m) and
    x (n, output) CUDA float64 tensors.  Returns the info as a dict."""
    ptr, ld = _colmajor_ptr(A, "A")
    m, n = A.shape
    if ld != m:
        raise ValueError("A must have leading dimension m")
    info = tqr_lstsq_info()
    rc = lib().tqr_lstsq(ptr, m, n, _dev(b, "b", "float64", m), _dev(x, "x", "float64", n), nb, ib,
                         int(tree), BS, int(precision), float(tol), int(maxit), _stream(stream), ctypes.byref(info))
    _check(rc, "tqr_lstsq")
    return {k: getattr(info, k) for k, _ in tqr_lstsq_info._fields_}


def tqr_factor_list(A, nb, ib, elims, ts=False, stream=None, reuse=None):
    """QR with a caller-given elimination list of 0-based (i, piv, k)."""
    ptr, ld = _colmajor_ptr(A, "A")
    m, n = A.shape
    arr = np.ascontiguousarray(np.asarray(elims, dtype=np.int32).reshape(-1, 3))
    h = ctypes.c_void_p(reuse.ptr if reuse is not None else None)
    rc = lib().tqr_factor_list(ptr, m, n, nb, ib, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               arr.shape[0], 1 if ts else 0, _stream(stream), ctypes.byref(h))
    _check(rc, "tqr_factor_list")
    if reuse is not None and h.value == reuse.ptr:
        reuse.A = A
        return reuse
    return Factors(h.value, A)


def _rhs(f, B):
    ptr, ld = _colmajor_ptr(B, "B")
    m = tqr_get_info(f)["m"]
    if B.shape[0] != m:
        raise ValueError("B must have m = %d rows, not %d" % (m, B.shape[0]))
    return ptr, ld


def tqr_apply_qt(f, B, stream=None):
    """B <- Q^T B in place (B: column-major CUDA tensor with m rows)."""
    ptr, ld = _rhs(f, B)
    _check(lib().tqr_apply_qt(ctypes.c_void_p(f.ptr), ptr, ld, B.shape[1], _stream(stream)), "tqr_apply_qt")
    return B


def tqr_apply_q(f, B, stream=None):
    """B <- Q B in place."""
    ptr, ld = _rhs(f, B)
    _check(lib().tqr_apply_q(ctypes.c_void_p(f.ptr), ptr, ld, B.shape[1], _stream(stream)), "tqr_apply_q")
    return B


def tqr_form_t(f, T_geqrt=None, T_elim=None, stream=None):
    """Fill the T factor arrays (CUDA float64 tensors of p*q*ib*nb elements)."""
    i = tqr_get_info(f)
    elems = i["p"] * i["q"] * i["ib"] * i["nb"]

    def p(t, what):
        return ctypes.c_void_p(None) if t is None else _dev(t, what, "float64", elems)
    _check(lib().tqr_form_t(ctypes.c_void_p(f.ptr), p(T_geqrt, "T_geqrt"), p(T_elim, "T_elim"), _stream(stream)),
           "tqr_form_t")


class Batch:
    """A tqr_batch handle; keeps the argument arrays alive for relaunches."""

    def __init__(self, ptr, args, As):
        self.ptr, self.args, self.As = ptr, args, As

    def info(self):
        return tqr_batch_get_info(self)

    def free(self):
        if self.ptr:
            lib().tqr_batch_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _per_matrix(v, count, dtype):
    a = np.asarray(v, dtype=dtype)
    if a.ndim == 0:
        a = np.full(count, a, dtype=dtype)
    if a.shape != (count,):
        raise ValueError("per-matrix parameter must be a scalar or have one entry per matrix")
    return np.ascontiguousarray(a)


def tqr_factor_batched(As, nb, ib, tree, BS=1, stream=None, reuse=None):
    """Factor the column-major CUDA tensors in As in one launch; nb, ib, tree
    and BS are scalars or one value per matrix.  ``reuse`` (a Batch built from
    the same tensors and parameters) relaunches without allocation."""
    count = len(As)
    ptrs = (ctypes.c_void_p * count)()
    m = np.zeros(count, dtype=np.int64)
    n = np.zeros(count, dtype=np.int64)
    for c, A in enumerate(As):
        p, ld = _colmajor_ptr(A, "A[%d]" % c)
        if ld != A.shape[0]:
            raise ValueError("A[%d] must have leading dimension m" % c)
        ptrs[c] = p.value
        m[c], n[c] = A.shape
    arrs = [_per_matrix(nb, count, np.int32), _per_matrix(ib, count, np.int32),
            _per_matrix(tree, count, np.int32), _per_matrix(BS, count, np.int32)]
    P32 = ctypes.POINTER(ctypes.c_int32)
    P64 = ctypes.POINTER(ctypes.c_int64)
    h = ctypes.c_void_p(reuse.ptr if reuse is not None else None)
    rc = lib().tqr_factor_batched(count, ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), m.ctypes.data_as(P64),
                                  n.ctypes.data_as(P64), *[a.ctypes.data_as(P32) for a in arrs], _stream(stream),
                                  ctypes.byref(h))
    _check(rc, "tqr_factor_batched")
    if reuse is not None and h.value == reuse.ptr:
        return reuse
    return Batch(h.value, (ptrs, m, n, arrs), list(As))


def tqr_factor_batched_f32(As, nb, stream=None, reuse=None):
    """FP32 batch (column-major float32 CUDA tensors), FlatTree-TS with one
    tile column per matrix (n <= nb, n <= 128); nb is a scalar or one value
    per matrix."""
    import torch
    count = len(As)
    ptrs = (ctypes.c_void_p * count)()
    m = np.zeros(count, dtype=np.int64)
    n = np.zeros(count, dtype=np.int64)
    for c, A in enumerate(As):
        p, ld = _colmajor_ptr(A, "A[%d]" % c, torch.float32)
        if ld != A.shape[0]:
            raise ValueError("A[%d] must have leading dimension m" % c)
        ptrs[c] = p.value
        m[c], n[c] = A.shape
    nbs = _per_matrix(nb, count, np.int32)
    h = ctypes.c_void_p(reuse.ptr if reuse is not None else None)
    rc = lib().tqr_factor_batched_f32(count, ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)),
                                      m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      nbs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream(stream),
                                      ctypes.byref(h))
    _check(rc, "tqr_factor_batched_f32")
    if reuse is not None and h.value == reuse.ptr:
        return reuse
    return Batch(h.value, (ptrs, m, n, nbs), list(As))


def tqr_batch_tau(b, c, m, n, nb, f32=False):
    """(tau_ge, tau_el) of matrix c of a batch as host arrays of p*q*nb."""
    p, q = -(-m // nb), -(-n // nb)
    dt = np.float32 if f32 else np.float64
    tg = np.zeros(p * q * nb, dtype=dt)
    te = np.zeros(p * q * nb, dtype=dt)
    _check(lib().tqr_batch_tau(ctypes.c_void_p(b.ptr), int(c), tg.ctypes.data_as(ctypes.c_void_p),
                               te.ctypes.data_as(ctypes.c_void_p)), "tqr_batch_tau")
    return tg, te


def tqr_batch_sync(b, raise_on_error=True):
    rc = lib().tqr_batch_sync(ctypes.c_void_p(b.ptr))
    if raise_on_error:
        _check(rc, "tqr_batch_sync")
    return rc


def tqr_batch_get_info(b):
    info = tqr_batch_info()
    _check(lib().tqr_batch_get_info(ctypes.c_void_p(b.ptr), ctypes.byref(info)), "tqr_batch_get_info")
    return {k: getattr(info, k) for k, _ in tqr_batch_info._fields_}


def tqr_batch_free(b):
    b.free()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, what, dtype, numel=None, min_numel=None):
    """Pointer of a contiguous CUDA tensor of `dtype`, checked before the call
    so that a wrong dtype, device, layout or size cannot reach the library."""
    import torch
    dtype = getattr(torch, dtype)
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be a contiguous %s CUDA tensor" % (what, str(dtype).replace("torch.", "")))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, not %d" % (what, numel, t.numel()))
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError("%s must have at least %d elements, not %d" % (what, min_numel, t.numel()))
    return _ptr(t)


def _f32(t, what, numel=None, min_numel=None):
    return _dev(t, what, "float32", numel, min_numel)


def _mlp_inputs(params, X):
    if X.dim() != 2:
        raise ValueError("X must be 2-D (samples x features)")
    B, d = X.shape
    return B, d, _f32(params, "params", tqr_mlp_param_count(d)), _f32(X, "X")


def tqr_mlp_param_count(in_dim):
    n = lib().tqr_mlp_param_count(int(in_dim))
    if n < 0:
        raise TqrError(n, "tqr_mlp_param_count")
    return n


def tqr_mlp_forward(params, X, y=None, stream=None):
    """Network outputs for the rows of X (float32 CUDA tensors)."""
    import torch
    B, d, pp, px = _mlp_inputs(params, X)
    if y is None:
        y = torch.empty(B, dtype=torch.float32, device=X.device)
    _check(lib().tqr_mlp_forward(pp, d, px, B, _f32(y, "y", B), _stream(stream)), "tqr_mlp_forward")
    return y


def tqr_mlp_loss_grad(params, X, t, grad, loss, work=None, stream=None):
    import torch
    B, d, pp, px = _mlp_inputs(params, X)
    if work is None:
        work = torch.empty(B * (4 * 64 + 2), dtype=torch.float32, device=X.device)
    _check(lib().tqr_mlp_loss_grad(pp, d, px, _f32(t, "t", B), B, _f32(work, "work", min_numel=B * (4 * 64 + 2)),
                                   _f32(grad, "grad", params.numel()), _f32(loss, "loss", min_numel=1),
                                   _stream(stream)), "tqr_mlp_loss_grad")
    return work


def tqr_mlp_adam_step(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    n = params.numel()
    _check(lib().tqr_mlp_adam_step(_f32(params, "params"), _f32(grad, "grad", n), _f32(m, "m", n), _f32(v, "v", n),
                                   n, lr, beta1, beta2, eps, int(step), _stream(stream)), "tqr_mlp_adam_step")


def tqr_set_trace(f, enable=True):
    _check(lib().tqr_set_trace(ctypes.c_void_p(f.ptr), 1 if enable else 0), "tqr_set_trace")


def tqr_get_trace(f):
    """(ntasks, 8) int64: kind, i, piv, k, j*65536+strip, start ns, end ns, SM."""
    cnt = ctypes.c_int64(0)
    rc = lib().tqr_get_trace(ctypes.c_void_p(f.ptr), None, 0, ctypes.byref(cnt))
    if rc not in (0, TQR_ERR_CAPACITY):
        _check(rc, "tqr_get_trace")
    out = np.zeros((max(1, cnt.value), 8), dtype=np.int64)
    _check(lib().tqr_get_trace(ctypes.c_void_p(f.ptr), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               out.shape[0], ctypes.byref(cnt)), "tqr_get_trace")
    return out[: cnt.value]


def tqr_get_edges(f):
    """(edges, 2) int32: (u, v) dependency edges of the factorization graph."""
    cnt = ctypes.c_int64(0)
    rc = lib().tqr_get_edges(ctypes.c_void_p(f.ptr), None, None, 0, ctypes.byref(cnt))
    if rc not in (0, TQR_ERR_CAPACITY):
        _check(rc, "tqr_get_edges")
    src = np.zeros(max(1, cnt.value), dtype=np.int32)
    dst = np.zeros(max(1, cnt.value), dtype=np.int32)
    P = ctypes.POINTER(ctypes.c_int32)
    _check(lib().tqr_get_edges(ctypes.c_void_p(f.ptr), src.ctypes.data_as(P), dst.ctypes.data_as(P), src.shape[0],
                               ctypes.byref(cnt)), "tqr_get_edges")
    return np.stack([src[: cnt.value], dst[: cnt.value]], axis=1)


def tqr_poison_workspace(f):
    _check(lib().tqr_poison_workspace(ctypes.c_void_p(f.ptr)), "tqr_poison_workspace")


def tqr_sync(f, raise_on_error=True):
    rc = lib().tqr_sync(ctypes.c_void_p(f.ptr))
    if raise_on_error:
        _check(rc, "tqr_sync")
    return rc


def tqr_get_info(f):
    info = tqr_info()
    _check(lib().tqr_get_info(ctypes.c_void_p(f.ptr), ctypes.byref(info)), "tqr_get_info")
    return {k: getattr(info, k) for k, _ in tqr_info._fields_}


def tqr_free(f):
    f.free()


def tqr_release_plans():
    """Drop the cached plans no live handle uses; returns how many."""
    rc = lib().tqr_release_plans()
    if rc < 0:
        raise TqrError(rc, "tqr_release_plans")
    return rc


def tqr_factor_host(A, nb, ib, tree, BS=1, B=None, stream=None, reuse=None, wait=True):
    """End to end on host arrays: A (m x n, Fortran-ordered float64 numpy
    array) is overwritten by R and V; B (m x nrhs, Fortran order) by Q^T B.
    wait=False enqueues everything on `stream` and returns at once
    (tqr_factor_host_async): call tqr_sync on the result before reading A or
    B, and keep them alive and unmodified until then."""
    if not (isinstance(A, np.ndarray) and A.dtype == np.float64 and A.flags.f_contiguous):
        raise TypeError("A must be a Fortran-ordered float64 numpy array")
    m, n = A.shape
    bp, nrhs = None, 0
    if B is not None:
        if not (isinstance(B, np.ndarray) and B.dtype == np.float64 and B.flags.f_contiguous and B.shape[0] == m):
            raise TypeError("B must be a Fortran-ordered float64 numpy array with m rows")
        bp, nrhs = ctypes.c_void_p(B.ctypes.data), (B.shape[1] if B.ndim == 2 else 1)
    h = ctypes.c_void_p(reuse.ptr if reuse is not None else None)
    fn = lib().tqr_factor_host if wait else lib().tqr_factor_host_async
    rc = fn(ctypes.c_void_p(A.ctypes.data), m, n, nb, ib, int(tree), BS, bp, nrhs, _stream(stream), ctypes.byref(h))
    if rc != 0 and h.value and (reuse is None or h.value != reuse.ptr):
        lib().tqr_free(h)                 # a handle made by the failed call
    _check(rc, "tqr_factor_host" if wait else "tqr_factor_host_async")
    if reuse is not None and h.value == reuse.ptr:
        return reuse
    return Factors(h.value, None)


# ---------------------------------------------------------------- host only
def tqr_elimination_list(p, q, tree, BS=1):
    """0-based (i, piv, k) triplets as an (count, 3) int32 array."""
    cnt = ctypes.c_int64(0)
    rc = lib().tqr_elimination_list(p, q, int(tree), BS, None, 0, ctypes.byref(cnt))
    if rc not in (0, TQR_ERR_CAPACITY):
        _check(rc, "tqr_elimination_list")
    out = np.zeros((max(1, cnt.value), 3), dtype=np.int32)
    _check(lib().tqr_elimination_list(p, q, int(tree), BS, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      out.shape[0], ctypes.byref(cnt)), "tqr_elimination_list")
    return out[: cnt.value]


def tqr_validate_list(p, q, elims):
    arr = np.ascontiguousarray(np.asarray(elims, dtype=np.int32).reshape(-1, 3))
    return lib().tqr_validate_list(p, q, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), arr.shape[0])


def tqr_critical_path(p, q, tree, BS=1, zero_time=False):
    cp = ctypes.c_int64(0)
    zt = np.zeros(p * q, dtype=np.int32) if zero_time else None
    zp = zt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if zero_time else None
    _check(lib().tqr_critical_path(p, q, int(tree), BS, ctypes.byref(cp), zp), "tqr_critical_path")
    if zero_time:
        return cp.value, zt.reshape(p, q)
    return cp.value


def tqr_tasks(p, q, tree, BS=1):
    """(tasks (count, 5) int32: kind, i, piv, k, j; finish (count,) int64)."""
    cnt = ctypes.c_int64(0)
    rc = lib().tqr_tasks(p, q, int(tree), BS, None, None, 0, ctypes.byref(cnt))
    if rc not in (0, TQR_ERR_CAPACITY):
        _check(rc, "tqr_tasks")
    out = np.zeros((max(1, cnt.value), 5), dtype=np.int32)
    fin = np.zeros(max(1, cnt.value), dtype=np.int64)
    _check(lib().tqr_tasks(p, q, int(tree), BS, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           fin.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), out.shape[0], ctypes.byref(cnt)),
           "tqr_tasks")
    return out[: cnt.value], fin[: cnt.value]


def tqr_noalloc_graph(m, n, nb, ib, elims, ts=False, strip=64):
    """The task graph tqr_factor_noalloc builds for these arguments, built on
    the host: (tasks (ntasks, 6) int32, edges (nedges, 2) int32) as
    tqr_device_graph returns them."""
    el = np.ascontiguousarray(elims, dtype=np.int32).reshape(-1, 3)
    p32 = ctypes.POINTER(ctypes.c_int32)
    nt, ne = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib().tqr_noalloc_graph(m, n, nb, ib, el.ctypes.data_as(p32), el.shape[0], int(bool(ts)), strip, None, 0,
                                 ctypes.byref(nt), None, None, 0, ctypes.byref(ne))
    if rc not in (0, TQR_ERR_CAPACITY):
        _check(rc, "tqr_noalloc_graph")
    tasks = np.zeros((max(1, nt.value), 6), dtype=np.int32)
    src = np.zeros(max(1, ne.value), dtype=np.int32)
    dst = np.zeros(max(1, ne.value), dtype=np.int32)
    _check(lib().tqr_noalloc_graph(m, n, nb, ib, el.ctypes.data_as(p32), el.shape[0], int(bool(ts)), strip,
                                   tasks.ctypes.data_as(p32), tasks.shape[0], ctypes.byref(nt), src.ctypes.data_as(p32),
                                   dst.ctypes.data_as(p32), src.shape[0], ctypes.byref(ne)), "tqr_noalloc_graph")
    return tasks[: nt.value], np.stack([src[: ne.value], dst[: ne.value]], axis=1)


def tqr_ts1_plan(m, n, nb, f32=False):
    """The queues of the batch's persistent one-tile-column launch, planned on
    the host (see tqr.h): (order, bounds (3, 2), quarter_bytes)."""
    m = np.ascontiguousarray(m, dtype=np.int64)
    n = np.ascontiguousarray(n, dtype=np.int64)
    nb = np.ascontiguousarray(np.broadcast_to(nb, m.shape), dtype=np.int32)
    count = m.shape[0]
    order = np.zeros(max(1, count), dtype=np.int32)
    bounds = np.zeros(6, dtype=np.int32)
    q = ctypes.c_int32(0)
    p32, p64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    _check(lib().tqr_ts1_plan(count, m.ctypes.data_as(p64), n.ctypes.data_as(p64), nb.ctypes.data_as(p32),
                              int(bool(f32)), order.ctypes.data_as(p32), bounds.ctypes.data_as(p32),
                              ctypes.byref(q)), "tqr_ts1_plan")
    return order[:count], bounds.reshape(3, 2), q.value


PEAK_DFMA, PEAK_DMMA, PEAK_FFMA, PEAK_TF32 = range(4)


def tqr_peak_probe(kind, iters, stream=None):
    """Enqueue one peak-rate probe launch (see tqr.h) on `stream`; returns the
    flops it performs.  Time it with CUDA events on the same stream."""
    fl = ctypes.c_double(0.0)
    _check(lib().tqr_peak_probe(int(kind), int(iters), _stream(stream), ctypes.byref(fl)), "tqr_peak_probe")
    return fl.value


def tqr_device_graph(m, n, nb, ib, tree, BS=1, strip=64):
    """The device task graph of tqr_factor for this problem, built on the
    host: (tasks (ntasks, 6) int32: kind, i, piv, k, j, strip; edges
    (nedges, 2) int32: src, dst)."""
    nt, ne = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib().tqr_device_graph(m, n, nb, ib, int(tree), BS, strip, None, 0, ctypes.byref(nt), None, None, 0,
                                ctypes.byref(ne))
    if rc not in (0, TQR_ERR_CAPACITY):
        _check(rc, "tqr_device_graph")
    tasks = np.zeros((max(1, nt.value), 6), dtype=np.int32)
    src = np.zeros(max(1, ne.value), dtype=np.int32)
    dst = np.zeros(max(1, ne.value), dtype=np.int32)
    p32 = ctypes.POINTER(ctypes.c_int32)
    _check(lib().tqr_device_graph(m, n, nb, ib, int(tree), BS, strip, tasks.ctypes.data_as(p32), tasks.shape[0],
                                  ctypes.byref(nt), src.ctypes.data_as(p32), dst.ctypes.data_as(p32), src.shape[0],
                                  ctypes.byref(ne)), "tqr_device_graph")
    return tasks[: nt.value], np.stack([src[: ne.value], dst[: ne.value]], axis=1)


def tqr_factor_noalloc(A, nb, ib, elims, tau_geqrt, tau_elim, status, ts=False, stream=None):
    """QR of A in place without any allocation (for callers that cannot
    allocate while they factor).  elims: 0-based (i, piv, k) list;
    tau_geqrt / tau_elim: float64 CUDA tensors of p*q*nb elements (outputs);
    status: int32 CUDA tensor of one element (output).  Returns the C status."""
    ptr, ld = _colmajor_ptr(A, "A")
    m, n = A.shape
    if ld != m:
        raise ValueError("A must have leading dimension m")
    arr = np.ascontiguousarray(np.asarray(elims, dtype=np.int32).reshape(-1, 3))
    ntau = -(-m // nb) * -(-n // nb) * nb if nb > 0 else 0
    tg = _dev(tau_geqrt, "tau_geqrt", "float64", min_numel=ntau)
    te = _dev(tau_elim, "tau_elim", "float64", min_numel=ntau)
    st = _dev(status, "status", "int32", min_numel=1)
    return lib().tqr_factor_noalloc(ptr, m, n, nb, ib, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    arr.shape[0], 1 if ts else 0, tg, te, st, _stream(stream))


def tqr_set_timeout_ms(ms):
    _check(lib().tqr_set_timeout_ms(float(ms)), "tqr_set_timeout_ms")


def tqr_inject_fault(kind):
    _check(lib().tqr_inject_fault(int(kind)), "tqr_inject_fault")


def tqr_strerror(code):
    return lib().tqr_strerror(int(code)).decode()
