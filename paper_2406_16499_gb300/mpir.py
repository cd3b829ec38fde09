"""Thin ctypes binding of libmpir.so (include/mpir.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  The C names are kept; tensors are passed as raw device pointers.
Matrices must be FP64 and column-major (stride(0) == 1); ``colmajor`` makes
such a tensor.  The library is loaded from the in-tree build; if it is
missing and cannot be built, importing the solver raises -- there is no CPU
fallback.
"""
import ctypes
import os

from . import build as _build

_lib = None

PREC = {"bf16": 0, "tf32": 1, "fp32": 2, "fp64": 3, "auto": 4}
REFINE = {"classical": 0, "gmres": 1, "direct": 2, "gmres_left": 3}
STATUS = {0: "ok", 1: "singular R", 2: "singular T", 3: "not converged", 4: "non-finite",
          5: "unsupported", 6: "cuda error", 7: "device timeout"}


class MpirError(RuntimeError):
    pass


class Opts(ctypes.Structure):
    _fields_ = [("fact", ctypes.c_int), ("refine", ctypes.c_int), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("restart", ctypes.c_int), ("inner_maxit", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("escalate", ctypes.c_int), ("resid_dd", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("fact_used", ctypes.c_int), ("refine_used", ctypes.c_int), ("escalated", ctypes.c_int),
                ("stop_ratio", ctypes.c_double * 3), ("time_ms", ctypes.c_double * 6)]

    def as_dict(self):
        return dict(status=self.status, iters=self.iters, inner_iters=self.inner_iters,
                    fact_used=self.fact_used, refine_used=self.refine_used, escalated=self.escalated,
                    stop_ratio=list(self.stop_ratio), time_ms=list(self.time_ms))


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIG = {
    "mpir_version": ([], ctypes.c_char_p),
    "mpir_default_opts": ([ctypes.POINTER(Opts)], None),
    "mpir_create": ([ctypes.POINTER(_P), _I, _P], _I),
    "mpir_destroy": ([_P], _I),
    "mpir_set_stream": ([_P, _P], _I),
    "mpir_set_workspace": ([_P, _P, ctypes.c_size_t], _I),
    "mpir_lse_workspace_size": ([_I, _I, _I, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_size_t)], _I),
    "mpir_gls_workspace_size": ([_I, _I, _I, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_size_t)], _I),
    "mpir_last_error": ([_P], ctypes.c_char_p),
    "lse_solve": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P, _P, ctypes.POINTER(Opts),
                   ctypes.POINTER(Info)], _I),
    "gls_solve": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P, ctypes.POINTER(Opts),
                   ctypes.POINTER(Info)], _I),
    "zlse_solve": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P, _P, ctypes.POINTER(Opts),
                    ctypes.POINTER(Info)], _I),
    "zgls_solve": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P, ctypes.POINTER(Opts),
                    ctypes.POINTER(Info)], _I),
    "lse_solve_batched": ([_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Opts),
                           ctypes.POINTER(Info)], _I),
    "gls_solve_batched": ([_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Opts),
                           ctypes.POINTER(Info)], _I),
    "zlse_solve_batched": ([_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Opts),
                            ctypes.POINTER(Info)], _I),
    "zgls_solve_batched": ([_P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Opts),
                            ctypes.POINTER(Info)], _I),
    "mpir_lse_factor": ([_P, _I, _I, _I, _P, _I, _P, _I, _I], _I),
    "mpir_gls_factor": ([_P, _I, _I, _I, _P, _I, _P, _I, _I], _I),
    "mpir_get_RT": ([_P, _P, _I, _P, _I], _I),
    "mpir_apply_factor": ([_P, _I, _I, _P], _I),
    "mpir_lse_initial": ([_P, _P, _P, _P], _I),
    "mpir_gls_initial": ([_P, _P, _P, _P], _I),
    "mpir_lse_multipliers": ([_P, _P, _I, _P, _P, _P, _P], _I),
    "mpir_gls_multipliers": ([_P, _P, _P], _I),
    "mpir_lse_residual": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P], _I),
    "mpir_gls_residual": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P], _I),
    "mpir_lse_correction": ([_P, _P, _P, _P, _P, _P, _P], _I),
    "mpir_gls_correction": ([_P, _P, _P, _P, _P, _P, _P], _I),
    "mpir_larfb": ([_P, _I, _I, _I, _I, _P, _I, _P, _I, _P, _I], _I),
    "mpir_lse_bd_apply": ([_P, _P, _I, _P, _I, ctypes.c_double, ctypes.c_double, _I, _P, _P], _I),
    "mpir_gls_bd_apply": ([_P, _P, _I, _P, _I, ctypes.c_double, ctypes.c_double, _I, _P, _P], _I),
    "mpir_gls_residual_noalloc": ([_I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P], _I),
    "mpir_batched_set_shape": ([_P, _I], _I),
    "mpir_batched_get_shape": ([_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_I)], _I),
    "mpir_lse_features": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P, _P], _I),
    "mpir_gls_features": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _P, _P], _I),
    "mpir_mlp_param_count": ([], _I),
    "mpir_mlp_forward": ([_P, _P, _P, _I, _P], _I),
    "mpir_mlp_train_step": ([_P, _P, _P, _P, _I, ctypes.c_float, _P, _P, _I, _P, _P], _I),
    "mpir_selector_set": ([_P, _P, _P, _P], _I),
    "mpir_profile": ([_I], _I),
    "mpir_profile_read": ([_P, _P, _I], _I),
    "mpir_launch_count": ([_I], ctypes.c_longlong),
    "mpir_kernel_kind_name": ([_I], ctypes.c_char_p),
}

NKINDS = 15


def profile(enable):
    """Enable (and clear) or disable per-launch event timing."""
    lib().mpir_profile(1 if enable else 0)


def profile_read():
    """{kind name: (ms, launches)} of the launches timed since profile(True)."""
    ms = (ctypes.c_double * NKINDS)()
    cnt = (ctypes.c_longlong * NKINDS)()
    lib().mpir_profile_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(cnt, ctypes.c_void_p), NKINDS)
    return {lib().mpir_kernel_kind_name(k).decode(): (ms[k], cnt[k]) for k in range(NKINDS)}


def launch_count(kind=-1):
    return int(lib().mpir_launch_count(kind))


def gls_residual_noalloc(W, V, d, x, y, z, f1, f2, f3, norms2=None, stream=None):
    """mpir_gls_residual_noalloc on CUDA tensors (no handle, no allocation
    inside the library); norms2: optional CUDA tensor of 6 doubles."""
    import torch
    n, m = W.shape
    p = V.shape[1]
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    return int(lib().mpir_gls_residual_noalloc(n, m, p, ptr(W), ld(W), ptr(V), ld(V), ptr(d), ptr(x), ptr(y),
                                               ptr(z), ptr(f1), ptr(f2), ptr(f3), ptr(norms2),
                                               ctypes.c_void_p(stream)))


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libmpir.so; build it in-tree first if it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise MpirError("libmpir.so not found at %s (run __graft_entry__.build())" % _build.LIB)
    L = ctypes.CDLL(_build.LIB)
    for name, (args, res) in _SIG.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def exported_symbols():
    return list(_SIG.keys())


_CTYPE = {"f64": "torch.float64", "f32": "torch.float32", "i32": "torch.int32", "c128": "torch.complex128"}


def ptr(t, ctype="f64"):
    """Device pointer of a CUDA tensor whose element type matches the C
    argument (ctype 'f64' for double*, 'f32' for float*, 'i32' for int*);
    None or an empty tensor -> NULL, an int is taken as a raw address.  A
    host tensor or another element type raises: the kernels would read past
    the end of the buffer."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise MpirError("expected a CUDA tensor, got one on %s" % t.device)
    if str(t.dtype) != _CTYPE[ctype]:
        raise MpirError("expected %s elements for this argument, got %s" % (_CTYPE[ctype], t.dtype))
    if t.numel() == 0:
        return None
    return t.data_ptr()


def colmajor(t):
    """Column-major copy of a 2-D tensor (stride(0) == 1)."""
    return t.t().contiguous().t()


def ld(t):
    """Leading dimension of a column-major matrix tensor."""
    if t.dim() != 2:
        raise MpirError("matrix must be 2-D")
    rows, cols = t.shape
    if rows == 0 or cols == 0:
        return max(1, rows)
    if t.stride(0) != 1 and rows > 1:
        raise MpirError("matrix must be column-major (stride(0) == 1)")
    return max(1, rows, t.stride(1) if cols > 1 else rows)


def make_opts(fact="fp32", refine="classical", tol=0.0, maxit=0, escalate=True, **kw):
    o = Opts()
    lib().mpir_default_opts(ctypes.byref(o))
    o.fact = PREC[fact] if isinstance(fact, str) else int(fact)
    o.refine = REFINE[refine] if isinstance(refine, str) else int(refine)
    if tol:
        o.tol = tol
    if maxit:
        o.maxit = maxit
    o.escalate = 1 if escalate else 0
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class LseBatch:
    """The host-side argument arrays of lse_solve_batched, built once for a
    list of problems (dicts of column-major FP64 device tensors A, B, b, d)
    and their output vectors, so that repeated solves skip the marshalling."""

    def __init__(self, probs, xs, ctype="f64"):
        import numpy as np
        cnt = len(probs)
        self.count = cnt
        self.keep = (list(probs), list(xs))       # the tensors must outlive the arrays
        sz = max(cnt, 1)
        ints = np.zeros((5, sz), dtype=np.int32)
        ptrs = np.zeros((5, sz), dtype=np.uint64)
        for i, pr in enumerate(probs):
            A, B = pr["A"], pr["B"]
            ints[0, i], ints[1, i] = A.shape
            ints[2, i] = B.shape[0]
            ints[3, i] = ld(A)
            ints[4, i] = ld(B) if B.shape[0] else 1
            ptrs[0, i] = ptr(A, ctype) or 0
            ptrs[1, i] = ptr(B, ctype) or 0
            ptrs[2, i] = ptr(pr["b"], ctype) or 0
            ptrs[3, i] = ptr(pr["d"], ctype) or 0
            ptrs[4, i] = ptr(xs[i], ctype) or 0
        self._ints, self._ptrs = np.ascontiguousarray(ints), np.ascontiguousarray(ptrs)
        ip = lambda k: ctypes.c_void_p(self._ints[k].ctypes.data)
        pp = lambda k: ctypes.c_void_p(self._ptrs[k].ctypes.data)
        # (m, n, p, A, lda, B, ldb, b, d, x) in the C argument order
        self.args = (ip(0), ip(1), ip(2), pp(0), ip(3), pp(1), ip(4), pp(2), pp(3), pp(4))
        self.infos = (Info * sz)()


class GlsBatch:
    """The host-side argument arrays of gls_solve_batched for a list of GLS
    problems (dicts of column-major FP64 device tensors W (n x m), V (n x p),
    d) and their output vectors xs (m), ys (p)."""

    def __init__(self, probs, xs, ys, ctype="f64"):
        import numpy as np
        cnt = len(probs)
        self.count = cnt
        self.keep = (list(probs), list(xs), list(ys))
        sz = max(cnt, 1)
        ints = np.zeros((5, sz), dtype=np.int32)
        ptrs = np.zeros((5, sz), dtype=np.uint64)
        for i, pr in enumerate(probs):
            W, V = pr["W"], pr["V"]
            ints[0, i], ints[1, i] = W.shape
            ints[2, i] = V.shape[1]
            ints[3, i] = ld(W)
            ints[4, i] = ld(V)
            ptrs[0, i] = ptr(W, ctype) or 0
            ptrs[1, i] = ptr(V, ctype) or 0
            ptrs[2, i] = ptr(pr["d"], ctype) or 0
            ptrs[3, i] = ptr(xs[i], ctype) or 0
            ptrs[4, i] = ptr(ys[i], ctype) or 0
        self._ints, self._ptrs = np.ascontiguousarray(ints), np.ascontiguousarray(ptrs)
        ip = lambda k: ctypes.c_void_p(self._ints[k].ctypes.data)
        pp = lambda k: ctypes.c_void_p(self._ptrs[k].ctypes.data)
        # (n, m, p, W, ldw, V, ldv, d, x, y) in the C argument order
        self.args = (ip(0), ip(1), ip(2), pp(0), ip(3), pp(1), ip(4), pp(2), pp(3), pp(4))
        self.infos = (Info * sz)()


class Handle:
    """Owns an mpir_handle bound to a device and a CUDA stream (the current
    torch stream by default)."""

    def __init__(self, device=None, stream=None):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.h = ctypes.c_void_p()
        rc = lib().mpir_create(ctypes.byref(self.h), int(device), ctypes.c_void_p(stream))
        if rc != 0:
            raise MpirError("mpir_create failed (%d)" % rc)

    def close(self):
        if self.h:
            lib().mpir_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self):
        return lib().mpir_last_error(self.h).decode()

    def check(self, rc, what):
        if rc < 0:
            raise MpirError("%s: illegal argument %d (%s)" % (what, -rc, self.last_error()))
        if rc in (5, 6, 7):
            raise MpirError("%s: %s (%s)" % (what, STATUS.get(rc, rc), self.last_error()))
        return rc

    # ---- full solves ------------------------------------------------------
    def lse_solve(self, A, B, b, d, x, r=None, v=None, opts=None):
        m, n = A.shape
        p = B.shape[0]
        info = Info()
        o = opts if opts is not None else make_opts()
        rc = lib().lse_solve(self.h, m, n, p, ptr(A), ld(A), ptr(B), ld(B) if p else 1, ptr(b), ptr(d),
                             ptr(x), ptr(r), ptr(v), ctypes.byref(o), ctypes.byref(info))
        return self.check(rc, "lse_solve"), info

    def lse_solve_batched(self, probs, xs=None, opts=None):
        """probs: an LseBatch, or a sequence of dicts with device tensors A, B,
        b, d (column-major FP64) together with xs, the device output vectors.
        Returns (status, [Info])."""
        batch = probs if isinstance(probs, LseBatch) else LseBatch(probs, xs)
        o = opts if opts is not None else make_opts()
        rc = lib().lse_solve_batched(self.h, batch.count, *batch.args, ctypes.byref(o),
                                     ctypes.cast(batch.infos, ctypes.POINTER(Info)))
        return self.check(rc, "lse_solve_batched"), list(batch.infos)[:batch.count]

    def gls_solve_batched(self, probs, xs=None, ys=None, opts=None):
        """probs: a GlsBatch, or a sequence of dicts with device tensors W, V,
        d together with xs, ys.  Returns (status, [Info])."""
        batch = probs if isinstance(probs, GlsBatch) else GlsBatch(probs, xs, ys)
        o = opts if opts is not None else make_opts()
        rc = lib().gls_solve_batched(self.h, batch.count, *batch.args, ctypes.byref(o),
                                     ctypes.cast(batch.infos, ctypes.POINTER(Info)))
        return self.check(rc, "gls_solve_batched"), list(batch.infos)[:batch.count]

    def zlse_solve_batched(self, probs, xs, opts=None):
        """Complex LSE batch: dicts of column-major complex128 device tensors
        A, B, b, d and the complex128 output vectors xs."""
        batch = LseBatch(probs, xs, "c128")
        o = opts if opts is not None else make_opts()
        rc = lib().zlse_solve_batched(self.h, batch.count, *batch.args, ctypes.byref(o),
                                      ctypes.cast(batch.infos, ctypes.POINTER(Info)))
        return self.check(rc, "zlse_solve_batched"), list(batch.infos)[:batch.count]

    def zgls_solve_batched(self, probs, xs, ys, opts=None):
        """Complex GLS batch: dicts of complex128 device tensors W, V, d and
        the outputs xs, ys."""
        batch = GlsBatch(probs, xs, ys, "c128")
        o = opts if opts is not None else make_opts()
        rc = lib().zgls_solve_batched(self.h, batch.count, *batch.args, ctypes.byref(o),
                                      ctypes.cast(batch.infos, ctypes.POINTER(Info)))
        return self.check(rc, "zgls_solve_batched"), list(batch.infos)[:batch.count]

    # ---- learned selector ------------------------------------------------
    def lse_features(self, A, B, b, d, s, out):
        p = B.shape[0]
        return self.check(lib().mpir_lse_features(self.h, A.shape[0], A.shape[1], p, ptr(A), ld(A), ptr(B),
                                                  ld(B) if p else 1, ptr(b), ptr(d), ptr(s), ptr(out, "f32")),
                          "mpir_lse_features")

    def gls_features(self, W, V, d, s, out):
        n, m = W.shape
        return self.check(lib().mpir_gls_features(self.h, n, m, V.shape[1], ptr(W), ld(W), ptr(V), ld(V), ptr(d),
                                                  ptr(s), ptr(out, "f32")), "mpir_gls_features")

    def mlp_forward(self, params, X, prob):
        return self.check(lib().mpir_mlp_forward(self.h, ptr(params, "f32"), ptr(X, "f32"), X.shape[0],
                                                 ptr(prob, "f32")),
                          "mpir_mlp_forward")

    def mlp_train_step(self, params, m, v, step, lr, X, y, grad=None, loss=None):
        return self.check(lib().mpir_mlp_train_step(self.h, ptr(params, "f32"), ptr(m, "f32"), ptr(v, "f32"),
                                                    int(step), float(lr), ptr(X, "f32"), ptr(y, "i32"), X.shape[0],
                                                    ptr(grad, "f32"), ptr(loss, "f32")),
                          "mpir_mlp_train_step")

    def selector_set(self, params, mean, scale):
        """params, mean, scale: host float32 numpy arrays (None removes)."""
        import numpy as np
        if params is None:
            return self.check(lib().mpir_selector_set(self.h, None, None, None), "mpir_selector_set")
        P = np.ascontiguousarray(params, dtype=np.float32)
        mu = np.ascontiguousarray(mean, dtype=np.float32)
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        return self.check(lib().mpir_selector_set(self.h, P.ctypes.data, mu.ctypes.data, sc.ctypes.data),
                          "mpir_selector_set")

    def batched_set_shape(self, group=0):
        """Force the batched group size (512/256/128/64) or 0 for autotuning."""
        return self.check(lib().mpir_batched_set_shape(self.h, int(group)), "mpir_batched_set_shape")

    def batched_get_shape(self, bucket):
        g, sm, cnt = ctypes.c_int(), ctypes.c_size_t(), ctypes.c_int()
        self.check(lib().mpir_batched_get_shape(self.h, bucket, ctypes.byref(g), ctypes.byref(sm), ctypes.byref(cnt)),
                   "mpir_batched_get_shape")
        return dict(group=g.value, smem=sm.value, problems=cnt.value)

    def gls_solve(self, W, V, d, x, y, z=None, opts=None):
        n, m = W.shape
        p = V.shape[1]
        info = Info()
        o = opts if opts is not None else make_opts()
        rc = lib().gls_solve(self.h, n, m, p, ptr(W), ld(W), ptr(V), ld(V), ptr(d), ptr(x), ptr(y),
                             ptr(z), ctypes.byref(o), ctypes.byref(info))
        return self.check(rc, "gls_solve"), info

    def zlse_solve(self, A, B, b, d, x, r=None, v=None, opts=None):
        """Complex LSE: complex128 device tensors, A and B column-major."""
        m, n = A.shape
        p = B.shape[0]
        info = Info()
        o = opts if opts is not None else make_opts()
        rc = lib().zlse_solve(self.h, m, n, p, ptr(A, "c128"), ld(A), ptr(B, "c128"), ld(B) if p else 1,
                              ptr(b, "c128"), ptr(d, "c128"), ptr(x, "c128"), ptr(r, "c128"), ptr(v, "c128"),
                              ctypes.byref(o), ctypes.byref(info))
        return self.check(rc, "zlse_solve"), info

    def zgls_solve(self, W, V, d, x, y, z=None, opts=None):
        """Complex GLS: complex128 device tensors, W and V column-major."""
        n, m = W.shape
        p = V.shape[1]
        info = Info()
        o = opts if opts is not None else make_opts()
        rc = lib().zgls_solve(self.h, n, m, p, ptr(W, "c128"), ld(W), ptr(V, "c128"), ld(V), ptr(d, "c128"),
                              ptr(x, "c128"), ptr(y, "c128"), ptr(z, "c128"), ctypes.byref(o), ctypes.byref(info))
        return self.check(rc, "zgls_solve"), info

    # ---- step-level ---------------------------------------------------------
    def lse_factor(self, A, B, fact="fp32"):
        m, n = A.shape
        p = B.shape[0]
        rc = lib().mpir_lse_factor(self.h, m, n, p, ptr(A), ld(A), ptr(B), ld(B) if p else 1, PREC[fact])
        return self.check(rc, "mpir_lse_factor")

    def gls_factor(self, W, V, fact="fp32"):
        n, m = W.shape
        p = V.shape[1]
        rc = lib().mpir_gls_factor(self.h, n, m, p, ptr(W), ld(W), ptr(V), ld(V), PREC[fact])
        return self.check(rc, "mpir_gls_factor")

    def get_RT(self, R, T):
        return self.check(lib().mpir_get_RT(self.h, ptr(R), ld(R) if R is not None else 1, ptr(T),
                                             ld(T) if T is not None else 1), "mpir_get_RT")

    def apply_factor(self, which, trans, vec):
        return self.check(lib().mpir_apply_factor(self.h, 0 if which == "Q" else 1, 1 if trans else 0,
                                                  ptr(vec)), "mpir_apply_factor")

    def lse_initial(self, b, d, x):
        return self.check(lib().mpir_lse_initial(self.h, ptr(b), ptr(d), ptr(x)), "mpir_lse_initial")

    def gls_initial(self, d, x, y):
        return self.check(lib().mpir_gls_initial(self.h, ptr(d), ptr(x), ptr(y)), "mpir_gls_initial")

    def lse_multipliers(self, A, b, x, r, v):
        return self.check(lib().mpir_lse_multipliers(self.h, ptr(A), ld(A), ptr(b), ptr(x), ptr(r), ptr(v)),
                          "mpir_lse_multipliers")

    def gls_multipliers(self, y, z):
        return self.check(lib().mpir_gls_multipliers(self.h, ptr(y), ptr(z)), "mpir_gls_multipliers")

    def lse_residual(self, A, B, b, d, x, r, v, f1, f2, f3, norms=None):
        m, n = A.shape
        p = B.shape[0]
        buf = (ctypes.c_double * 8)()
        rc = lib().mpir_lse_residual(self.h, m, n, p, ptr(A), ld(A), ptr(B), ld(B) if p else 1, ptr(b),
                                     ptr(d), ptr(x), ptr(r), ptr(v), ptr(f1), ptr(f2), ptr(f3),
                                     ctypes.cast(buf, ctypes.c_void_p))
        self.check(rc, "mpir_lse_residual")
        return list(buf)

    def gls_residual(self, W, V, d, x, y, z, f1, f2, f3):
        n, m = W.shape
        p = V.shape[1]
        buf = (ctypes.c_double * 8)()
        rc = lib().mpir_gls_residual(self.h, n, m, p, ptr(W), ld(W), ptr(V), ld(V), ptr(d), ptr(x), ptr(y),
                                     ptr(z), ptr(f1), ptr(f2), ptr(f3), ctypes.cast(buf, ctypes.c_void_p))
        self.check(rc, "mpir_gls_residual")
        return list(buf)

    def lse_correction(self, f1, f2, f3, dr, dv, dx):
        return self.check(lib().mpir_lse_correction(self.h, ptr(f1), ptr(f2), ptr(f3), ptr(dr), ptr(dv),
                                                    ptr(dx)), "mpir_lse_correction")

    def larfb(self, V, T, C, trans=True, prec="fp32"):
        """C <- (I - V X V^T) C on the tensor cores (FP32 tensors; V M x K
        panel, T K x K with leading dimension 128, C M x N column-major)."""
        M, K = V.shape
        N = C.shape[1]
        rc = lib().mpir_larfb(self.h, PREC[prec], M, N, K, ptr(V, "f32"), ld(V), ptr(T, "f32"), 1 if trans else 0,
                              ptr(C, "f32"), ld(C))
        return self.check(rc, "mpir_larfb")

    BD_WHICH = {"F": 0, "Ml": 1, "Mr": 2, "op": 3, "M": 4, "left_op": 5}

    def lse_bd_apply(self, A, B, alpha, beta, which, vin, vout):
        """F~, M_l, M_r or M_l F~ M_r (Sec. 5.2), or the left preconditioner M
        and M F~ (Sec. 5.1), on [m; p; n] vectors."""
        p = B.shape[0]
        return self.check(lib().mpir_lse_bd_apply(self.h, ptr(A), ld(A), ptr(B), ld(B) if p else 1, float(alpha),
                                                  float(beta), self.BD_WHICH[which], ptr(vin), ptr(vout)),
                          "mpir_lse_bd_apply")

    def gls_bd_apply(self, W, V, alpha, beta, which, vin, vout):
        """F~, M_l, M_r or M_l F~ M_r (Sec. 5.3), or the left preconditioner M
        and M F~ (Sec. 5.1), on [p; n; m] vectors."""
        return self.check(lib().mpir_gls_bd_apply(self.h, ptr(W), ld(W), ptr(V), ld(V), float(alpha), float(beta),
                                                  self.BD_WHICH[which], ptr(vin), ptr(vout)),
                          "mpir_gls_bd_apply")

    def gls_correction(self, f1, f2, f3, dy, dz, dx):
        return self.check(lib().mpir_gls_correction(self.h, ptr(f1), ptr(f2), ptr(f3), ptr(dy), ptr(dz),
                                                    ptr(dx)), "mpir_gls_correction")
