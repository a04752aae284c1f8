"""Python binding of libminnorm.so (include/minnorm.h): argument marshalling only.

Every function has the name of the C entry point it calls and passes plain
pointers and sizes; torch tensors supply device memory and the current CUDA
stream. All computation happens in the library's sm_103a kernels. If the
library is missing or cannot be loaded this module raises: there is no CPU
fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libminnorm.so")

OK, EINVAL, ESTATE, ENOMEM, ECUDA, ERANK, ENOCONV, EFLOOR, ETIMEOUT, ENOTSUP = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ESTATE", "ENOMEM", "ECUDA", "ERANK", "ENOCONV", "EFLOOR",
                "ETIMEOUT", "ENOTSUP"]
C64, C128 = 1, 2
FP64, MIXED = 0, 1
FLAG_TIMING, FLAG_KEEP_SKETCH = 1, 2

# every symbol include/minnorm.h declares
EXPORTS = ["minnorm_plan_create", "minnorm_plan_set_params", "minnorm_plan_export_params", "minnorm_sketch", "minnorm_solve", "minnorm_solve_wait", "minnorm_plan_set_wait_limit", "minnorm_trailing_products",
           "minnorm_solve_host", "minnorm_plan_destroy", "minnorm_status_string", "minnorm_get_sketch",
           "minnorm_get_factor", "minnorm_get_preconditioner", "minnorm_cg_products", "minnorm_residual_dd", "minnorm_kernel_stats",
           "minnorm_launch_count", "minnorm_qr_noalloc", "minnorm_solve_many", "minnorm_batch_create",
           "minnorm_batch_solve", "minnorm_batch_destroy", "minnorm_batch_kernel_stats", "minnorm_block_products", "minnorm_plan_tuning"]


class MinnormError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s" % (where, status_string(status)))


class Info(C.Structure):
    _fields_ = [("outer_steps", C.c_int32), ("cg_iters", C.c_int32), ("exact_passes", C.c_int32),
                ("status", C.c_int32), ("err_bound", C.c_double), ("resid_rel", C.c_double),
                ("rdiag_max", C.c_double), ("rdiag_min", C.c_double), ("sigma_min_R", C.c_double),
                ("sigma_max_R", C.c_double), ("cert_delta", C.c_double), ("ms_sketch", C.c_float),
                ("ms_qr", C.c_float), ("ms_solve", C.c_float), ("ms_cg", C.c_float), ("ms_refine", C.c_float),
                ("reserved", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


_lib = None


def lib():
    """Load libminnorm.so (build it first with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libminnorm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        p, i64, u64, u32, i32, d = C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.c_int32, C.c_double
        L.minnorm_plan_create.argtypes = [C.POINTER(p), i64, i64, i64, C.c_int, C.c_int, u64, u32, p]
        L.minnorm_plan_set_params.argtypes = [p] * 9
        L.minnorm_plan_export_params.argtypes = [p] * 9
        L.minnorm_sketch.argtypes = [p, p, i64]
        L.minnorm_solve.argtypes = [p, p, i64, p, d, p, C.POINTER(Info)]
        L.minnorm_solve_wait.argtypes = [p, C.POINTER(Info)]
        L.minnorm_plan_set_wait_limit.argtypes = [p, u64, i32]
        L.minnorm_trailing_products.argtypes = [p, p, i64, p, i64, i64, i64, p, i64, p]
        L.minnorm_solve_host.argtypes = [p, p, i64, p, d, p, C.POINTER(Info)]
        L.minnorm_solve_many.argtypes = [p, p, i64, p, i64, i64, d, p, i64, C.POINTER(Info)]
        L.minnorm_batch_create.argtypes = [C.POINTER(p), i32, C.POINTER(i64), C.POINTER(i64), C.c_int, C.c_int,
                                           u64, u32, p]
        L.minnorm_batch_solve.argtypes = [p, C.POINTER(p), C.POINTER(i64), C.POINTER(p), d, C.POINTER(p),
                                          C.POINTER(Info)]
        L.minnorm_batch_destroy.argtypes = [p]
        L.minnorm_batch_kernel_stats.argtypes = [p, i32, i32, C.POINTER(i32), C.POINTER(d)]
        L.minnorm_plan_destroy.argtypes = [p]
        L.minnorm_status_string.argtypes = [C.c_int]
        L.minnorm_status_string.restype = C.c_char_p
        L.minnorm_get_sketch.argtypes = [p, p]
        L.minnorm_get_factor.argtypes = [p, p, p]
        L.minnorm_get_preconditioner.argtypes = [p, p]
        L.minnorm_cg_products.argtypes = [p, p, i64, p, p, p]
        L.minnorm_block_products.argtypes = [p, p, i64, p, p, p]
        L.minnorm_plan_tuning.argtypes = [p, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.minnorm_residual_dd.argtypes = [p, p, i64, p, p, p, p, p, p]
        L.minnorm_kernel_stats.argtypes = [p, i32, C.POINTER(i32), C.POINTER(d)]
        L.minnorm_qr_noalloc.argtypes = [p, i64, i64, i64, p, p, p]
        L.minnorm_launch_count.argtypes = []
        L.minnorm_launch_count.restype = C.c_int64
        for name in EXPORTS:
            if name not in ("minnorm_status_string", "minnorm_launch_count"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def status_string(status):
    return lib().minnorm_status_string(int(status)).decode()


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError("expected a tensor, an array or an address")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _check(status, where, allow=(OK,)):
    if status not in allow:
        raise MinnormError(status, where)
    return status


def minnorm_plan_create(m, n, l=0, dtype=C128, precision=FP64, seed=1, flags=0, stream=None):
    h = C.c_void_p()
    st = lib().minnorm_plan_create(C.byref(h), int(m), int(n), int(l), int(dtype), int(precision),
                                   int(seed) & 0xFFFFFFFFFFFFFFFF, int(flags), _stream(stream))
    _check(st, "minnorm_plan_create")
    return h


def minnorm_plan_set_params(plan, zeta_t, pi_t, theta_t, zeta, pi, theta, d, s):
    """Host numpy arrays: complex128 phases, int64 permutations/sample, float64 angles."""
    import numpy as np
    arrs = [np.ascontiguousarray(zeta_t, np.complex128), np.ascontiguousarray(pi_t, np.int64),
            np.ascontiguousarray(theta_t, np.float64), np.ascontiguousarray(zeta, np.complex128),
            np.ascontiguousarray(pi, np.int64), np.ascontiguousarray(theta, np.float64),
            np.ascontiguousarray(d, np.complex128), np.ascontiguousarray(s, np.int64)]
    st = lib().minnorm_plan_set_params(plan, *[a.ctypes.data for a in arrs])
    return _check(st, "minnorm_plan_set_params")


def minnorm_plan_export_params(plan, n, l):
    """The plan's SRFT realization as host numpy arrays (zeta_t, pi_t, theta_t, zeta, pi, theta, d, s),
    in the form minnorm_plan_set_params and the oracle's parameter set take."""
    import numpy as np
    arrs = [np.empty(n, np.complex128), np.empty(n, np.int64), np.empty(n - 1, np.float64),
            np.empty(n, np.complex128), np.empty(n, np.int64), np.empty(n - 1, np.float64),
            np.empty(n, np.complex128), np.empty(l, np.int64)]
    _check(lib().minnorm_plan_export_params(plan, *[a.ctypes.data for a in arrs]), "minnorm_plan_export_params")
    return tuple(arrs)


def minnorm_sketch(plan, A, lda=None, allow=(OK,)):
    lda = A.shape[-1] if lda is None else lda
    return _check(lib().minnorm_sketch(plan, _ptr(A), int(lda)), "minnorm_sketch", allow)


def minnorm_solve(plan, A, b, eps, x, lda=None, info=True, allow=(OK,)):
    lda = A.shape[-1] if lda is None else lda
    inf = Info() if info else None
    st = lib().minnorm_solve(plan, _ptr(A), int(lda), _ptr(b), float(eps), _ptr(x),
                             C.byref(inf) if inf is not None else None)
    _check(st, "minnorm_solve", allow)
    return st, (inf.as_dict() if inf is not None else None)


def minnorm_plan_set_wait_limit(plan, limit_ns, withhold=0):
    return _check(lib().minnorm_plan_set_wait_limit(plan, int(limit_ns), int(withhold)),
                  "minnorm_plan_set_wait_limit")


def minnorm_trailing_products(plan, V, C, Z=None, W=None):
    """W = V^H C, then C -= V Z (complex128 column-major device tensors: V rows x 32, C rows x cols,
    Z 32 x cols, W 32 x cols; pass the transposed-contiguous views, e.g. X.T.contiguous().T)."""
    rows, cols = C.shape
    return _check(lib().minnorm_trailing_products(plan, _ptr(V), int(V.stride(1)), _ptr(C), int(C.stride(1)),
                                                  int(rows), int(cols), _ptr(Z),
                                                  int(Z.stride(1)) if Z is not None else 0, _ptr(W)),
                  "minnorm_trailing_products")


def minnorm_solve_wait(plan, info=True, allow=(OK,)):
    """Status (and info) of the plan's last asynchronous minnorm_solve (minnorm_solve(..., info=False))."""
    inf = Info() if info else None
    st = lib().minnorm_solve_wait(plan, C.byref(inf) if inf is not None else None)
    _check(st, "minnorm_solve_wait", allow)
    return st, (inf.as_dict() if inf is not None else None)


def minnorm_solve_many(plan, A, B, eps, X, lda=None, info=True, allow=(OK,)):
    """B: m x nrhs and X: n x nrhs complex128 device tensors, column-major (their .T contiguous),
    i.e. column j at B + j*ldb; ldb/ldx are taken from the tensors' column strides."""
    lda = A.shape[-1] if lda is None else lda
    nrhs = B.shape[1]
    ldb, ldx = B.stride(1), X.stride(1)
    if B.stride(0) != 1 or X.stride(0) != 1 or X.shape[1] != nrhs:
        raise ValueError("B and X must be column-major with matching column counts")
    infos = (Info * nrhs)() if info else None
    st = lib().minnorm_solve_many(plan, _ptr(A), int(lda), _ptr(B), int(ldb), int(nrhs), float(eps), _ptr(X),
                                  int(ldx), infos)
    _check(st, "minnorm_solve_many", allow)
    return st, ([i.as_dict() for i in infos] if infos is not None else None)


def minnorm_batch_create(ms, ns, dtype=C128, precision=FP64, seed=1, flags=0, stream=None):
    """A batch of len(ms) systems, system i of size ms[i] x ns[i] (SRFT seed: seed + i)."""
    count = len(ms)
    if len(ns) != count:
        raise ValueError("ms and ns differ in length")
    am = (C.c_int64 * count)(*[int(v) for v in ms])
    an = (C.c_int64 * count)(*[int(v) for v in ns])
    h = C.c_void_p()
    st = lib().minnorm_batch_create(C.byref(h), count, am, an, int(dtype), int(precision),
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, int(flags), _stream(stream))
    _check(st, "minnorm_batch_create")
    return h


def minnorm_batch_solve(batch, As, bs, eps, xs, ldas=None, info=True, allow=(OK,)):
    """As, bs, xs: sequences of device tensors (system i: m_i x n_i, m_i, n_i)."""
    count = len(As)
    pa = (C.c_void_p * count)(*[_ptr(a) for a in As])
    pb = (C.c_void_p * count)(*[_ptr(v) for v in bs])
    px = (C.c_void_p * count)(*[_ptr(v) for v in xs])
    pl = (C.c_int64 * count)(*[int(v) for v in ldas]) if ldas is not None else None
    infos = (Info * count)() if info else None
    st = lib().minnorm_batch_solve(batch, pa, pl, pb, float(eps), px, infos)
    _check(st, "minnorm_batch_solve", allow)
    return st, ([i.as_dict() for i in infos] if infos is not None else None)


def minnorm_batch_kernel_stats(batch, system, k):
    n = C.c_int32()
    ms = C.c_double()
    _check(lib().minnorm_batch_kernel_stats(batch, int(system), int(k), C.byref(n), C.byref(ms)),
           "minnorm_batch_kernel_stats")
    return n.value, ms.value


def minnorm_batch_destroy(batch):
    return _check(lib().minnorm_batch_destroy(batch), "minnorm_batch_destroy")


def minnorm_solve_host(plan, A, b, eps, x, lda=None, info=True, allow=(OK,)):
    lda = A.shape[-1] if lda is None else lda
    inf = Info() if info else None
    st = lib().minnorm_solve_host(plan, _ptr(A), int(lda), _ptr(b), float(eps), _ptr(x),
                                  C.byref(inf) if inf is not None else None)
    _check(st, "minnorm_solve_host", allow)
    return st, (inf.as_dict() if inf is not None else None)


def minnorm_plan_destroy(plan):
    return _check(lib().minnorm_plan_destroy(plan), "minnorm_plan_destroy")


def minnorm_get_sketch(plan, Y_out):
    return _check(lib().minnorm_get_sketch(plan, _ptr(Y_out)), "minnorm_get_sketch")


def minnorm_get_factor(plan, R_out, piv_out):
    return _check(lib().minnorm_get_factor(plan, _ptr(R_out), _ptr(piv_out)), "minnorm_get_factor")


def minnorm_get_preconditioner(plan, W_out):
    return _check(lib().minnorm_get_preconditioner(plan, _ptr(W_out)), "minnorm_get_preconditioner")


def minnorm_cg_products(plan, A, w, q=None, t=None, lda=None):
    lda = A.shape[-1] if lda is None else lda
    return _check(lib().minnorm_cg_products(plan, _ptr(A), int(lda), _ptr(w), _ptr(q), _ptr(t)),
                  "minnorm_cg_products")


def minnorm_block_products(plan, A, W, Q, T, lda=None):
    lda = A.shape[-1] if lda is None else lda
    return _check(lib().minnorm_block_products(plan, _ptr(A), int(lda), _ptr(W), _ptr(Q), _ptr(T)),
                  "minnorm_block_products")


def minnorm_residual_dd(plan, A, y_hi, y_lo, b, r, x_hi, x_lo, lda=None):
    lda = A.shape[-1] if lda is None else lda
    return _check(lib().minnorm_residual_dd(plan, _ptr(A), int(lda), _ptr(y_hi), _ptr(y_lo), _ptr(b),
                                            _ptr(r), _ptr(x_hi), _ptr(x_lo)), "minnorm_residual_dd")


def minnorm_plan_tuning(plan):
    """(exact-residual column chunks, row splits, fused-CG L2 share in percent, tuned)."""
    c, r, k = C.c_int32(), C.c_int32(), C.c_int32()
    st = lib().minnorm_plan_tuning(plan, C.byref(c), C.byref(r), C.byref(k))
    if st not in (OK, ESTATE):
        raise MinnormError(st, "minnorm_plan_tuning")
    return c.value, r.value, k.value, st == OK


def minnorm_kernel_stats(plan, k):
    n = C.c_int32()
    ms = C.c_double()
    _check(lib().minnorm_kernel_stats(plan, int(k), C.byref(n), C.byref(ms)), "minnorm_kernel_stats")
    return n.value, ms.value


def minnorm_launch_count():
    return int(lib().minnorm_launch_count())


def minnorm_qr_noalloc(Y, l, m, R_out, piv_out, stream=None):
    """Pivoted QR of Y (l x m, column-major, overwritten) with the library's fixed scratch."""
    return _check(lib().minnorm_qr_noalloc(_ptr(Y), int(l), int(l), int(m), _ptr(R_out), _ptr(piv_out),
                                           _stream(stream)), "minnorm_qr_noalloc")
