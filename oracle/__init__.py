"""CPU FP64 oracle for Tygert's randomized minimal-norm solver (arXiv:0905.4745).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg are the only callers. Nothing under paper_0905_4745_gb300/
imports this package, and this package imports nothing from there.

Thin ctypes marshalling over liboracle.so (plain C, see oracle.h); every
function names the passage of the paper it follows. Arrays are numpy
complex128 / int64 / float64; A is row-major m x n, the sketch Y is returned as
an l x m array (column i = T conj(A[i, :])).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


_p = C.c_void_p
_i64 = C.c_int64
_u64 = C.c_uint64
_i32 = C.c_int32
_d = C.c_double


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("rank_ok", C.c_int32),
                ("resid0", C.c_double), ("resid", C.c_double)]


class _Srft(C.Structure):
    _fields_ = [("n", C.c_int64), ("l", C.c_int64),
                ("zeta_t", _p), ("pi_t", _p), ("theta_t", _p),
                ("zeta", _p), ("pi", _p), ("theta", _p),
                ("d", _p), ("s", _p)]


def _declare(L):
    L.orc_mix64.argtypes = [_u64]; L.orc_mix64.restype = _u64
    L.orc_draw.argtypes = [_u64, _u64, _u64]; L.orc_draw.restype = _u64
    L.orc_draw_params.argtypes = [_u64, _i64, _i64] + [_p] * 8
    L.orc_dft.argtypes = [_p, _i64, C.c_int]
    L.orc_dft_brute.argtypes = [_p, _p, _i64, C.c_int]
    L.orc_chain.argtypes = [_p, _i64, _p]
    L.orc_chain_adjoint.argtypes = [_p, _i64, _p]
    L.orc_apply_H.argtypes = [C.POINTER(_Srft), _p, _p]
    L.orc_srft_apply.argtypes = [C.POINTER(_Srft), _p, _p, _p]
    L.orc_srft_adjoint.argtypes = [C.POINTER(_Srft), _p, _p, _p]
    L.orc_sketch.argtypes = [C.POINTER(_Srft), _i64, _p, _i64, _p, _i64]
    L.orc_qrp.argtypes = [_p, _i64, _i64, _i64, _p, _p]
    L.orc_apply_q.argtypes = [_p, _i64, _i64, _i64, _p, _p, C.c_int]
    L.orc_solve_r.argtypes = [_p, _i64, _i64, _p]
    L.orc_solve_rh.argtypes = [_p, _i64, _i64, _p]
    L.orc_adj_matvec_dd.argtypes = [_i64, _i64, _p, _i64, _p, _p, _p, _p]
    L.orc_matvec_dd.argtypes = [_i64, _i64, _p, _i64, _p, _p, _p, _p]
    L.orc_residual_dd.argtypes = [_i64, _i64, _p, _i64, _p, _p, _p, _p, _p, _p]
    L.orc_adj_matvec.argtypes = [_i64, _i64, _p, _i64, _p, _p]
    L.orc_matvec.argtypes = [_i64, _i64, _p, _i64, _p, _p]
    L.orc_minnorm_direct.argtypes = [_i64, _i64, _p, _i64, _p, _i32, _p, _p, _p, C.POINTER(_Info)]
    L.orc_minnorm_direct.restype = C.c_int
    L.orc_minnorm_randomized.argtypes = [C.POINTER(_Srft), _i64, _p, _i64, _p, _d, _i32,
                                         _p, _p, _p, _p, _p, C.POINTER(_Info)]
    L.orc_minnorm_randomized.restype = C.c_int
    L.orc_pcg_normal.argtypes = [_i64, _i64, _p, _i64, _p, _p, _i64, _p, _p, _i32, _p, _p]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _z(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _info_dict(info):
    return {"iters": info.iters, "rank_ok": bool(info.rank_ok),
            "resid0": info.resid0, "resid": info.resid}


# ------------------------------------------------------------------ rng ----
def mix64(z: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014)."""
    return lib().orc_mix64(z & 0xFFFFFFFFFFFFFFFF)


def draw(seed: int, kind: int, j: int) -> int:
    """j-th draw of parameter stream `kind` (kind 0 = the published SplitMix64 stream)."""
    return lib().orc_draw(seed & 0xFFFFFFFFFFFFFFFF, kind, j)


class Params:
    """One SRFT realization (Section 3): phases zeta~, zeta, d; permutations
    pi~, pi; angles theta~, theta; sorted sample s (l distinct rows of F)."""

    def __init__(self, n, l, zeta_t, pi_t, theta_t, zeta, pi, theta, d, s):
        self.n, self.l = int(n), int(l)
        self.zeta_t = _z(zeta_t); self.zeta = _z(zeta); self.d = _z(d)
        self.pi_t = np.ascontiguousarray(pi_t, dtype=np.int64)
        self.pi = np.ascontiguousarray(pi, dtype=np.int64)
        self.theta_t = np.ascontiguousarray(theta_t, dtype=np.float64)
        self.theta = np.ascontiguousarray(theta, dtype=np.float64)
        self.s = np.ascontiguousarray(s, dtype=np.int64)

    def _struct(self):
        return _Srft(self.n, self.l, _ptr(self.zeta_t), _ptr(self.pi_t), _ptr(self.theta_t),
                     _ptr(self.zeta), _ptr(self.pi), _ptr(self.theta), _ptr(self.d), _ptr(self.s))


def draw_params(n: int, l: int, seed: int) -> Params:
    """Parameters drawn from SplitMix64 streams 0..7 (zeta~, pi~, theta~, zeta, pi, theta, d, s)."""
    zt = np.empty(n, np.complex128); z = np.empty(n, np.complex128); d = np.empty(n, np.complex128)
    pt = np.empty(n, np.int64); p = np.empty(n, np.int64)
    tt = np.empty(max(n - 1, 1), np.float64); t = np.empty(max(n - 1, 1), np.float64)
    s = np.empty(l, np.int64)
    lib().orc_draw_params(seed & 0xFFFFFFFFFFFFFFFF, n, l, _ptr(zt), _ptr(pt), _ptr(tt),
                          _ptr(z), _ptr(p), _ptr(t), _ptr(d), _ptr(s))
    return Params(n, l, zt, pt, tt[: n - 1], z, p, t[: n - 1], d, s)


# ------------------------------------------------------------------ fft ----
def dft(x, sign=-1):
    """Unitary DFT of Eq. (DFT) (sign -1: F; +1: F^*)."""
    y = _z(x).copy()
    lib().orc_dft(_ptr(y), y.size, sign)
    return y


def dft_brute(x, sign=-1):
    x = _z(x)
    out = np.empty_like(x)
    lib().orc_dft_brute(_ptr(x), _ptr(out), x.size, sign)
    return out


# ----------------------------------------------------------------- srft ----
def chain(v, theta):
    """Theta v for the Givens chain of Eq. big_def."""
    v = _z(v).copy()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lib().orc_chain(_ptr(v), v.size, _ptr(th))
    return v


def chain_adjoint(v, theta):
    v = _z(v).copy()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lib().orc_chain_adjoint(_ptr(v), v.size, _ptr(th))
    return v


def apply_H(P: Params, v):
    """H v, Eq. Rokhlin_trans."""
    v = _z(v).copy()
    w = np.empty_like(v)
    S = P._struct()
    lib().orc_apply_H(C.byref(S), _ptr(v), _ptr(w))
    return v


def srft_apply(P: Params, v):
    """T v, Eqs. SRFT and SRFT2."""
    v = _z(v)
    y = np.empty(P.l, np.complex128)
    work = np.empty(2 * P.n, np.complex128)
    S = P._struct()
    lib().orc_srft_apply(C.byref(S), _ptr(v), _ptr(y), _ptr(work))
    return y


def srft_adjoint(P: Params, y):
    """T^* y."""
    y = _z(y)
    v = np.empty(P.n, np.complex128)
    work = np.empty(P.n, np.complex128)
    S = P._struct()
    lib().orc_srft_adjoint(C.byref(S), _ptr(y), _ptr(v), _ptr(work))
    return v


def srft_dense(P: Params):
    """T as a dense l x n matrix (columns T e_k); tiny n only."""
    T = np.empty((P.l, P.n), np.complex128)
    e = np.zeros(P.n, np.complex128)
    for k in range(P.n):
        e[:] = 0
        e[k] = 1
        T[:, k] = srft_apply(P, e)
    return T


def sketch(P: Params, A):
    """Step 1, Eq. randmat: Y = T A^*; returns Y as an l x m array."""
    A = _z(A)
    m = A.shape[0]
    Yt = np.empty((m, P.l), np.complex128)          # row i = column i of Y
    S = P._struct()
    lib().orc_sketch(C.byref(S), m, _ptr(A), A.shape[1], _ptr(Yt), P.l)
    return Yt.T


# ------------------------------------------------------------------- qr ----
class QR:
    """Result of orc_qrp: Y[:, piv] = Q R."""

    def __init__(self, F, piv, tau):
        self.F, self.piv, self.tau = F, piv, tau     # F: column-major factors (Fortran order)

    @property
    def R(self):
        k = self.tau.size
        return np.triu(self.F[:k, :k])

    def apply_q(self, x, conj=False):
        x = _z(x).copy()
        rows = self.F.shape[0]
        Ft = np.asfortranarray(self.F)
        lib().orc_apply_q(Ft.ctypes.data_as(C.c_void_p), rows, rows, self.tau.size,
                          _ptr(self.tau), _ptr(x), 1 if conj else 0)
        return x

    def Q(self):
        rows, k = self.F.shape[0], self.tau.size
        return np.stack([self.apply_q(np.eye(rows, 1, -j)[:, 0]) for j in range(k)], axis=1)


def qrp(Y) -> QR:
    """Pivoted Householder QR (Section 7; GVL ch. 5; LAPACK zgeqp3 conventions)."""
    F = np.array(Y, dtype=np.complex128, order="F", copy=True)
    rows, cols = F.shape
    k = min(rows, cols)
    piv = np.empty(cols, np.int64)
    tau = np.empty(k, np.complex128)
    lib().orc_qrp(F.ctypes.data_as(C.c_void_p), rows, rows, cols, _ptr(piv), _ptr(tau))
    return QR(F, piv, tau)


def solve_r(R, x):
    Rf = np.asfortranarray(R, dtype=np.complex128)
    x = _z(x).copy()
    lib().orc_solve_r(Rf.ctypes.data_as(C.c_void_p), Rf.shape[0], Rf.shape[0], _ptr(x))
    return x


def solve_rh(R, x):
    Rf = np.asfortranarray(R, dtype=np.complex128)
    x = _z(x).copy()
    lib().orc_solve_rh(Rf.ctypes.data_as(C.c_void_p), Rf.shape[0], Rf.shape[0], _ptr(x))
    return x


# ------------------------------------------------------------- products ----
def adj_matvec(A, y):
    A = _z(A); y = _z(y)
    x = np.empty(A.shape[1], np.complex128)
    lib().orc_adj_matvec(A.shape[0], A.shape[1], _ptr(A), A.shape[1], _ptr(y), _ptr(x))
    return x


def matvec(A, x):
    A = _z(A); x = _z(x)
    v = np.empty(A.shape[0], np.complex128)
    lib().orc_matvec(A.shape[0], A.shape[1], _ptr(A), A.shape[1], _ptr(x), _ptr(v))
    return v


def adj_matvec_dd(A, y_hi, y_lo=None):
    """x = A^* (y_hi + y_lo) with double-double sums; returns (x_hi, x_lo)."""
    A = _z(A); yh = _z(y_hi); yl = None if y_lo is None else _z(y_lo)
    xh = np.empty(A.shape[1], np.complex128); xl = np.empty_like(xh)
    lib().orc_adj_matvec_dd(A.shape[0], A.shape[1], _ptr(A), A.shape[1], _ptr(yh), _ptr(yl),
                            _ptr(xh), _ptr(xl))
    return xh, xl


def matvec_dd(A, x_hi, x_lo=None):
    A = _z(A); xh = _z(x_hi); xl = None if x_lo is None else _z(x_lo)
    vh = np.empty(A.shape[0], np.complex128); vl = np.empty_like(vh)
    lib().orc_matvec_dd(A.shape[0], A.shape[1], _ptr(A), A.shape[1], _ptr(xh), _ptr(xl),
                        _ptr(vh), _ptr(vl))
    return vh, vl


def residual_dd(A, y_hi, y_lo, b):
    """r = b - A A^* y with double-double sums; returns (r, x_hi, x_lo)."""
    A = _z(A); yh = _z(y_hi); yl = None if y_lo is None else _z(y_lo); b = _z(b)
    m, n = A.shape
    r = np.empty(m, np.complex128); xh = np.empty(n, np.complex128); xl = np.empty_like(xh)
    lib().orc_residual_dd(m, n, _ptr(A), n, _ptr(yh), _ptr(yl), _ptr(b), _ptr(r), _ptr(xh), _ptr(xl))
    return r, xh, xl


# -------------------------------------------------------------- solvers ----
def minnorm_direct(A, b, steps=6):
    """O1: direct pivoted-QR minimal-norm solve (Section 7) + double-double refinement.
    Returns dict(p, y, x0, info)."""
    A = _z(A); b = _z(b)
    m, n = A.shape
    p = np.empty(n, np.complex128); y = np.empty(m, np.complex128); x0 = np.empty(n, np.complex128)
    info = _Info()
    rc = lib().orc_minnorm_direct(m, n, _ptr(A), n, _ptr(b), steps, _ptr(p), _ptr(y), _ptr(x0),
                                  C.byref(info))
    return {"rc": rc, "p": p, "y": y, "x0": x0, "info": _info_dict(info)}


def minnorm_randomized(P: Params, A, b, delta, maxit=1000):
    """O2: Section 4, Steps 1-5, literally (FP64). Returns dict(x, y, z, c, u0, info)."""
    A = _z(A); b = _z(b)
    m, n = A.shape
    x = np.empty(n, np.complex128); y = np.empty(m, np.complex128)
    z = np.empty(P.l, np.complex128); c = np.empty(n, np.complex128); u0 = np.empty(m, np.complex128)
    info = _Info()
    S = P._struct()
    rc = lib().orc_minnorm_randomized(C.byref(S), m, _ptr(A), n, _ptr(b), float(delta), int(maxit),
                                      _ptr(x), _ptr(y), _ptr(z), _ptr(c), _ptr(u0), C.byref(info))
    return {"rc": rc, "x": x, "y": y, "z": z, "c": c, "u0": u0, "info": _info_dict(info)}


def pcg_normal(A, b, R, piv, iters, u_start=None):
    """CG on R^{-*} P^T A A^* P R^{-1} u = R^{-*} P^T b (the GPU path's form of Step 4).
    Returns (u_hist (iters x m), y)."""
    A = _z(A); b = _z(b)
    m, n = A.shape
    Rf = np.asfortranarray(R, dtype=np.complex128)
    piv = np.ascontiguousarray(piv, dtype=np.int64)
    us = None if u_start is None else _z(u_start)
    hist = np.empty((max(iters, 1), m), np.complex128)
    y = np.empty(m, np.complex128)
    lib().orc_pcg_normal(m, n, _ptr(A), n, _ptr(b), Rf.ctypes.data_as(C.c_void_p), m, _ptr(piv),
                         _ptr(us), int(iters), _ptr(hist), _ptr(y))
    return hist[:iters], y


# ----------------------------------------------------------- certificate ----
def error_certificate(A, b, X, seed=1, l=None):
    """A posteriori bound on ||x - p|| / ||x|| for each column x of X, computed on the host
    from the oracle's own FP64 sketch (Section 5's argument, applied after the fact).

    Y = T A^* is the oracle's sketch (Step 1, Eq. randmat) for the SRFT drawn from `seed`, and
    Y = Q R any QR of it (LAPACK's unpivoted one: Steps 2-4 need only some R with Y R^{-1}
    orthonormal). Then T A^* R^{-1} = Q, and since T has orthonormal rows (Section 3),
    sigma_min(A^* R^{-1}) >= 1 - delta, delta covering the FP64 rounding of the sketch and the
    QR (a priori: 8 (n + log2 n + 2 m) 2^-53 ||A||_F ||R^{-1}||_F). For x = A^* y (the form of
    Step 5, Eq. output) and p = A^* y*, x - p = A^* (y - y*) and R^{-*} A (x - p) =
    (A^* R^{-1})^* (x - p), so ||x - p|| <= ||R^{-*} (b - A x)|| / (1 - delta); the residual
    b - A x is formed with double-double sums (Dot2). A column rounded to complex128 after
    x = A^* y adds at most 2^-53 ||x||, included. Returns (bounds, delta); a bound is +inf when
    delta >= 1/2 (no certificate)."""
    A = _z(A)
    X = np.asarray(X, dtype=np.complex128)
    cols = X[:, None] if X.ndim == 1 else X
    B = np.asarray(b, dtype=np.complex128)
    B = B[:, None] if B.ndim == 1 else B
    m, n = A.shape
    l = min(4 * m, n) if l is None else l
    P = draw_params(n, l, seed)
    Y = np.ascontiguousarray(sketch(P, A))
    R = np.linalg.qr(Y, mode="r")
    Rinv_f = np.linalg.norm(np.linalg.solve(R, np.eye(m)))          # ||R^{-1}||_F
    u = 2.0 ** -53
    delta = 8.0 * (n + np.log2(n) + 2 * m) * u * np.linalg.norm(A) * Rinv_f
    bounds = []
    for j in range(cols.shape[1]):
        x = np.ascontiguousarray(cols[:, j])
        vh, vl = matvec_dd(A, x)
        r = (B[:, j] - vh) - vl
        g = np.linalg.solve(R.conj().T, r)                            # R^{-*} r
        xn = np.linalg.norm(x)
        if delta >= 0.5 or xn == 0.0:
            bounds.append(np.inf)
        else:
            bounds.append(np.linalg.norm(g) / (1.0 - delta) / xn + u)
    return np.array(bounds), float(delta)
