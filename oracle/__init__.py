"""Oracle: plain sequential FP64 CPU reference for the Kalman filter, the
RTS smoother, the two-filter smoother and the parallel-form elements and
operators of arXiv 2511.10363 (Sec. III, Sec. IV-C/IV-D, Lemmas 1 and 2).

TEST INFRASTRUCTURE ONLY.  The arithmetic lives in ``kf_oracle.c`` (built
with gcc into ``oracle/_build/liborc.so``); this module only marshals numpy
arrays.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import it.  It shares no code with the CUDA library and never
imports it.

Every function is pinned by ``tests/test_oracle_pins.py`` (closed forms, a
dense joint-Gaussian brute force, special cases, algebraic identities); no
function is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile kf_oracle.c with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.POINTER(ctypes.c_double)
        i, l = ctypes.c_int, ctypes.c_long
        lib.orc_kf.argtypes = [i, i, D, D, D, D, D, D, l, D, D, D, D, D, D]
        lib.orc_rts.argtypes = [i, D, D, l, D, D, D, D]
        lib.orc_tf.argtypes = [i, i, D, D, D, D, l, D, D, D, D, D, D, D]
        lib.orc_filter_element.argtypes = [i, i, D, D, D, D, D, D, l, D, D]
        lib.orc_filter_combine.argtypes = [i, D, D, D]
        lib.orc_rts_element.argtypes = [i, D, D, i, D, D, D]
        lib.orc_rts_combine.argtypes = [i, D, D, D]
        lib.orc_rts_combine.restype = None
        lib.orc_tv_kf.argtypes = [i, i, D, D, D, D, D, D, D, D, l, D, D, D, D]
        lib.orc_tv_rts.argtypes = [i, D, D, D, l, D, D, D, D]
        lib.orc_tv_tf.argtypes = [i, i, D, D, D, D, D, D, l, D, D, D, D, D, D, D]
        lib.orc_tv_filter_element.argtypes = [i, i, D, D, D, D, D, D, D, D, i, D, D]
        lib.orc_tv_rts_element.argtypes = [i, D, D, D, i, D, D, D]
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _model(model):
    F, Q, H, R = (_c(model[k]) for k in ("F", "Q", "H", "R"))
    m0, P0 = _c(model["m0"]), _c(model["P0"])
    return F, Q, H, R, m0, P0


def kf(model, y, want_pred=False):
    """Sequential Kalman filter (Sec. III-A).  Returns (m [T,n], P [T,n,n],
    loglik) and, with want_pred, also the predicted (m, P)."""
    F, Q, H, R, m0, P0 = _model(model)
    y = _c(y)
    T, ny = y.shape
    nx = F.shape[0]
    m = np.empty((T, nx))
    P = np.empty((T, nx, nx))
    mp = np.empty((T, nx)) if want_pred else None
    Pp = np.empty((T, nx, nx)) if want_pred else None
    ll = np.zeros(1)
    rc = _load().orc_kf(nx, ny, _p(F), _p(Q), _p(H), _p(R), _p(m0), _p(P0), T, _p(y), _p(m), _p(P),
                        _p(mp), _p(Pp), _p(ll))
    if rc:
        raise ArithmeticError("oracle KF: innovation covariance not positive definite")
    if want_pred:
        return m, P, float(ll[0]), mp, Pp
    return m, P, float(ll[0])


def rts(model, mf, Pf):
    """Sequential RTS smoother (Sec. III-B) from filtering results."""
    F, Q = _c(model["F"]), _c(model["Q"])
    mf, Pf = _c(mf), _c(Pf)
    T, nx = mf.shape
    ms = np.empty_like(mf)
    Ps = np.empty_like(Pf)
    if _load().orc_rts(nx, _p(F), _p(Q), T, _p(mf), _p(Pf), _p(ms), _p(Ps)):
        raise ArithmeticError("oracle RTS: singular predicted covariance")
    return ms, Ps


def tf(model, y, mf, Pf, want_info=False):
    """Sequential two-filter smoother (Sec. III-B): backward information
    filter plus the merge of Eqs. mean/cov_tf_combination."""
    F, Q, H, R, _, _ = _model(model)
    y, mf, Pf = _c(y), _c(mf), _c(Pf)
    T, ny = y.shape
    nx = F.shape[0]
    ms = np.empty_like(mf)
    Ps = np.empty_like(Pf)
    eta = np.empty((T, nx)) if want_info else None
    J = np.empty((T, nx, nx)) if want_info else None
    if _load().orc_tf(nx, ny, _p(F), _p(Q), _p(H), _p(R), T, _p(y), _p(mf), _p(Pf), _p(ms), _p(Ps),
                      _p(eta), _p(J)):
        raise ArithmeticError("oracle TF: singular system")
    if want_info:
        return ms, Ps, eta, J
    return ms, Ps


def smooth(model, y, kind="rts"):
    """Filter then smooth: returns (ms, Ps, mf, Pf, loglik)."""
    mf, Pf, ll = kf(model, y)
    if kind == "rts":
        ms, Ps = rts(model, mf, Pf)
    elif kind == "tf":
        ms, Ps = tf(model, y, mf, Pf)
    else:
        raise ValueError(kind)
    return ms, Ps, mf, Pf, ll


# ---- parallel-form elements and operators (Sec. IV-C/D) -------------------

class FilterElem:
    """(A, b, C, eta, J) of Sec. IV-C held as numpy arrays."""

    def __init__(self, A, b, C, eta, J):
        self.A, self.b, self.C, self.eta, self.J = A, b, C, eta, J

    @staticmethod
    def identity(n):
        """(I, 0, 0, 0, 0): the neutral element of Lemma 1."""
        z = np.zeros((n, n))
        return FilterElem(np.eye(n), np.zeros(n), z.copy(), np.zeros(n), z.copy())

    @staticmethod
    def zero(n):
        """(0, 0, 0, 0, 0), printed as the terminal element of Alg. ptf."""
        z = np.zeros((n, n))
        return FilterElem(z.copy(), np.zeros(n), z.copy(), np.zeros(n), z.copy())

    def flat(self):
        return np.concatenate([self.A.ravel(), self.b, self.C.ravel(), self.eta, self.J.ravel()])

    @staticmethod
    def unflat(v, n):
        v = np.asarray(v, dtype=np.float64)
        o = [0, n * n, n * n + n, 2 * n * n + n, 2 * n * n + 2 * n, 3 * n * n + 2 * n]
        return FilterElem(v[o[0]:o[1]].reshape(n, n).copy(), v[o[1]:o[2]].copy(),
                          v[o[2]:o[3]].reshape(n, n).copy(), v[o[3]:o[4]].copy(),
                          v[o[4]:o[5]].reshape(n, n).copy())


class RtsElem:
    """(E, g, L) of Sec. IV-D."""

    def __init__(self, E, g, L):
        self.E, self.g, self.L = E, g, L

    @staticmethod
    def identity(n):
        return RtsElem(np.eye(n), np.zeros(n), np.zeros((n, n)))

    def flat(self):
        return np.concatenate([self.E.ravel(), self.g, self.L.ravel()])

    @staticmethod
    def unflat(v, n):
        v = np.asarray(v, dtype=np.float64)
        return RtsElem(v[:n * n].reshape(n, n).copy(), v[n * n:n * n + n].copy(),
                       v[n * n + n:].reshape(n, n).copy())


def filter_element(model, k, yk):
    """Element a_k (k 1-based) of Eqs. pkf_init1/2/3."""
    F, Q, H, R, m0, P0 = _model(model)
    nx, ny = F.shape[0], H.shape[0]
    out = np.empty(3 * nx * nx + 2 * nx)
    if _load().orc_filter_element(nx, ny, _p(F), _p(Q), _p(H), _p(R), _p(m0), _p(P0), int(k), _p(_c(yk)), _p(out)):
        raise ArithmeticError("oracle element: S not positive definite")
    return FilterElem.unflat(out, nx)


def filter_combine(ei: FilterElem, ej: FilterElem) -> FilterElem:
    """Lemma 1."""
    n = ei.A.shape[0]
    a, b = _c(ei.flat()), _c(ej.flat())
    out = np.empty_like(a)
    if _load().orc_filter_combine(n, _p(a), _p(b), _p(out)):
        raise ArithmeticError("oracle Lemma 1: singular I + C_i J_j")
    return FilterElem.unflat(out, n)


def rts_element(model, last, xk, Pk):
    """Element of Eqs. prts_init1 (last=False) / prts_init2 (last=True)."""
    F, Q = _c(model["F"]), _c(model["Q"])
    n = F.shape[0]
    out = np.empty(2 * n * n + n)
    if _load().orc_rts_element(n, _p(F), _p(Q), int(bool(last)), _p(_c(xk)), _p(_c(Pk)), _p(out)):
        raise ArithmeticError("oracle RTS element: singular predicted covariance")
    return RtsElem.unflat(out, n)


def rts_combine(ei: RtsElem, ej: RtsElem) -> RtsElem:
    """Lemma 2."""
    n = ei.E.shape[0]
    a, b = _c(ei.flat()), _c(ej.flat())
    out = np.empty_like(a)
    _load().orc_rts_combine(n, _p(a), _p(b), _p(out))
    return RtsElem.unflat(out, n)


# ---- time-varying model (Sec. III-A with per-step F, Q, u, H, R, d) -------
#
# A time-varying model is a dict of per-step arrays: record t = 0 .. T-1
# belongs to time k = t + 1 and holds F[t] = F_{k-1}, Q[t] = Q_{k-1},
# u[t] = u_{k-1} (or u = None), H[t] = H_k, R[t] = R_k, d[t] = d_k (or
# d = None); m0, P0 are the prior xbar_{0|0}, P_{0|0}.

def _tv(model):
    F, Q, H, R = (_c(model[k]) for k in ("F", "Q", "H", "R"))
    u = None if model.get("u") is None else _c(model["u"])
    d = None if model.get("d") is None else _c(model["d"])
    return F, Q, u, H, R, d, _c(model["m0"]), _c(model["P0"])


def tv_kf(model, y):
    """Sequential Kalman filter for a time-varying model: (m, P, loglik)."""
    F, Q, u, H, R, d, m0, P0 = _tv(model)
    y = _c(y)
    T, ny = y.shape
    nx = F.shape[1]
    m = np.empty((T, nx))
    P = np.empty((T, nx, nx))
    ll = np.zeros(1)
    if _load().orc_tv_kf(nx, ny, _p(F), _p(Q), _p(u), _p(H), _p(R), _p(d), _p(m0), _p(P0), T, _p(y), _p(m),
                         _p(P), _p(ll)):
        raise ArithmeticError("oracle TV KF: innovation covariance not positive definite")
    return m, P, float(ll[0])


def tv_rts(model, mf, Pf):
    """Sequential RTS smoother for a time-varying model."""
    F, Q, u, _, _, _, _, _ = _tv(model)
    mf, Pf = _c(mf), _c(Pf)
    T, nx = mf.shape
    ms = np.empty_like(mf)
    Ps = np.empty_like(Pf)
    if _load().orc_tv_rts(nx, _p(F), _p(Q), _p(u), T, _p(mf), _p(Pf), _p(ms), _p(Ps)):
        raise ArithmeticError("oracle TV RTS: singular predicted covariance")
    return ms, Ps


def tv_tf(model, y, mf, Pf, want_info=False):
    """Sequential two-filter smoother for a time-varying model."""
    F, Q, u, H, R, d, _, _ = _tv(model)
    y, mf, Pf = _c(y), _c(mf), _c(Pf)
    T, ny = y.shape
    nx = F.shape[1]
    ms = np.empty_like(mf)
    Ps = np.empty_like(Pf)
    eta = np.empty((T, nx)) if want_info else None
    J = np.empty((T, nx, nx)) if want_info else None
    if _load().orc_tv_tf(nx, ny, _p(F), _p(Q), _p(u), _p(H), _p(R), _p(d), T, _p(y), _p(mf), _p(Pf), _p(ms),
                         _p(Ps), _p(eta), _p(J)):
        raise ArithmeticError("oracle TV TF: singular system")
    if want_info:
        return ms, Ps, eta, J
    return ms, Ps


def tv_smooth(model, y, kind="rts"):
    """Filter then smooth a time-varying model: (ms, Ps, mf, Pf, loglik)."""
    mf, Pf, ll = tv_kf(model, y)
    if kind == "rts":
        ms, Ps = tv_rts(model, mf, Pf)
    elif kind == "tf":
        ms, Ps = tv_tf(model, y, mf, Pf)
    else:
        raise ValueError(kind)
    return ms, Ps, mf, Pf, ll


def tv_filter_element(model, k, yk):
    """Element a_k (k 1-based) of Eqs. pkf_init1/2/3 with the step's
    F_{k-1}, Q_{k-1}, u_{k-1}, H_k, R_k, d_k."""
    F, Q, u, H, R, d, m0, P0 = _tv(model)
    t = int(k) - 1
    nx, ny = F.shape[1], H.shape[1]
    out = np.empty(3 * nx * nx + 2 * nx)
    ut = None if u is None else _c(u[t])
    dt = None if d is None else _c(d[t])
    if _load().orc_tv_filter_element(nx, ny, _p(_c(F[t])), _p(_c(Q[t])), _p(ut), _p(_c(H[t])), _p(_c(R[t])),
                                     _p(dt), _p(m0), _p(P0), int(k == 1), _p(_c(yk)), _p(out)):
        raise ArithmeticError("oracle TV element: S not positive definite")
    return FilterElem.unflat(out, nx)


def tv_rts_element(model, k, T, xk, Pk):
    """Element of Eqs. prts_init1 (k < T, with F_k, Q_k, u_k) / prts_init2 (k = T)."""
    F, Q, u, _, _, _, _, _ = _tv(model)
    n = F.shape[1]
    out = np.empty(2 * n * n + n)
    last = int(k == T)
    t = min(int(k), F.shape[0] - 1)          # record k holds F_k, Q_k, u_k (unused at k = T)
    ut = None if u is None else _c(u[t])
    if _load().orc_tv_rts_element(n, _p(_c(F[t])), _p(_c(Q[t])), _p(ut), last, _p(_c(xk)), _p(_c(Pk)), _p(out)):
        raise ArithmeticError("oracle TV RTS element: singular predicted covariance")
    return RtsElem.unflat(out, n)
