"""FP64 CPU oracle for the Fast Coherent Point Drift EM loop (arXiv 2006.06281).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The CUDA
library never imports, links or runs anything here, and nothing here imports
the CUDA package.

The arithmetic lives in ``cpd_oracle.c`` (plain double loops, compiled with
gcc, no fast-math, no FMA contraction).  This module adds:
  * the eigendecomposition of the Gram matrix (Eq. 16) by LAPACK
    (``numpy.linalg.eigh``), sorted descending, eigenvalues clamped at 0 and
    truncated to the top K for the low-rank variant (Eq. 19);
  * numpy-array marshalling for the C functions.

Parity: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, invariants, textbook solves and symmetries.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpd_oracle.c")
_LIB = os.path.join(_HERE, "libcpd_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ENUMERIC = 5


def build(force: bool = False) -> str:
    """Compile cpd_oracle.c into oracle/libcpd_oracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-std=c11", "-D_DEFAULT_SOURCE", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # FCPD_ORACLE_LIB lets the mutation test load a deliberately broken
            # copy of this oracle; normal runs build and load cpd_oracle.c.
            path = os.environ.get("FCPD_ORACLE_LIB") or build()
            lib = C.CDLL(path)
            d, i64, i32, vp = C.c_double, C.c_int64, C.c_int32, C.c_void_p
            lib.fcpd_oracle_gram.argtypes = [vp, i64, i32, d, vp]
            lib.fcpd_oracle_gram.restype = None
            lib.fcpd_oracle_sigma2_init.argtypes = [vp, i64, vp, i64, i32]
            lib.fcpd_oracle_sigma2_init.restype = d
            lib.fcpd_oracle_outlier_c.argtypes = [d, d, i64, i64, i32]
            lib.fcpd_oracle_outlier_c.restype = d
            lib.fcpd_oracle_estep.argtypes = [vp, i64, vp, i64, i32, d, d, vp, vp, vp, vp, vp, vp]
            lib.fcpd_oracle_estep.restype = C.c_int
            lib.fcpd_oracle_mstep.argtypes = [vp, vp, i64, i64, vp, vp, i32, d, d, vp, vp, vp]
            lib.fcpd_oracle_mstep.restype = None
            lib.fcpd_oracle_sigma2.argtypes = [vp, vp, vp, vp, i64, i32]
            lib.fcpd_oracle_sigma2.restype = d
            lib.fcpd_oracle_register.argtypes = [vp, i64, vp, i64, i32, vp, vp, i64, d, d, d, i32,
                                                 vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.fcpd_oracle_register.restype = C.c_int
            lib.fcpd_oracle_rmse.argtypes = [vp, vp, i64, i32]
            lib.fcpd_oracle_rmse.restype = d
            _lib = lib
    return _lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def gram(X: np.ndarray, beta: float) -> np.ndarray:
    """Eq. 11: the M x M Gaussian Gram matrix of the model points."""
    X = _c(X)
    M, D = X.shape
    Phi = np.empty((M, M))
    _load().fcpd_oracle_gram(_p(X), M, D, float(beta), _p(Phi))
    return Phi


_eig_cache: dict = {}


def eig(X: np.ndarray, beta: float, K: int = 0):
    """Eq. 16 / Eq. 19: eigenpairs of the Gram matrix of X, descending.

    Returns (U, lam): U is M x K (columns = eigenvectors), lam the K largest
    eigenvalues clamped at 0 (the Gram matrix is positive semidefinite; LAPACK
    returns tiny negative values at rounding level).  K = 0 or K >= M keeps
    the full basis.  Results are memoised per (X, beta)."""
    X = _c(X)
    M = X.shape[0]
    key = (hashlib.sha1(X.tobytes()).hexdigest(), float(beta))
    if key not in _eig_cache:
        w, V = np.linalg.eigh(gram(X, beta))
        order = np.argsort(-w, kind="stable")
        _eig_cache.clear()
        _eig_cache[key] = (np.ascontiguousarray(V[:, order]), np.maximum(w[order], 0.0))
    U, lam = _eig_cache[key]
    if K and K < M:
        return np.ascontiguousarray(U[:, :K]), lam[:K].copy()
    return U, lam


def eig_top(X: np.ndarray, beta: float, K: int):
    """Eq. 19: the K largest eigenpairs of the Gram matrix of X by the
    Lanczos method (``scipy.sparse.linalg.eigsh``, a library primitive), for
    model sets too large for the dense eigensolver on the host.  Same
    conventions as eig(): descending, clamped at 0."""
    import scipy.sparse.linalg as sla
    w, V = sla.eigsh(gram(X, beta), k=int(K), which="LA")
    order = np.argsort(-w, kind="stable")
    return np.ascontiguousarray(V[:, order]), np.maximum(w[order], 0.0)


def sigma2_init(X: np.ndarray, Y: np.ndarray) -> float:
    """sigma2_0 = sum_mn |y_n - x_m|^2 / (D M N)  (the paper is silent; reading)."""
    X, Y = _c(X), _c(Y)
    return _load().fcpd_oracle_sigma2_init(_p(X), X.shape[0], _p(Y), Y.shape[0], X.shape[1])


def outlier_c(sigma2: float, w: float, M: int, N: int, D: int) -> float:
    """The constant c of Eq. 4."""
    return _load().fcpd_oracle_outlier_c(float(sigma2), float(w), int(M), int(N), int(D))


def estep(T: np.ndarray, Y: np.ndarray, sigma2: float, w: float) -> dict:
    """Eq. 4 + Eq. 5.  Returns den, P1, PY, S, Ytil, loglik, status."""
    T, Y = _c(T), _c(Y)
    M, D = T.shape
    N = Y.shape[0]
    out = dict(den=np.empty(N), P1=np.empty(M), PY=np.empty((M, D)), S=np.empty(M),
               Ytil=np.empty((M, D)))
    ll = C.c_double(0.0)
    st = _load().fcpd_oracle_estep(_p(T), M, _p(Y), N, D, float(sigma2), float(w),
                                   _p(out["den"]), _p(out["P1"]), _p(out["PY"]), _p(out["S"]),
                                   _p(out["Ytil"]), C.byref(ll))
    out["loglik"] = ll.value
    out["status"] = st
    return out


def mstep(U: np.ndarray, lam: np.ndarray, X: np.ndarray, Ytil: np.ndarray,
          lam_reg: float, sigma2: float):
    """Eq. 17 (K = M) / Eq. 20 (K < M).  Returns (T, W, A) with A = U^T (Ytil - X)."""
    U, lam, X, Ytil = _c(U), _c(lam), _c(X), _c(Ytil)
    M, D = X.shape
    K = U.shape[1]
    T, W, A = np.empty((M, D)), np.empty((M, D)), np.empty((K, D))
    _load().fcpd_oracle_mstep(_p(U), _p(lam), M, K, _p(X), _p(Ytil), D, float(lam_reg),
                              float(sigma2), _p(T), _p(W), _p(A))
    return T, W, A


def sigma2_update(S, P1, Ytil, T) -> float:
    """Eq. 18 over the row-normalised posterior, with the new T."""
    S, P1, Ytil, T = _c(S), _c(P1), _c(Ytil), _c(T)
    M, D = T.shape
    return _load().fcpd_oracle_sigma2(_p(S), _p(P1), _p(Ytil), _p(T), M, D)


def rmse(T, Yhat) -> float:
    """Eq. 22."""
    T, Yhat = _c(T), _c(Yhat)
    return _load().fcpd_oracle_rmse(_p(T), _p(Yhat), T.shape[0], T.shape[1])


def register(X, Y, w: float, beta: float, lam_reg: float, n_iter: int, K: int = 0,
             sigma2_0: float | None = None, eigpairs=None) -> dict:
    """The whole loop: setup (Gram matrix, eigendecomposition, sigma2_0), then
    n_iter EM iterations.  Returns T, W, sigma2, iters, status, and the
    per-iteration sigma2 / log-likelihood histories."""
    X, Y = _c(X), _c(Y)
    M, D = X.shape
    N = Y.shape[0]
    U, lam = eigpairs if eigpairs is not None else eig(X, beta, K)
    U, lam = _c(U), _c(lam)
    Kk = U.shape[1]
    s0 = sigma2_init(X, Y) if sigma2_0 is None or sigma2_0 <= 0 else float(sigma2_0)
    T = X.copy()
    W = np.zeros((M, D))
    s2 = C.c_double(0.0)
    done = C.c_int32(0)
    hist = np.zeros(max(n_iter, 1))
    llh = np.zeros(max(n_iter, 1))
    scratch = [np.empty(N), np.empty(M), np.empty((M, D)), np.empty(M), np.empty((M, D)),
               np.empty((Kk, D))]
    st = _load().fcpd_oracle_register(_p(X), M, _p(Y), N, D, _p(U), _p(lam), Kk, float(w),
                                      float(lam_reg), s0, int(n_iter), _p(T), _p(W),
                                      C.byref(s2), C.byref(done), _p(hist), _p(llh),
                                      *[_p(a) for a in scratch])
    return dict(T=T, W=W, sigma2=s2.value, iters=done.value, status=st, sigma2_0=s0,
                sigma2_hist=hist[:done.value].copy(), loglik_hist=llh[:done.value].copy())
