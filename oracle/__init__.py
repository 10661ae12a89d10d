"""FastMuyGPs oracle: plain FP64 CPU restatement of the posterior-mean path
(Algorithms 1 and 2, Eqs. 2-7 of Dunton, Priest & Muyskens).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline and reference legs may import this package.  It shares no code
with paper_2205_10879_gb300 (the CUDA path) and imports nothing from it.

Parity pins live in tests/test_oracle_pins.py (closed forms vs the Bessel form
of Eq. 3, brute-force kNN vs an all-pairs sort, SPD blocks, k = n vs the dense
GP mean of Eq. 2, interpolation and leave-one-out identities, sigma^2
invariance, long-double rounding bound, the Metropolis calibration chain of
Sec. 4.2 against the closed-form posterior of a linear response).  Parity against numbers printed in
the paper is unpinned: the paper prints no worked example.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class _Kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nu", ctypes.c_double),
                ("length_scale", ctypes.c_double), ("variance", ctypes.c_double),
                ("nugget", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64, I32, D = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        KP = ctypes.POINTER(_Kernel)
        lib.fmgp_oracle_knn.argtypes = [P, I64, I32, P, I64, I32, P, P, P]
        lib.fmgp_oracle_knn.restype = I32
        lib.fmgp_oracle_key.argtypes = [P, P, I32]
        lib.fmgp_oracle_key.restype = D
        lib.fmgp_oracle_assemble.argtypes = [P, I32, P, I32, KP, P]
        lib.fmgp_oracle_phi.argtypes = [KP, P, I64, P]
        lib.fmgp_oracle_precompute.argtypes = [P, P, I64, I32, I32, P, I32, I32, KP, P, I64, P, P]
        lib.fmgp_oracle_precompute.restype = I64
        lib.fmgp_oracle_precompute_ld.argtypes = lib.fmgp_oracle_precompute.argtypes
        lib.fmgp_oracle_precompute_ld.restype = I64
        lib.fmgp_oracle_predict.argtypes = [P, I64, I32, P, I32, P, I32, I32, KP, P, I64, P, P]
        lib.fmgp_oracle_predict_given.argtypes = [P, I32, P, I32, P, I32, I32, KP, P, I64, P, P]
        lib.fmgp_oracle_fit_predict_ld.argtypes = [P, P, I64, I32, I32, P, I32, I32, KP, P, I64,
                                                   P, P]
        lib.fmgp_oracle_loocv.argtypes = [P, P, I64, I32, I32, P, I32, I32, P, I64, KP, P, P]
        lib.fmgp_oracle_loocv.restype = I64
        lib.fmgp_oracle_loocv_ld.argtypes = lib.fmgp_oracle_loocv.argtypes
        lib.fmgp_oracle_loocv_ld.restype = I64
        lib.fmgp_oracle_muygps_predict.argtypes = [P, P, I64, I32, I32, P, I64, I32, KP, P, P]
        lib.fmgp_oracle_muygps_predict.restype = I64
        lib.fmgp_oracle_mcmc.argtypes = [P, I64, I32, P, I32, P, I32, I32, KP, P, I32, D, D, D,
                                         I32, D, D, I32, I64, P, P, P, P, P, P]
        lib.fmgp_oracle_mcmc.restype = I64
        lib.fmgp_oracle_set_threads.argtypes = [I32]
        lib.fmgp_oracle_max_threads.restype = I32
        _lib = lib
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of the
    oracle (used by the mutation test to run the pins against planted bugs)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _lib = None
        real = _build.build
        _build.build = lambda *a, **k: self.path
        try:
            _load()
        finally:
            _build.build = real
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def kernel(kind="matern", nu=1.5, length_scale=0.1, variance=1.0, nugget=1e-4):
    """Hyperparameters theta = [sigma, rho, nu, tau] of Eq. 3 (variance = sigma^2,
    nugget = tau^2).  kind is 'matern' (nu in {0.5, 1.5, 2.5}) or 'rbf'."""
    return _Kernel(0 if kind == "matern" else 1, float(nu), float(length_scale),
                   float(variance), float(nugget))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(t: int) -> None:
    _load().fmgp_oracle_set_threads(int(t))


def max_threads() -> int:
    return int(_load().fmgp_oracle_max_threads())


def key(a, b) -> float:
    """Canonical FP64 squared-distance key of two feature vectors."""
    a = _c(a, np.float64)
    b = _c(b, np.float64)
    return float(_load().fmgp_oracle_key(_p(a), _p(b), a.shape[0]))


def knn(X, Q, kq, exclude=None):
    """Indices (m x kq, int32) and keys (m x kq) of the kq nearest training
    points of each query row, ties to the lowest index.  exclude: per-query
    training index to skip (the query's own index for self-queries), or None."""
    X = _c(X, np.float64)
    Q = _c(Q, np.float64).reshape(-1, X.shape[1])
    n, d = X.shape
    m = Q.shape[0]
    idx = np.zeros((m, kq), np.int32)
    keys = np.zeros((m, kq), np.float64)
    ex = None if exclude is None else _c(exclude, np.int64)
    rc = _load().fmgp_oracle_knn(_p(X), n, d, _p(Q), m, int(kq),
                                 _p(ex) if ex is not None else None, _p(idx), _p(keys))
    if rc:
        raise ValueError("oracle knn: bad arguments")
    return idx, keys


def phi(kern, D):
    D = _c(D, np.float64).ravel()
    out = np.zeros_like(D)
    if _load().fmgp_oracle_phi(ctypes.byref(kern), _p(D), D.size, _p(out)):
        raise ValueError("oracle phi: bad kernel")
    return out


def assemble(X, S, kern):
    X = _c(X, np.float64)
    S = _c(S, np.int32)
    k = S.shape[0]
    K = np.zeros((k, k), np.float64)
    if _load().fmgp_oracle_assemble(_p(X), X.shape[1], _p(S), k, ctypes.byref(kern), _p(K)):
        raise ValueError("oracle assemble: bad arguments")
    return K


def self_knn(X, kq):
    """Self kNN table (n x kq): each training point's kq nearest others."""
    X = _c(X, np.float64)
    return knn(X, X, kq, np.arange(X.shape[0], dtype=np.int64))


def precompute(X, Y, nbr, k, kern, long_double=False, rows=None):
    """C (n x k x r, or len(rows) x k x r) and per-point status (int8) of Eq. 6."""
    X = _c(X, np.float64)
    Y = _c(Y, np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    nbr = _c(nbr, np.int32)
    n, d = X.shape
    r = Y.shape[1]
    rws = None if rows is None else _c(rows, np.int64)
    cnt = n if rws is None else rws.shape[0]
    C = np.zeros((cnt, k, r), np.float64)
    st = np.zeros(cnt, np.int8)
    fn = _load().fmgp_oracle_precompute_ld if long_double else _load().fmgp_oracle_precompute
    f = fn(_p(X), _p(Y), n, d, r, _p(nbr), nbr.shape[1], int(k), ctypes.byref(kern),
           _p(rws) if rws is not None else None, cnt, _p(C), _p(st))
    if f < 0:
        raise ValueError("oracle precompute: bad arguments")
    return C, st


def predict(X, nbr, C, kern, Z):
    """(Yhat m x r, nearest m) of Eq. 7 with a brute-force 1-NN lookup."""
    X = _c(X, np.float64)
    Z = _c(Z, np.float64).reshape(-1, X.shape[1])
    nbr = _c(nbr, np.int32)
    C = _c(C, np.float64)
    n, d = X.shape
    _, k, r = C.shape
    m = Z.shape[0]
    Yh = np.zeros((m, r), np.float64)
    near = np.zeros(m, np.int32)
    rc = _load().fmgp_oracle_predict(_p(X), n, d, _p(nbr), nbr.shape[1], _p(C), k, r,
                                     ctypes.byref(kern), _p(Z), m, _p(Yh), _p(near))
    if rc:
        raise ValueError("oracle predict: bad arguments")
    return Yh, near


def predict_given(X, nbr, C, kern, Z, nearest):
    """Eq. 7 with the nearest training point of each test row supplied."""
    X = _c(X, np.float64)
    Z = _c(Z, np.float64).reshape(-1, X.shape[1])
    nbr = _c(nbr, np.int32)
    C = _c(C, np.float64)
    nearest = _c(nearest, np.int32)
    _, k, r = C.shape
    m = Z.shape[0]
    Yh = np.zeros((m, r), np.float64)
    rc = _load().fmgp_oracle_predict_given(_p(X), X.shape[1], _p(nbr), nbr.shape[1], _p(C), k, r,
                                           ctypes.byref(kern), _p(Z), m, _p(nearest), _p(Yh))
    if rc:
        raise ValueError("oracle predict_given: bad arguments")
    return Yh


def fit_predict_ld(X, Y, nbr, k, kern, Z, nearest):
    """Eqs. 6-7 in long double end to end (rounded to FP64 only at the end)."""
    X = _c(X, np.float64)
    Y = _c(Y, np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    Z = _c(Z, np.float64).reshape(-1, X.shape[1])
    nbr = _c(nbr, np.int32)
    nearest = _c(nearest, np.int32)
    n, d = X.shape
    r = Y.shape[1]
    m = Z.shape[0]
    Yh = np.zeros((m, r), np.float64)
    rc = _load().fmgp_oracle_fit_predict_ld(_p(X), _p(Y), n, d, r, _p(nbr), nbr.shape[1], int(k),
                                            ctypes.byref(kern), _p(Z), m, _p(nearest), _p(Yh))
    if rc:
        raise ValueError("oracle fit_predict_ld: bad arguments")
    return Yh


def loocv(X, Y, nbr, k, batch, kern, long_double=False):
    """(Q, per-point squared residuals) of Eq. 5 over the batch."""
    X = _c(X, np.float64)
    Y = _c(Y, np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    nbr = _c(nbr, np.int32)
    batch = _c(batch, np.int64)
    n, d = X.shape
    r = Y.shape[1]
    b = batch.shape[0]
    res = np.zeros(b, np.float64)
    Q = np.zeros(1, np.float64)
    fn = _load().fmgp_oracle_loocv_ld if long_double else _load().fmgp_oracle_loocv
    f = fn(_p(X), _p(Y), n, d, r, _p(nbr), nbr.shape[1], int(k), _p(batch), b,
           ctypes.byref(kern), _p(res), _p(Q))
    if f < 0:
        raise ValueError("oracle loocv: bad arguments")
    return float(Q[0]), res


def predict_rows(X, nbr, rows, C, kern, Z):
    """Prediction from a subsampled precompute (the subsampling of the
    precomputed coefficients proposed in Sec. 5): C (s x k x r) holds Eq. 6
    for the training points rows[0..s) only (oracle.precompute(..., rows=rows)).
    Each test point takes its nearest centre x_rows[p] (canonical key, ties to
    the lower position p) and Eq. 7 with S_rows[p] and C[p].
    Returns (Yhat m x r, the chosen centres' training indices m)."""
    X = _c(X, np.float64)
    rows = np.asarray(rows, np.int64)
    C = _c(C, np.float64)
    pos, _ = knn(X[rows], Z, 1)
    centre = rows[pos[:, 0]]
    Cfull = np.zeros((X.shape[0],) + C.shape[1:], np.float64)
    Cfull[rows[::-1]] = C[::-1]  # a repeated row keeps its first position's coefficients
    return predict_given(X, nbr, Cfull, kern, Z, centre.astype(np.int32)), centre.astype(np.int32)


def mcmc(X, nbr, C, kern, z0, dim, lo, hi, f_obs, sigma, step, x0, noise, expo, col=0):
    """Metropolis calibration of input coordinate `dim` (Sec. 4.2).  noise and
    expo are (steps x chains) N(0,1) and Exp(1) draws.  Returns (samples
    steps x chains, accepted per chain, margin steps x chains)."""
    X = _c(X, np.float64)
    nbr = _c(nbr, np.int32)
    C = _c(C, np.float64)
    z0 = _c(z0, np.float64)
    x0 = _c(x0, np.float64)
    noise = _c(noise, np.float64)
    expo = _c(expo, np.float64)
    n, d = X.shape
    _, k, r = C.shape
    steps, chains = noise.shape
    samples = np.zeros((steps, chains), np.float64)
    margin = np.zeros((steps, chains), np.float64)
    acc = np.zeros(chains, np.int64)
    rc = _load().fmgp_oracle_mcmc(_p(X), n, d, _p(nbr), nbr.shape[1], _p(C), k, r,
                                  ctypes.byref(kern), _p(z0), int(dim), float(lo), float(hi),
                                  float(f_obs), int(col), float(sigma), float(step), int(chains),
                                  int(steps), _p(x0), _p(noise), _p(expo), _p(samples), _p(acc),
                                  _p(margin))
    if rc:
        raise ValueError("oracle mcmc: bad arguments")
    return samples, acc, margin


def muygps_predict(X, Y, Z, k, kern):
    """MuyGPs prediction (Eq. 8): (Yhat m x r, neighbour table m x k) with each
    test point's own k nearest training points."""
    X = _c(X, np.float64)
    Y = _c(Y, np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    Z = _c(Z, np.float64).reshape(-1, X.shape[1])
    n, d = X.shape
    r = Y.shape[1]
    m = Z.shape[0]
    Yh = np.zeros((m, r), np.float64)
    N = np.zeros((m, k), np.int32)
    f = _load().fmgp_oracle_muygps_predict(_p(X), _p(Y), n, d, r, _p(Z), m, int(k),
                                           ctypes.byref(kern), _p(Yh), _p(N))
    if f < 0:
        raise ValueError("oracle muygps_predict: bad arguments")
    return Yh, N
