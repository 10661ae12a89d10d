"""ctypes binding of libfmgp.so: argument marshalling only.

Every compute step runs in the CUDA library; this module turns torch tensors
into device pointers and sizes, picks the current torch stream, and turns
status codes into exceptions.  There is no CPU fallback: without the built
library every call raises."""
import ctypes
import os

import torch

from . import build as _build

(FMGP_OK, FMGP_EINVAL, FMGP_ENOMEM, FMGP_ECUDA, FMGP_ENOTSPD, FMGP_ETIMEOUT, FMGP_EUNSUPPORTED,
 FMGP_EIO) = range(8)
F32, F64 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
KERNEL_MATERN, KERNEL_RBF = 0, 1
BLOCK_OK, BLOCK_NOT_SPD, BLOCK_FP64_RETRY, BLOCK_BAD_INDEX = range(4)

_STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTSPD", 5: "ETIMEOUT", 6: "EUNSUPPORTED"}


class FmgpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fmgp {_STATUS.get(code, code)}: {msg}")
        self.code = code


class Kernel(ctypes.Structure):
    """fmgp_kernel: sigma^2 phi(d) with phi Matern (nu in {0.5,1.5,2.5}) or RBF;
    nugget tau^2 on the diagonal of training blocks."""
    _fields_ = [("kind", ctypes.c_int32), ("nu", ctypes.c_double),
                ("length_scale", ctypes.c_double), ("variance", ctypes.c_double),
                ("nugget", ctypes.c_double)]


def make_kernel(kind="matern", nu=1.5, length_scale=0.1, variance=1.0, nugget=1e-4):
    return Kernel(KERNEL_MATERN if kind == "matern" else KERNEL_RBF, float(nu),
                  float(length_scale), float(variance), float(nugget))


class ModelInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("r", ctypes.c_int32),
                ("k", ctypes.c_int32), ("nbr_ld", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("kernel", Kernel)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_int64), ("host_staging_bytes", ctypes.c_int64),
                ("streams", ctypes.c_int32), ("max_batch_points", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("points", ctypes.c_int64), ("mean_batch_requests", ctypes.c_double)]


_lib = None


def lib_path():
    return _build.TARGET


def load(build_if_missing=True):
    """Load libfmgp.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.TARGET):
        raise RuntimeError("libfmgp.so is not built; run paper_2205_10879_gb300.build.build()")
    lib = ctypes.CDLL(_build.TARGET)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    KP = ctypes.POINTER(Kernel)
    lib.fmgp_build_knn.argtypes = [P, I32, I64, I32, I32, P, P, I32, P]
    lib.fmgp_precompute.argtypes = [P, I32, P, I64, I32, I32, P, I32, I32, KP, I32, P, P, P]
    lib.fmgp_predict.argtypes = [P, I32, I64, I32, P, I32, P, I32, I32, KP, I32, P, I64, P, P, P]
    lib.fmgp_precompute_rows.argtypes = [P, I32, P, I64, I32, I32, P, I32, I32, P, I64, KP, I32,
                                         P, P, P]
    lib.fmgp_predict_rows.argtypes = [P, I32, I64, I32, P, I32, P, I64, P, I32, I32, KP, I32, P,
                                      I64, P, P, P]
    lib.fmgp_loocv_objective.argtypes = [P, I32, P, I64, I32, I32, P, I32, I32, P, I64, KP, I32,
                                         P, P, P]
    for f in ("fmgp_build_knn", "fmgp_precompute", "fmgp_predict", "fmgp_loocv_objective"):
        getattr(lib, f).restype = I32
    lib.fmgp_last_error.restype = ctypes.c_char_p
    lib.fmgp_version.restype = ctypes.c_char_p
    lib.fmgp_peak_probe.argtypes = [I32, ctypes.POINTER(ctypes.c_double), P]
    lib.fmgp_df_eval.argtypes = [I32, P, I64, P, P]
    lib.fmgp_df_eval.restype = I32
    lib.fmgp_loocv_objective_device.argtypes = [P, I32, P, I64, I32, I32, P, I32, I32, P, I64,
                                                KP, I32, P, P, P, P]
    lib.fmgp_loocv_objective_device.restype = I32
    lib.fmgp_autotune_choice.argtypes = [I32, I32, I32, I32, I32, ctypes.POINTER(I32),
                                         ctypes.POINTER(I32), ctypes.POINTER(I32)]
    lib.fmgp_autotune_choice.restype = I32
    lib.fmgp_model_get_info.argtypes = [P, ctypes.POINTER(ModelInfo)]
    lib.fmgp_model_get_info.restype = I32
    lib.fmgp_model_save.argtypes = [P, ctypes.c_char_p, P]
    lib.fmgp_model_save.restype = I32
    lib.fmgp_model_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p), P]
    lib.fmgp_model_load.restype = I32
    lib.fmgp_context_create.argtypes = [I64, ctypes.POINTER(ctypes.c_void_p)]
    lib.fmgp_context_create.restype = I32
    lib.fmgp_context_bind.argtypes = [P]
    lib.fmgp_context_bind.restype = I32
    lib.fmgp_context_bytes_in_use.argtypes = [P]
    lib.fmgp_context_bytes_in_use.restype = I64
    lib.fmgp_context_destroy.argtypes = [P]
    lib.fmgp_context_destroy.restype = I32
    lib.fmgp_peak_probe.restype = I32
    lib.fmgp_kernel_launches.restype = ctypes.c_uint64
    lib.fmgp_muygps_predict.argtypes = [P, I32, P, I64, I32, I32, P, I64, I32, KP, I32, P, P, P]
    lib.fmgp_muygps_predict.restype = I32
    lib.fmgp_tune_set.argtypes = [ctypes.c_char_p, ctypes.c_double]
    lib.fmgp_tune_set.restype = I32
    lib.fmgp_tune_get.argtypes = [ctypes.c_char_p]
    lib.fmgp_tune_get.restype = ctypes.c_double
    lib.fmgp_diag_counter.argtypes = [I32]
    lib.fmgp_diag_counter.restype = I64
    lib.fmgp_autotune_precompute.argtypes = [P, I32, P, I64, I32, I32, P, I32, I32, KP, I32, I64,
                                             ctypes.POINTER(I32), P]
    lib.fmgp_autotune_precompute.restype = I32
    lib.fmgp_autotune_knn.argtypes = [P, I32, I64, I32, I32, ctypes.POINTER(ctypes.c_double), P]
    lib.fmgp_autotune_knn.restype = I32
    lib.fmgp_autotune_reset.restype = I32
    lib.fmgp_model_create.argtypes = [P, I32, I64, I32, P, I32, P, I32, I32, KP, I32, I32,
                                      ctypes.POINTER(ctypes.c_void_p), P]
    lib.fmgp_model_predict.argtypes = [P, P, I64, P, P, P]
    lib.fmgp_model_destroy.argtypes = [P]
    lib.fmgp_model_device_bytes.argtypes = [P]
    lib.fmgp_model_device_bytes.restype = I64
    D = ctypes.c_double
    lib.fmgp_model_mcmc.argtypes = [P, P, I32, D, D, D, I32, D, D, I64, I64, P, P, P, P, P, P, P]
    lib.fmgp_server_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), I32,
                                       ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]
    lib.fmgp_server_submit.argtypes = [P, I32, P, I64, P, P, ctypes.POINTER(ctypes.c_uint64)]
    lib.fmgp_server_wait.argtypes = [P, ctypes.c_uint64, I32]
    lib.fmgp_server_request_times.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]
    lib.fmgp_server_release.argtypes = [P, ctypes.c_uint64]
    lib.fmgp_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.fmgp_server_destroy.argtypes = [P]
    for f in ("fmgp_model_create", "fmgp_model_predict", "fmgp_model_destroy", "fmgp_server_create",
              "fmgp_server_submit", "fmgp_server_wait", "fmgp_server_request_times",
              "fmgp_server_release", "fmgp_server_get_stats", "fmgp_server_destroy"):
        getattr(lib, f).restype = I32
    _lib = lib
    return lib


def _check(rc):
    if rc != FMGP_OK:
        raise FmgpError(rc, load().fmgp_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dev(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _dtype_code(X):
    if X.dtype == torch.float64:
        return F64
    if X.dtype == torch.float32:
        return F32
    raise TypeError("features must be float32 or float64")


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def fmgp_build_knn(X, kq, nbr_out=None, dist_out=None, with_dist=False, stream=None):
    """Self kNN table of X (n x d): (nbr n x kq int32, dist n x kq float64 or None)."""
    _dev(X, "X")
    n, d = X.shape
    if nbr_out is None:
        nbr_out = torch.empty((n, kq), dtype=torch.int32, device=X.device)
    if with_dist and dist_out is None:
        dist_out = torch.empty((n, kq), dtype=torch.float64, device=X.device)
    _check(load().fmgp_build_knn(_ptr(X), _dtype_code(X), n, d, int(kq), _ptr(nbr_out),
                                 _ptr(dist_out), 0, _stream(stream)))
    return nbr_out, dist_out


def coeff_shape(n, k, r, precision):
    return (n, k, r) if precision == PREC_FP64 else (n, k, r, 2)


def fmgp_precompute(X, Y, nbr, k, kernel, precision=PREC_FP64, C_out=None, status_out=None,
                    with_status=True, stream=None):
    """C (n x k x r float64, or n x k x r x 2 float32 double-float pairs when
    precision is PREC_MIXED) and the per-point status (int8) of Eq. 6."""
    _dev(X, "X"); _dev(Y, "Y"); _dev(nbr, "nbr")
    n, d = X.shape
    r = Y.shape[1]
    if C_out is None:
        C_out = torch.empty(coeff_shape(n, k, r, precision),
                            dtype=torch.float64 if precision == PREC_FP64 else torch.float32,
                            device=X.device)
    if with_status and status_out is None:
        status_out = torch.empty(n, dtype=torch.int8, device=X.device)
    _check(load().fmgp_precompute(_ptr(X), _dtype_code(X), _ptr(Y), n, d, r, _ptr(nbr),
                                  nbr.shape[1], int(k), ctypes.byref(kernel), int(precision),
                                  _ptr(C_out), _ptr(status_out), _stream(stream)))
    return C_out, status_out


def fmgp_predict(X, nbr, C, k, kernel, Z, precision=PREC_FP64, Yhat_out=None, nearest_out=None,
                 with_nearest=True, stream=None):
    """Eq. 7 posterior means (m x r float64) and j* (m int32)."""
    _dev(X, "X"); _dev(nbr, "nbr"); _dev(C, "C"); _dev(Z, "Z")
    n, d = X.shape
    r = C.shape[2]
    m = Z.shape[0]
    if Yhat_out is None:
        Yhat_out = torch.empty((m, r), dtype=torch.float64, device=X.device)
    if with_nearest and nearest_out is None:
        nearest_out = torch.empty(m, dtype=torch.int32, device=X.device)
    _check(load().fmgp_predict(_ptr(X), _dtype_code(X), n, d, _ptr(nbr), nbr.shape[1], _ptr(C),
                               int(k), r, ctypes.byref(kernel), int(precision), _ptr(Z), m,
                               _ptr(Yhat_out), _ptr(nearest_out), _stream(stream)))
    return Yhat_out, nearest_out


def fmgp_precompute_rows(X, Y, nbr, k, kernel, rows, precision=PREC_FP64, C_out=None,
                         status_out=None, with_status=True, stream=None):
    """Eq. 6 for the centres rows (int32 CUDA tensor of s training indices):
    (C s x k x r [x 2 for PREC_MIXED], status s int8)."""
    _dev(X, "X"); _dev(Y, "Y"); _dev(nbr, "nbr"); _dev(rows, "rows")
    if rows.dtype != torch.int32:
        raise TypeError("rows must be int32")
    n, d = X.shape
    r = Y.shape[1]
    s = rows.shape[0]
    if C_out is None:
        C_out = torch.empty(coeff_shape(s, k, r, precision),
                            dtype=torch.float64 if precision == PREC_FP64 else torch.float32,
                            device=X.device)
    if with_status and status_out is None:
        status_out = torch.empty(s, dtype=torch.int8, device=X.device)
    _check(load().fmgp_precompute_rows(_ptr(X), _dtype_code(X), _ptr(Y), n, d, r, _ptr(nbr),
                                       nbr.shape[1], int(k), _ptr(rows), s, ctypes.byref(kernel),
                                       int(precision), _ptr(C_out), _ptr(status_out),
                                       _stream(stream)))
    return C_out, status_out


def fmgp_predict_rows(X, nbr, rows, C, k, kernel, Z, precision=PREC_FP64, Yhat_out=None,
                      nearest_out=None, with_nearest=True, stream=None):
    """Prediction from fmgp_precompute_rows: (Yhat m x r, centre index m int32)."""
    _dev(X, "X"); _dev(nbr, "nbr"); _dev(rows, "rows"); _dev(C, "C"); _dev(Z, "Z")
    if rows.dtype != torch.int32:
        raise TypeError("rows must be int32")
    n, d = X.shape
    r = C.shape[2]
    m = Z.shape[0]
    if Yhat_out is None:
        Yhat_out = torch.empty((m, r), dtype=torch.float64, device=X.device)
    if with_nearest and nearest_out is None:
        nearest_out = torch.empty(m, dtype=torch.int32, device=X.device)
    _check(load().fmgp_predict_rows(_ptr(X), _dtype_code(X), n, d, _ptr(nbr), nbr.shape[1],
                                    _ptr(rows), rows.shape[0], _ptr(C), int(k), r,
                                    ctypes.byref(kernel), int(precision), _ptr(Z), m,
                                    _ptr(Yhat_out), _ptr(nearest_out), _stream(stream)))
    return Yhat_out, nearest_out


def df_eval(fn, x, stream=None):
    """Diagnostic: the mixed path's double-float exp(-x) (fn "exp_neg") or
    sqrt(x) (fn "sqrt") of a float64 device tensor, as float64."""
    _dev(x, "x")
    y = torch.empty_like(x)
    _check(load().fmgp_df_eval({"exp_neg": 0, "sqrt": 1}[fn], _ptr(x), x.numel(), _ptr(y),
                               _stream(stream)))
    return y


def peak_probe(pipe, stream=None):
    """Measured FMA throughput of the current device in flop/s: pipe "fp32"
    or "fp64" (fmgp_peak_probe; synchronises the stream)."""
    code = {"fp32": 0, "fp64": 1}[pipe]
    v = ctypes.c_double(0.0)
    _check(load().fmgp_peak_probe(code, ctypes.byref(v), _stream(stream)))
    return v.value


def fmgp_loocv_objective_device(X, Y, nbr, k, batch, kernel, precision=PREC_FP64, Q_out=None,
                                fails_out=None, resid_out=None, stream=None):
    """Eq. 5 objective into a 1-element float64 CUDA tensor without
    synchronising (graph-capturable): (Q, fails or None, residuals or None)."""
    _dev(X, "X"); _dev(Y, "Y"); _dev(nbr, "nbr"); _dev(batch, "batch")
    n, d = X.shape
    r = Y.shape[1]
    b = batch.shape[0]
    if Q_out is None:
        Q_out = torch.empty(1, dtype=torch.float64, device=X.device)
    _check(load().fmgp_loocv_objective_device(
        _ptr(X), _dtype_code(X), _ptr(Y), n, d, r, _ptr(nbr), nbr.shape[1], int(k), _ptr(batch),
        b, ctypes.byref(kernel), int(precision), _ptr(Q_out), _ptr(fails_out), _ptr(resid_out),
        _stream(stream)))
    return Q_out, fails_out, resid_out


def fmgp_muygps_predict(X, Y, Z, k, kernel, precision=PREC_FP64, Yhat_out=None, nbr_out=None,
                        with_nbr=False, stream=None):
    """MuyGPs prediction (Eq. 8): (Yhat m x r, neighbour table m x k or None)."""
    _dev(X, "X"); _dev(Y, "Y"); _dev(Z, "Z")
    n, d = X.shape
    r = Y.shape[1]
    m = Z.shape[0]
    if Yhat_out is None:
        Yhat_out = torch.empty((m, r), dtype=torch.float64, device=X.device)
    if with_nbr and nbr_out is None:
        nbr_out = torch.empty((m, k), dtype=torch.int32, device=X.device)
    _check(load().fmgp_muygps_predict(_ptr(X), _dtype_code(X), _ptr(Y), n, d, r, _ptr(Z), m,
                                      int(k), ctypes.byref(kernel), int(precision),
                                      _ptr(Yhat_out), _ptr(nbr_out), _stream(stream)))
    return Yhat_out, nbr_out


def fmgp_loocv_objective(X, Y, nbr, k, batch, kernel, precision=PREC_FP64, resid_out=None,
                         stream=None, raise_on_not_spd=True):
    """Eq. 5 objective Q over the batch (host float) and per-point residuals."""
    _dev(X, "X"); _dev(Y, "Y"); _dev(nbr, "nbr"); _dev(batch, "batch")
    n, d = X.shape
    r = Y.shape[1]
    b = batch.shape[0]
    if resid_out is None:
        resid_out = torch.empty(b, dtype=torch.float64, device=X.device)
    Q = ctypes.c_double(0.0)
    rc = load().fmgp_loocv_objective(_ptr(X), _dtype_code(X), _ptr(Y), n, d, r, _ptr(nbr),
                                     nbr.shape[1], int(k), _ptr(batch), b, ctypes.byref(kernel),
                                     int(precision), ctypes.byref(Q), _ptr(resid_out),
                                     _stream(stream))
    if rc == FMGP_ENOTSPD and not raise_on_not_spd:
        return float("nan"), resid_out
    _check(rc)
    return Q.value, resid_out


def version():
    return load().fmgp_version().decode()


def fmgp_autotune_precompute(X, Y, nbr, k, kernel, precision=PREC_FP64, sample_rows=20_000,
                             stream=None):
    """Pick (and cache) the fastest warps-per-CTA for this precompute shape."""
    n, d = X.shape
    w = ctypes.c_int32(0)
    _check(load().fmgp_autotune_precompute(_ptr(X), _dtype_code(X), _ptr(Y), n, d, Y.shape[1],
                                           _ptr(nbr), nbr.shape[1], int(k), ctypes.byref(kernel),
                                           int(precision), int(sample_rows), ctypes.byref(w),
                                           _stream(stream)))
    return w.value


def fmgp_autotune_knn(X, kq, stream=None):
    """Pick (and cache) the fastest grid occupancy for this kNN shape (d <= 3)."""
    n, d = X.shape
    t = ctypes.c_double(0)
    _check(load().fmgp_autotune_knn(_ptr(X), _dtype_code(X), n, d, int(kq), ctypes.byref(t),
                                    _stream(stream)))
    return t.value


def autotune_choice(k, d, r, precision, dtype=torch.float64):
    """The cached launch shape for a precompute key: (warps per CTA, Cholesky
    panel width, persistent 1 / eight waves 0); 0, 0, -1 where nothing is
    cached (the defaults are used)."""
    w, p, q = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().fmgp_autotune_choice(int(precision), int(k), int(d), int(r),
                                       F64 if dtype == torch.float64 else F32,
                                       ctypes.byref(w), ctypes.byref(p), ctypes.byref(q)))
    return w.value, p.value, q.value


def autotune_reset():
    _check(load().fmgp_autotune_reset())


def tune_set(key, value):
    _check(load().fmgp_tune_set(key.encode(), float(value)))


def tune_get(key):
    return float(load().fmgp_tune_get(key.encode()))


def diag_counter(which):
    return int(load().fmgp_diag_counter(int(which)))


def kernel_launches():
    """Kernels libfmgp has enqueued since it was loaded."""
    return int(load().fmgp_kernel_launches())


MODEL_BORROW, MODEL_COPY = 0, 1


class FmgpModel:
    """fmgp_model_create / fmgp_model_predict / fmgp_model_destroy.  A
    borrowing model keeps references to the tensors X, nbr and C for its
    lifetime; with copy=True the library keeps copies of its own and the
    tensors may be freed or reused after construction."""

    def __init__(self, X, nbr, C, k, kernel, precision=PREC_FP64, stream=None, copy=False):
        _dev(X, "X"); _dev(nbr, "nbr"); _dev(C, "C")
        self.k, self.kernel, self.precision = k, kernel, precision
        self.X, self.nbr, self.C = (None, None, None) if copy else (X, nbr, C)
        self.n, self.d = X.shape
        self.r = C.shape[2]
        self.dtype = X.dtype
        h = ctypes.c_void_p()
        _check(load().fmgp_model_create(_ptr(X), _dtype_code(X), self.n, self.d, _ptr(nbr),
                                        nbr.shape[1], _ptr(C), int(k), self.r,
                                        ctypes.byref(kernel), int(precision),
                                        MODEL_COPY if copy else MODEL_BORROW, ctypes.byref(h),
                                        _stream(stream)))
        self.handle = h

    @classmethod
    def load(cls, path, stream=None):
        """fmgp_model_load: a model read from a file (it owns its X, table and C)."""
        h = ctypes.c_void_p()
        _check(load().fmgp_model_load(os.fsencode(path), ctypes.byref(h), _stream(stream)))
        self = cls.__new__(cls)
        self.handle = h
        self.X = self.nbr = self.C = None
        info = ModelInfo()
        _check(load().fmgp_model_get_info(h, ctypes.byref(info)))
        self.n, self.d, self.r, self.k = int(info.n), int(info.d), int(info.r), int(info.k)
        self.kernel = Kernel(info.kernel.kind, info.kernel.nu, info.kernel.length_scale,
                             info.kernel.variance, info.kernel.nugget)
        self.precision = int(info.precision)
        self.dtype = torch.float64 if info.dtype == F64 else torch.float32
        return self

    def save(self, path, stream=None):
        """fmgp_model_save: write the fitted model to a file."""
        _check(load().fmgp_model_save(self.handle, os.fsencode(path), _stream(stream)))

    def predict(self, Z, Yhat_out=None, nearest_out=None, with_nearest=True, stream=None):
        _dev(Z, "Z")
        m = Z.shape[0]
        if Yhat_out is None:
            Yhat_out = torch.empty((m, self.r), dtype=torch.float64, device=Z.device)
        if with_nearest and nearest_out is None:
            nearest_out = torch.empty(m, dtype=torch.int32, device=Z.device)
        _check(load().fmgp_model_predict(self.handle, _ptr(Z), m, _ptr(Yhat_out),
                                         _ptr(nearest_out), _stream(stream)))
        return Yhat_out, nearest_out

    def device_bytes(self):
        return int(load().fmgp_model_device_bytes(self.handle))

    def mcmc(self, z0, dim, lo, hi, f_obs, sigma, step, x0, noise, expo, col=0,
             samples_out=None, accepted_out=None, x_out=None, with_samples=True, stream=None):
        """fmgp_model_mcmc: z0 (d) and x0 (chains) host arrays; noise and expo
        CUDA tensors (steps x chains FP64).  Returns (samples steps x chains or
        None, accepted per chain, final states), all on the device."""
        import numpy as np
        z0 = np.ascontiguousarray(z0, dtype=np.float64)
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        _dev(noise, "noise"); _dev(expo, "expo")
        if noise.dtype != torch.float64 or expo.dtype != torch.float64:
            raise TypeError("noise and expo must be float64")
        steps, chains = noise.shape
        if tuple(expo.shape) != (steps, chains) or x0.shape[0] != chains:
            raise ValueError("noise, expo must be steps x chains and x0 must have chains entries")
        if z0.shape[0] != self.d:
            raise ValueError("z0 must have d entries")
        dev = noise.device
        if with_samples and samples_out is None:
            samples_out = torch.empty((steps, chains), dtype=torch.float64, device=dev)
        if accepted_out is None:
            accepted_out = torch.empty(chains, dtype=torch.int64, device=dev)
        if x_out is None:
            x_out = torch.empty(chains, dtype=torch.float64, device=dev)
        _check(load().fmgp_model_mcmc(self.handle, z0.ctypes.data_as(ctypes.c_void_p), int(dim),
                                      float(lo), float(hi), float(f_obs), int(col), float(sigma),
                                      float(step), int(chains), int(steps),
                                      x0.ctypes.data_as(ctypes.c_void_p), _ptr(noise), _ptr(expo),
                                      _ptr(samples_out if with_samples else None),
                                      _ptr(accepted_out), _ptr(x_out), _stream(stream)))
        return samples_out if with_samples else None, accepted_out, x_out

    def close(self):
        if self.handle:
            load().fmgp_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """fmgp_context_*: a reserved, size-capped workspace pool on the current
    device; `with ctx:` binds it to this thread for the block."""

    def __init__(self, nbytes):
        h = ctypes.c_void_p()
        _check(load().fmgp_context_create(int(nbytes), ctypes.byref(h)))
        self.handle = h

    def bind(self):
        _check(load().fmgp_context_bind(self.handle))

    @staticmethod
    def unbind():
        _check(load().fmgp_context_bind(None))

    def bytes_in_use(self):
        return int(load().fmgp_context_bytes_in_use(self.handle))

    def __enter__(self):
        self.bind()
        return self

    def __exit__(self, *exc):
        Context.unbind()

    def close(self):
        if self.handle:
            _check(load().fmgp_context_destroy(self.handle))
            self.handle = None


class FmgpServer:
    """fmgp_server_*: continuous-batching prediction service over resident
    models.  submit() takes host numpy test points and returns the request id;
    results land in host arrays returned by result()."""

    def __init__(self, models, device_budget_bytes=1 << 28, host_staging_bytes=1 << 28,
                 streams=4, max_batch_points=1 << 20):
        self.models = list(models)
        arr = (ctypes.c_void_p * len(self.models))(*[m.handle for m in self.models])
        cfg = ServerConfig(int(device_budget_bytes), int(host_staging_bytes), int(streams),
                           int(max_batch_points))
        h = ctypes.c_void_p()
        _check(load().fmgp_server_create(arr, len(self.models), ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self.live = {}

    def submit(self, model, Z, with_nearest=False):
        md = self.models[model]
        import numpy as np
        Z = np.ascontiguousarray(Z, dtype=np.float64 if md.dtype == torch.float64 else np.float32)
        m = Z.shape[0]
        Y = np.empty((m, md.r), np.float64)
        N = np.empty(m, np.int32) if with_nearest else None
        rid = ctypes.c_uint64()
        _check(load().fmgp_server_submit(self.handle, int(model), Z.ctypes.data_as(ctypes.c_void_p), m,
                                         Y.ctypes.data_as(ctypes.c_void_p),
                                         N.ctypes.data_as(ctypes.c_void_p) if N is not None else None,
                                         ctypes.byref(rid)))
        self.live[rid.value] = (Z, Y, N)
        return rid.value

    def wait(self, rid, timeout_ms=-1):
        rc = load().fmgp_server_wait(self.handle, ctypes.c_uint64(rid), int(timeout_ms))
        if rc == FMGP_ETIMEOUT:
            return False
        _check(rc)
        return True

    def result(self, rid):
        _, Y, N = self.live[rid]
        return Y, N

    def times(self, rid):
        q = ctypes.c_double()
        t = ctypes.c_double()
        _check(load().fmgp_server_request_times(self.handle, ctypes.c_uint64(rid), ctypes.byref(q),
                                                ctypes.byref(t)))
        return q.value, t.value

    def release(self, rid):
        _check(load().fmgp_server_release(self.handle, ctypes.c_uint64(rid)))
        return self.live.pop(rid)

    def stats(self):
        st = ServerStats()
        _check(load().fmgp_server_get_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            load().fmgp_server_destroy(self.handle)
            self.handle = None
