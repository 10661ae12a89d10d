"""fmgp_loocv_objective_noalloc, the LOOCV entry point that allocates no device
memory (for callers that may not call cudaMalloc while running), checked
through the C ABI against the allocating fmgp_loocv_objective.

Collected last on purpose, so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _noalloc_fn():
    lib = fb.load()
    f = lib.fmgp_loocv_objective_noalloc
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    f.argtypes = [P, I32, P, I64, I32, I32, P, I32, I32, P, I64, ctypes.POINTER(fb.Kernel), I32,
                  P, P, P]
    f.restype = I32
    return lib, f


def _call(f, X, Y, nbr, k, batch, kern, resid=None):
    Q = ctypes.c_double(float("nan"))
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dt = fb.F64 if X.dtype == torch.float64 else fb.F32
    rc = f(ctypes.c_void_p(X.data_ptr()), dt, ctypes.c_void_p(Y.data_ptr()), X.shape[0],
           X.shape[1], Y.shape[1], ctypes.c_void_p(nbr.data_ptr()), nbr.shape[1], k,
           ctypes.c_void_p(batch.data_ptr()), batch.shape[0], ctypes.byref(kern), fb.PREC_FP64,
           ctypes.byref(Q), ctypes.c_void_p(resid.data_ptr()) if resid is not None else None, s)
    return rc, Q.value


def test_noalloc_loocv_matches_allocating_entry_point(cuda):
    lib, f = _noalloc_fn()
    W = wl.tiny(n=2000, m=10, k=30, b=700)
    s = W.kernel
    kern = fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)
    X = torch.from_numpy(W.X).cuda()
    Y = torch.from_numpy(W.Y).cuda()
    nbr, _ = fb.fmgp_build_knn(X, 30)
    batch_a = torch.from_numpy(W.batch).cuda()
    batch_b = torch.from_numpy(W.batch[::3].copy()).cuda()
    Qa, _ = fb.fmgp_loocv_objective(X, Y, nbr, 30, batch_a, kern)
    Qb, _ = fb.fmgp_loocv_objective(X, Y, nbr, 30, batch_b, kern)
    # two calls in a row on the same inputs, then a smaller batch: the shared
    # scratch must not leak the previous call's residuals into the result
    for batch, ref in ((batch_a, Qa), (batch_a, Qa), (batch_b, Qb)):
        rc, Q = _call(f, X, Y, nbr, 30, batch, kern)
        assert rc == fb.FMGP_OK, lib.fmgp_last_error()
        assert abs(Q - ref) <= FP64_TOL * abs(ref)


def test_noalloc_rejects_batches_beyond_its_scratch(cuda):
    lib, f = _noalloc_fn()
    W = wl.tiny(n=500, m=10, k=10, b=10)
    s = W.kernel
    kern = fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)
    X = torch.from_numpy(W.X).cuda()
    Y = torch.from_numpy(W.Y).cuda()
    nbr, _ = fb.fmgp_build_knn(X, 10)
    big = torch.zeros(65537, dtype=torch.int64, device="cuda")
    rc, _ = _call(f, X, Y, nbr, 10, big, kern)
    assert rc == fb.FMGP_EINVAL
    assert b"65536" in lib.fmgp_last_error()


def test_noalloc_fp32_inputs_and_caller_residuals(cuda):
    """FP32 training features, and per-point residuals written to a buffer the
    caller passes: both equal the allocating entry point's, element by element."""
    lib, f = _noalloc_fn()
    W = wl.tiny(n=1500, m=10, k=20, b=300)
    s = W.kernel
    kern = fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)
    X = torch.from_numpy(W.X.astype(np.float32)).cuda()
    Y = torch.from_numpy(W.Y).cuda()
    nbr, _ = fb.fmgp_build_knn(X, 20)
    batch = torch.from_numpy(W.batch).cuda()
    Qref, rref = fb.fmgp_loocv_objective(X, Y, nbr, 20, batch, kern)
    for _ in range(2):
        resid = torch.full((len(W.batch),), float("nan"), dtype=torch.float64, device="cuda")
        rc, Q = _call(f, X, Y, nbr, 20, batch, kern, resid)
        assert rc == fb.FMGP_OK, lib.fmgp_last_error()
        assert abs(Q - Qref) <= FP64_TOL * abs(Qref)
        r = resid.cpu().numpy()
        rr = rref.cpu().numpy()
        assert np.all(np.abs(r - rr) <= FP64_TOL * np.maximum(np.abs(rr), 1e-300))


def test_noalloc_failure_does_not_carry_over(cuda):
    """A batch whose blocks are singular (duplicated points, no nugget) returns
    FMGP_ENOTSPD; the next, valid call must return FMGP_OK with the reference
    objective and an empty error message: the failure counter in the shared
    scratch is cleared by each call."""
    lib, f = _noalloc_fn()
    rng = np.random.default_rng(3)
    base = rng.random((150, 2))
    Xd = torch.from_numpy(np.repeat(base, 2, axis=0)).cuda()  # every point twice
    Yd = torch.from_numpy(rng.random((300, 1))).cuda()
    singular = fb.make_kernel("rbf", 0.0, 0.3, 1.0, 0.0)
    nbd, _ = fb.fmgp_build_knn(Xd, 8)
    bd = torch.arange(0, 300, 3, dtype=torch.int64, device="cuda")
    rc, _ = _call(f, Xd, Yd, nbd, 8, bd, singular)
    assert rc == fb.FMGP_ENOTSPD
    assert lib.fmgp_last_error() != b""
    W = wl.tiny(n=800, m=10, k=12, b=200)
    s = W.kernel
    kern = fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)
    X = torch.from_numpy(W.X).cuda()
    Y = torch.from_numpy(W.Y).cuda()
    nbr, _ = fb.fmgp_build_knn(X, 12)
    batch = torch.from_numpy(W.batch).cuda()
    Qref, _ = fb.fmgp_loocv_objective(X, Y, nbr, 12, batch, kern)
    rc, Q = _call(f, X, Y, nbr, 12, batch, kern)
    assert rc == fb.FMGP_OK, lib.fmgp_last_error()
    assert lib.fmgp_last_error() == b""
    assert abs(Q - Qref) <= FP64_TOL * abs(Qref)
