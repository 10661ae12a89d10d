"""Workspace contexts, allocation failure and the finite-input check.

- A bound context (a reserved, size-capped pool) serves every entry point's
  workspace: results equal the default pool's bit for bit, and the context
  holds nothing once the work is done.
- With workspace allocations refused (a context too small, or the host-side
  failure hook), every entry point returns FMGP_ENOMEM and nothing is left
  allocated; the next unhindered call succeeds.
- With "check_finite" on, a NaN or an infinity in X, Y or Z is refused with
  FMGP_EINVAL before anything else runs."""
import numpy as np
import pytest
import torch

from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import dev

pytestmark = pytest.mark.gpu


def _inputs():
    W = wl.tiny(n=3000, m=400, k=30, b=300)
    s = W.kernel
    return W, fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)


def _pipeline(W, gk, prec):
    X, Y, Z, B = dev(W.X), dev(W.Y), dev(W.Z), dev(W.batch)
    nbr, _ = fb.fmgp_build_knn(X, 30)
    C, st = fb.fmgp_precompute(X, Y, nbr, 30, gk, prec)
    yh, near = fb.fmgp_predict(X, nbr, C, 30, gk, Z, prec)
    Q, res = fb.fmgp_loocv_objective(X, Y, nbr, 30, B, gk, prec)
    ym, _ = fb.fmgp_muygps_predict(X, Y, Z, 30, gk, prec)
    rows = torch.arange(0, W.n, 3, dtype=torch.int32, device="cuda")
    Cr, _ = fb.fmgp_precompute_rows(X, Y, nbr, 30, gk, rows, prec)
    yr, _ = fb.fmgp_predict_rows(X, nbr, rows, Cr, 30, gk, Z, prec)
    torch.cuda.synchronize()
    return [nbr, C, st, yh, near, torch.tensor([Q]), res, ym, Cr, yr]


@pytest.mark.parametrize("prec", [fb.PREC_FP64, fb.PREC_MIXED])
def test_bound_context_gives_the_same_results(cuda, prec):
    W, gk = _inputs()
    ref = _pipeline(W, gk, prec)
    ctx = fb.Context(256 << 20)
    try:
        with ctx:
            got = _pipeline(W, gk, prec)
        assert all(torch.equal(a, b) for a, b in zip(ref, got))
        torch.cuda.synchronize()
        assert ctx.bytes_in_use() == 0
    finally:
        ctx.close()


def _each_entry_point(W, gk, prec):
    """Call every entry point once; return their status codes."""
    X, Y, Z, B = dev(W.X), dev(W.Y), dev(W.Z), dev(W.batch)
    nbr = torch.zeros((W.n, 30), dtype=torch.int32, device="cuda")
    nbr[:, :] = torch.arange(1, 31, dtype=torch.int32, device="cuda")
    C = torch.zeros(fb.coeff_shape(W.n, 30, 1, prec),
                    dtype=torch.float64 if prec == fb.PREC_FP64 else torch.float32, device="cuda")
    rows = torch.arange(0, 100, dtype=torch.int32, device="cuda")
    calls = {
        "build_knn": lambda: fb.fmgp_build_knn(X, 30),
        "precompute": lambda: fb.fmgp_precompute(X, Y, nbr, 30, gk, prec),
        "predict": lambda: fb.fmgp_predict(X, nbr, C, 30, gk, Z, prec),
        "loocv": lambda: fb.fmgp_loocv_objective(X, Y, nbr, 30, B, gk, prec),
        "muygps": lambda: fb.fmgp_muygps_predict(X, Y, Z, 30, gk, prec),
        "precompute_rows": lambda: fb.fmgp_precompute_rows(X, Y, nbr, 30, gk, rows, prec),
        "predict_rows": lambda: fb.fmgp_predict_rows(X, nbr, rows, C[:100].contiguous(), 30, gk,
                                                     Z, prec),
        "model": lambda: fb.FmgpModel(X, nbr, C, 30, gk, prec),
    }
    out = {}
    for name, f in calls.items():
        try:
            f()
            out[name] = fb.FMGP_OK
        except fb.FmgpError as e:
            out[name] = e.code
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec", [fb.PREC_FP64, fb.PREC_MIXED])
def test_injected_allocation_failure(cuda, prec):
    W, gk = _inputs()
    fb.tune_set("fail_alloc_after", 0)
    try:
        codes = _each_entry_point(W, gk, prec)
    finally:
        fb.tune_set("fail_alloc_after", -1)
    assert all(c == fb.FMGP_ENOMEM for c in codes.values()), codes
    # unhindered again: the same calls succeed
    codes = _each_entry_point(W, gk, prec)
    assert all(c == fb.FMGP_OK for c in codes.values()), codes


def test_context_too_small_refuses_and_leaks_nothing(cuda):
    W = wl.tiny(n=150_000, m=400, k=30, b=300)  # X alone is 2.4 MB
    s = W.kernel
    gk = fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)
    ctx = fb.Context(1)  # the smallest context: 2 MiB
    try:
        with ctx:
            codes = _each_entry_point(W, gk, fb.PREC_MIXED)
        assert codes["build_knn"] == fb.FMGP_ENOMEM and codes["precompute"] == fb.FMGP_ENOMEM
        assert all(c in (fb.FMGP_OK, fb.FMGP_ENOMEM) for c in codes.values()), codes
        torch.cuda.synchronize()
        assert ctx.bytes_in_use() == 0
    finally:
        ctx.close()
    assert all(c == fb.FMGP_OK for c in _each_entry_point(W, gk, fb.PREC_MIXED).values())


def test_partial_allocation_failure_leaks_nothing(cuda):
    """Failures after some allocations succeeded (the k-th of a call's
    allocations refused) release what was taken: the context is empty after."""
    W, gk = _inputs()
    ctx = fb.Context(256 << 20)
    try:
        with ctx:
            for after in (1, 2, 3, 5):
                fb.tune_set("fail_alloc_after", after)
                try:
                    _each_entry_point(W, gk, fb.PREC_MIXED)
                finally:
                    fb.tune_set("fail_alloc_after", -1)
        torch.cuda.synchronize()
        assert ctx.bytes_in_use() == 0
    finally:
        ctx.close()


@pytest.mark.parametrize("where", ["X", "Y", "Z"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_check_finite_refuses_non_finite_inputs(cuda, where, bad):
    W, gk = _inputs()
    X, Y, Z = W.X.copy(), W.Y.copy(), W.Z.copy()
    {"X": X, "Y": Y, "Z": Z}[where][17, 0] = bad
    Xd, Yd, Zd = dev(X), dev(Y), dev(Z)
    nbr, _ = fb.fmgp_build_knn(dev(W.X), 30)
    C, _ = fb.fmgp_precompute(dev(W.X), dev(W.Y), nbr, 30, gk)
    fb.tune_set("check_finite", 1)
    try:
        calls = {"X": [lambda: fb.fmgp_build_knn(Xd, 30),
                       lambda: fb.fmgp_precompute(Xd, Yd, nbr, 30, gk)],
                 "Y": [lambda: fb.fmgp_precompute(Xd, Yd, nbr, 30, gk),
                       lambda: fb.fmgp_loocv_objective(Xd, Yd, nbr, 30, dev(W.batch), gk)],
                 "Z": [lambda: fb.fmgp_predict(Xd, nbr, C, 30, gk, Zd),
                       lambda: fb.fmgp_muygps_predict(Xd, Yd, Zd, 30, gk)]}[where]
        for f in calls:
            with pytest.raises(fb.FmgpError) as e:
                f()
            assert e.value.code == fb.FMGP_EINVAL and where in str(e.value)
        # finite inputs pass the check
        fb.fmgp_predict(dev(W.X), nbr, C, 30, gk, dev(W.Z))
    finally:
        fb.tune_set("check_finite", 0)
