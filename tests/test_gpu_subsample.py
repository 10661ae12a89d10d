"""Subsampled precompute (Sec. 5): coefficients for a set of centre rows only,
prediction from the nearest centre.  Centres chosen bit-exactly like the
oracle's; coefficients and means within the path's tolerance; with every row
as a centre the results are those of fmgp_precompute / fmgp_predict."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import FP64_TOL, MIXED_TOL, coeffs_to_f64, dev, kern_pair, rel_rms

pytestmark = pytest.mark.gpu


def _workload(name):
    if name == "tiny":
        return wl.tiny(m=400)
    if name == "borehole":
        return wl.borehole(n=5000, m=300, k=40, nugget=1e-4)
    rng = np.random.default_rng(16)
    X = rng.random((3000, 16))
    Z = rng.random((300, 16))
    return wl.Workload("d16", X, np.sin(3 * X.sum(1, keepdims=True)), Z, Z[:, :1], 20,
                       wl.KernelSpec("rbf", 0.0, 0.5, 1.0, 1e-3), np.arange(5))


@pytest.mark.parametrize("prec", [fb.PREC_FP64, fb.PREC_MIXED])
@pytest.mark.parametrize("name", ["tiny", "borehole", "d16"])
def test_subsample_matches_oracle(cuda, name, prec):
    W = _workload(name)
    ok, gk = kern_pair(W.kernel)
    rows = np.sort(np.random.default_rng(8).choice(W.n, W.n // 3, replace=False)).astype(np.int32)
    X, Y = dev(W.X), dev(W.Y)
    nbr, _ = fb.fmgp_build_knn(X, W.k - 1)
    C, st = fb.fmgp_precompute_rows(X, Y, nbr, W.k, gk, dev(rows), prec)
    yh, cen = fb.fmgp_predict_rows(X, nbr, dev(rows), C, W.k, gk, dev(W.Z), prec)
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert np.all((s == fb.BLOCK_OK) | (s == fb.BLOCK_FP64_RETRY))
    onbr, _ = oracle.self_knn(W.X, W.k - 1)
    np.testing.assert_array_equal(nbr.cpu().numpy(), onbr)
    Cr, _ = oracle.precompute(W.X, W.Y, onbr, W.k, ok, rows=rows)
    yr, cr = oracle.predict_rows(W.X, onbr, rows, Cr, ok, W.Z)
    np.testing.assert_array_equal(cen.cpu().numpy(), cr)
    tol = FP64_TOL if prec == fb.PREC_FP64 else MIXED_TOL
    assert rel_rms(coeffs_to_f64(C, prec), Cr) < (tol if prec == fb.PREC_FP64 else 1e-4)
    assert rel_rms(yh.cpu().numpy(), yr) < tol


@pytest.mark.parametrize("prec", [fb.PREC_FP64, fb.PREC_MIXED])
def test_every_row_as_centre_is_the_full_method(cuda, prec):
    W = wl.spatial(n=8000, m=500, nu=1.5)
    _, gk = kern_pair(W.kernel)
    X, Y, Z = dev(W.X), dev(W.Y), dev(W.Z)
    nbr, _ = fb.fmgp_build_knn(X, W.k - 1)
    rows = torch.arange(W.n, dtype=torch.int32, device="cuda")
    C, _ = fb.fmgp_precompute(X, Y, nbr, W.k, gk, prec)
    Cs, _ = fb.fmgp_precompute_rows(X, Y, nbr, W.k, gk, rows, prec)
    assert torch.equal(C, Cs)
    yf, nf = fb.fmgp_predict(X, nbr, C, W.k, gk, Z, prec)
    ys, ns = fb.fmgp_predict_rows(X, nbr, rows, Cs, W.k, gk, Z, prec)
    assert torch.equal(nf, ns)
    assert torch.equal(yf, ys)


def test_subsample_edge_cases(cuda):
    W = wl.tiny(n=600, m=50)
    ok, gk = kern_pair(W.kernel)
    X, Y, Z = dev(W.X), dev(W.Y), dev(W.Z)
    nbr, _ = fb.fmgp_build_knn(X, W.k - 1)
    # a repeated centre: the first position is chosen, results as with one copy
    rows = np.array([5, 17, 17, 300, 599], np.int32)
    C, st = fb.fmgp_precompute_rows(X, Y, nbr, W.k, gk, dev(rows), fb.PREC_FP64)
    assert (st.cpu().numpy() == fb.BLOCK_OK).all()
    yh, cen = fb.fmgp_predict_rows(X, nbr, dev(rows), C, W.k, gk, Z, fb.PREC_FP64)
    onbr, _ = oracle.self_knn(W.X, W.k - 1)
    Cr, _ = oracle.precompute(W.X, W.Y, onbr, W.k, ok, rows=rows)
    yr, cr = oracle.predict_rows(W.X, onbr, rows, Cr, ok, W.Z)
    np.testing.assert_array_equal(cen.cpu().numpy(), cr)
    assert rel_rms(yh.cpu().numpy(), yr) < FP64_TOL
    # an index outside [0, n): a zero row flagged BAD_INDEX when precomputing,
    # refused before anything runs when predicting
    bad = dev(np.array([3, 600, 7], np.int32))
    C2, st2 = fb.fmgp_precompute_rows(X, Y, nbr, W.k, gk, bad, fb.PREC_FP64)
    assert st2.cpu().numpy().tolist() == [fb.BLOCK_OK, fb.BLOCK_BAD_INDEX, fb.BLOCK_OK]
    assert torch.count_nonzero(C2[1]).item() == 0
    out = torch.full((W.m, 1), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(fb.FmgpError) as ei:
        fb.fmgp_predict_rows(X, nbr, bad, C2, W.k, gk, Z, fb.PREC_FP64, Yhat_out=out)
    assert ei.value.code == fb.FMGP_EINVAL
    assert torch.all(out == 7.0)
    # no centres: precompute is a no-op, prediction is refused
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    C0, _ = fb.fmgp_precompute_rows(X, Y, nbr, W.k, gk, empty, fb.PREC_FP64)
    assert C0.shape[0] == 0
    with pytest.raises(fb.FmgpError):
        fb.fmgp_predict_rows(X, nbr, empty, C0, W.k, gk, Z, fb.PREC_FP64)
