"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one: kNN rows
bit-exactly, precomputed rows and predictions within the path's tolerance,
nearest training points exactly, and the LOOCV objective over its whole
batch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import FP64_TOL, MIXED_TOL, coeffs_to_f64, dev, kern_pair, rel_rms

pytestmark = pytest.mark.gpu


def _run(W, prec, kq):
    ok, gk = kern_pair(W.kernel)
    X, Y, Z = dev(W.X), dev(W.Y), dev(W.Z)
    k = W.k
    nbr, dist = fb.fmgp_build_knn(X, kq, with_dist=True)
    C, st = fb.fmgp_precompute(X, Y, nbr, k, gk, prec)
    yh, near = fb.fmgp_predict(X, nbr, C, k, gk, Z, prec)
    Q, res = fb.fmgp_loocv_objective(X, Y, nbr, k, dev(W.batch), gk, prec)
    torch.cuda.synchronize()
    return ok, nbr, dist, C, st, yh, near, Q, res


def _check(W, prec, kq, nsamp, rng):
    ok, nbr, dist, C, st, yh, near, Q, res = _run(W, prec, kq)
    tol = FP64_TOL if prec == fb.PREC_FP64 else MIXED_TOL
    Xd = W.X.astype(np.float64)
    # kNN rows, bit-exact
    rows = np.sort(rng.choice(W.n, nsamp, replace=False))
    ref_i, ref_k = oracle.knn(Xd, Xd[rows], kq, rows)
    nb = nbr.cpu().numpy()
    np.testing.assert_array_equal(nb[rows], ref_i)
    np.testing.assert_array_equal(dist.cpu().numpy()[rows], ref_k)
    s = st.cpu().numpy()
    assert np.all((s == fb.BLOCK_OK) | (s == fb.BLOCK_FP64_RETRY))
    # nearest training point of sampled test points, exact
    tz = np.sort(rng.choice(W.m, nsamp, replace=False))
    ref_near, _ = oracle.knn(Xd, W.Z[tz].astype(np.float64), 1)
    nr = near.cpu().numpy()
    np.testing.assert_array_equal(nr[tz], ref_near[:, 0])
    # predictions of the sampled test points: the oracle's own rows of C
    jr = np.unique(nr[tz])
    Cr, _ = oracle.precompute(Xd, W.Y, nb, W.k, ok, rows=jr)
    Cfull = np.zeros((W.n, W.k, W.r))
    Cfull[jr] = Cr
    yr = oracle.predict_given(Xd, nb, Cfull, ok, W.Z[tz].astype(np.float64), nr[tz])
    assert rel_rms(yh.cpu().numpy()[tz], yr) < tol
    # LOOCV over the whole batch
    Qr, resr = oracle.loocv(Xd, W.Y, nb, W.k, W.batch, ok)
    assert abs(Q - Qr) / abs(Qr) < tol
    assert rel_rms(res.cpu().numpy(), resr) < tol


@pytest.mark.parametrize("prec", [fb.PREC_MIXED, fb.PREC_FP64])
def test_spatial_full_size(cuda, prec):
    """n = 150,000 training and m = 50,000 test points, k = 50 (the bench step)."""
    _check(wl.spatial(), prec, 50, 300, np.random.default_rng(21))


def test_large_full_size(cuda):
    """n = 10,000,000 training and m = 1,000,000 test points in 3-D, k = 64,
    Matern 5/2 with nugget 1e-5 (ill-conditioned blocks), mixed precision."""
    _check(wl.large(), fb.PREC_MIXED, 64, 150, np.random.default_rng(22))
