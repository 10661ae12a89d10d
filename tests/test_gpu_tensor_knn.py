"""Tensor-core (tcgen05, BF16) candidate search for kNN at d >= 16: results
must equal the oracle bit-exactly, and most queries must be certified
(i.e. the tensor-core distances were good enough that the exact fallback
scan was not needed), which shows the tensor-core path actually worked."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import dev

pytestmark = pytest.mark.gpu


def _data(kind, n, d, seed):
    rng = np.random.default_rng(seed)
    if kind == "sparse32":
        X = (1.0 - rng.random((n, d), dtype=np.float32))
        X[rng.random((n, d)) < 0.8] = 0.0
        return X
    X = rng.random((n, d))
    X[5] = X[17]  # a duplicate pair
    return X if kind == "u64" else X.astype(np.float32)


@pytest.mark.parametrize("kind,n,d,kq", [("sparse32", 6000, 784, 29), ("u64", 5000, 16, 1),
                                         ("u64", 9000, 64, 31), ("u32", 8000, 64, 63)])
def test_tensor_core_knn_bitexact_and_certified(cuda, kind, n, d, kq):
    X = _data(kind, n, d, n + d)
    c0 = fb.diag_counter(1)
    nbr, dist = fb.fmgp_build_knn(dev(X), kq, with_dist=True)
    torch.cuda.synchronize()
    assert fb.diag_counter(1) == c0 + 1, "tensor-core path not taken"
    fallbacks = fb.diag_counter(2)
    assert 0 <= fallbacks <= 0.2 * n, fallbacks
    rows = np.random.default_rng(1).choice(n, 300, replace=False)
    ref_i, ref_k = oracle.knn(X.astype(np.float64), X.astype(np.float64)[rows], kq, rows)
    np.testing.assert_array_equal(nbr.cpu().numpy()[rows], ref_i)
    np.testing.assert_array_equal(dist.cpu().numpy()[rows], ref_k)
    # the exhaustive scan gives the same table
    fb.tune_set("tensor_cores", 0)
    try:
        nbr2, dist2 = fb.fmgp_build_knn(dev(X), kq, with_dist=True)
    finally:
        fb.tune_set("tensor_cores", 1)
    assert torch.equal(nbr, nbr2) and torch.equal(dist, dist2)


def test_tensor_core_nearest_for_prediction(cuda):
    W = wl.highdim(n=5000, m=700)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, 4)
    C = torch.zeros((W.n, 5, W.r), dtype=torch.float64, device="cuda")
    k = fb.make_kernel("rbf", 0.0, 7.0, 1.0, 1e-2)
    c0 = fb.diag_counter(1)
    _, near = fb.fmgp_predict(X, nbr, C, 5, k, dev(W.Z))
    torch.cuda.synchronize()
    assert fb.diag_counter(1) == c0 + 1
    assert fb.diag_counter(2) <= 0.05 * W.m
    ref, _ = oracle.knn(W.X.astype(np.float64), W.Z.astype(np.float64), 1)
    np.testing.assert_array_equal(near.cpu().numpy(), ref[:, 0])
