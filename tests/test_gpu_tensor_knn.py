"""Tensor-core (tcgen05, BF16) candidate search for kNN at d >= 16: results
must equal the oracle bit-exactly, and most queries must be certified
(i.e. the tensor-core distances were good enough that the exact fallback
scan was not needed), which shows the tensor-core path actually worked.
Both forms of the candidate selection are covered: inside the distance
kernel (kq <= 32) and through the pass buffer."""
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


class _Fused:
    """Select the candidate-selection form for the block's duration."""

    def __init__(self, on):
        self.on = on

    def __enter__(self):
        self.prev = fb.tune_get("tc_fused_select")
        fb.tune_set("tc_fused_select", self.on)

    def __exit__(self, *exc):
        fb.tune_set("tc_fused_select", self.prev)


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("kind,n,d,kq", [("sparse32", 6000, 784, 29), ("u64", 5000, 16, 1),
                                         ("u64", 9000, 64, 31), ("u32", 8000, 64, 63),
                                         ("u32", 4099, 16, 4), ("u64", 4500, 40, 5),
                                         ("u32", 7001, 24, 32), ("u64", 6100, 32, 16)])
def test_tensor_core_knn_bitexact_and_certified(cuda, kind, n, d, kq, fused):
    X = _data(kind, n, d, n + d)
    c0 = fb.diag_counter(1)
    with _Fused(fused):
        nbr, dist = fb.fmgp_build_knn(dev(X), kq, with_dist=True)
        nbr_i, _ = fb.fmgp_build_knn(dev(X), kq)
    torch.cuda.synchronize()
    assert torch.equal(nbr, nbr_i)
    assert fb.diag_counter(1) == c0 + 2, "tensor-core path not taken"
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


@pytest.mark.parametrize("n,d,m", [(4096, 16, 128), (20_011, 64, 129), (30_000, 24, 5_000),
                                   (9_000, 130, 700)])
def test_tensor_core_nearest_both_forms(cuda, n, d, m):
    """Nearest training point of m queries (one query block with many
    candidate ranges up to many blocks with a ragged last one): both forms
    of the selection equal the oracle's exact answer."""
    rng = np.random.default_rng(n + m)
    X = rng.random((n, d))
    Z = rng.random((m, d))
    Z[: m // 8] = X[rng.choice(n, m // 8, replace=False)]  # queries on training points
    kern = fb.make_kernel("rbf", 0.0, 1.0, 1.0, 1e-2)
    C = torch.zeros((n, 2, 1), dtype=torch.float64, device="cuda")
    nbr = torch.zeros((n, 1), dtype=torch.int32, device="cuda")
    ref, _ = oracle.knn(X, Z, 1)
    for fused in (1, 0):
        with _Fused(fused):
            c0 = fb.diag_counter(1)
            _, near = fb.fmgp_predict(dev(X), nbr, C, 2, kern, dev(Z))
            torch.cuda.synchronize()
            assert fb.diag_counter(1) == c0 + 1
            assert fb.diag_counter(2) <= 0.05 * m
        np.testing.assert_array_equal(near.cpu().numpy(), ref[:, 0])


def test_oversampling_changes_no_result(cuda):
    """The re-rank's candidate count is a speed setting: the certificate
    (or the exhaustive fallback) makes every setting give the same table."""
    X = _data("sparse32", 6000, 784, 11)
    tables = []
    prev = fb.tune_get("tc_oversample")
    try:
        for ovs in (2, 3, 4):
            fb.tune_set("tc_oversample", ovs)
            nbr, _ = fb.fmgp_build_knn(dev(X), 29)
            tables.append(nbr)
    finally:
        fb.tune_set("tc_oversample", prev)
    assert all(torch.equal(tables[0], t) for t in tables[1:])
    rows = np.arange(0, 6000, 97)
    ref_i, _ = oracle.knn(X.astype(np.float64), X.astype(np.float64)[rows], 29, rows)
    np.testing.assert_array_equal(tables[0].cpu().numpy()[rows], ref_i)


@pytest.mark.parametrize("r", [8, 16, 32])
def test_fused_list_length_changes_no_result(cuda, r):
    """The per-range list length of the fused selection is a speed setting:
    every length gives the oracle's table (uncertified queries, if any, go
    through the exact scan)."""
    X = _data("u32", 5000, 48, 7)
    prev = fb.tune_get("tc_fused_r")
    try:
        fb.tune_set("tc_fused_r", r)
        nbr, dist = fb.fmgp_build_knn(dev(X), 12, with_dist=True)
    finally:
        fb.tune_set("tc_fused_r", prev)
    rows = np.arange(0, 5000, 41)
    ref_i, ref_k = oracle.knn(X.astype(np.float64), X.astype(np.float64)[rows], 12, rows)
    np.testing.assert_array_equal(nbr.cpu().numpy()[rows], ref_i)
    np.testing.assert_array_equal(dist.cpu().numpy()[rows], ref_k)


@pytest.mark.parametrize("kind,n,d,kq,r", [("sparse32", 6000, 784, 29, 8), ("u64", 6000, 40, 20, 8)])
def test_exact_fallback_of_uncertified_queries(cuda, kind, n, d, kq, r):
    """Per-range lists too short for kq leave many queries without a
    certificate; the exhaustive scan over the device-side list (the first
    positions split over candidate ranges and merged, the rest scanned whole)
    must still give the oracle's table."""
    X = _data(kind, n, d, 5)
    prev = fb.tune_get("tc_fused_r")
    try:
        fb.tune_set("tc_fused_r", r)
        nbr, dist = fb.fmgp_build_knn(dev(X), kq, with_dist=True)
        torch.cuda.synchronize()
        redone = fb.diag_counter(2)
    finally:
        fb.tune_set("tc_fused_r", prev)
    assert redone > 64, redone  # both the split and the whole-scan positions ran
    rows = np.arange(0, n, 37)
    ref_i, ref_k = oracle.knn(X.astype(np.float64), X.astype(np.float64)[rows], kq, rows)
    np.testing.assert_array_equal(nbr.cpu().numpy()[rows], ref_i)
    np.testing.assert_array_equal(dist.cpu().numpy()[rows], ref_k)
    ref_all, _ = fb.fmgp_build_knn(dev(X), kq)
    assert torch.equal(nbr, ref_all)


@pytest.mark.parametrize("fused", [1, 0])
def test_bf16_useless_data_still_exact(cuda, fused):
    """Coordinates near 1000 with spread 10: BF16 (spacing 4 there) cannot
    separate the points, so the certificate fails for nearly every query and
    the exact scan answers them; the table must still be the oracle's."""
    rng = np.random.default_rng(21)
    X = 1000.0 + 10.0 * rng.random((5000, 24))
    with _Fused(fused):
        nbr, dist = fb.fmgp_build_knn(dev(X), 6, with_dist=True)
        torch.cuda.synchronize()
        redone = fb.diag_counter(2)
    assert redone > 100, redone
    rows = np.arange(0, 5000, 23)
    ref_i, ref_k = oracle.knn(X, X[rows], 6, rows)
    np.testing.assert_array_equal(nbr.cpu().numpy()[rows], ref_i)
    np.testing.assert_array_equal(dist.cpu().numpy()[rows], ref_k)


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("kind,n,d,kq", [("u64", 9000, 16, 127), ("u32", 9000, 16, 159),
                                         ("u32", 8500, 64, 127), ("u64", 8003, 64, 159),
                                         ("u32", 6000, 40, 97)])
def test_tensor_core_knn_large_kq(cuda, kind, n, d, kq, fused):
    """Neighbour counts above 96 (the k - 1 = 127 table of a k = 128 model, and
    the largest, 159): fused selection with 32-entry lists over at least
    kq / 8 candidate ranges, or the pass buffer; re-rank lists of 2 kq.  The
    table equals the oracle's bit for bit and most queries are certified."""
    X = _data(kind, n, d, n + d + kq)
    c0 = fb.diag_counter(1)
    with _Fused(fused):
        nbr, dist = fb.fmgp_build_knn(dev(X), kq, with_dist=True)
        torch.cuda.synchronize()
        fallbacks = fb.diag_counter(2)
    assert fb.diag_counter(1) == c0 + 1, "tensor-core path not taken"
    assert 0 <= fallbacks <= 0.2 * n, fallbacks
    rows = np.random.default_rng(2).choice(n, 200, replace=False)
    ref_i, ref_k = oracle.knn(X.astype(np.float64), X.astype(np.float64)[rows], kq, rows)
    np.testing.assert_array_equal(nbr.cpu().numpy()[rows], ref_i)
    np.testing.assert_array_equal(dist.cpu().numpy()[rows], ref_k)
    fb.tune_set("tensor_cores", 0)
    try:
        nbr2, dist2 = fb.fmgp_build_knn(dev(X), kq, with_dist=True)
    finally:
        fb.tune_set("tensor_cores", 1)
    assert torch.equal(nbr, nbr2) and torch.equal(dist, dist2)


@pytest.mark.parametrize("kq", [31, 127])
def test_fused_selection_in_query_chunks(cuda, kq):
    """The fused selection processed in passes over blocks of queries (here
    3 blocks of 128 per pass, the last pass ragged) gives the same table as
    one pass, for self kNN and for external queries."""
    rng = np.random.default_rng(kq)
    n, m, d = 7000, 1000, 32
    X = rng.random((n, d))
    Z = rng.random((m, d))
    prev = fb.tune_get("tc_chunk_queries")
    try:
        fb.tune_set("tc_chunk_queries", 0)
        one, _ = fb.fmgp_build_knn(dev(X), kq)
        fb.tune_set("tc_chunk_queries", 384)
        c0 = fb.diag_counter(1)
        chunked, _ = fb.fmgp_build_knn(dev(X), kq)
        torch.cuda.synchronize()
        assert fb.diag_counter(1) == c0 + 1
    finally:
        fb.tune_set("tc_chunk_queries", prev)
    assert torch.equal(one, chunked)
    rows = np.arange(0, n, 53)
    ref_i, _ = oracle.knn(X, X[rows], kq, rows)
    np.testing.assert_array_equal(chunked.cpu().numpy()[rows], ref_i)
    # plain MuyGPs neighbours of external queries: the same search with self = false
    Y = dev(np.sin(X[:, :1] * 3.0))
    kern = fb.make_kernel("rbf", 0.0, 1.5, 1.0, 1e-2)
    k = kq + 1 if kq < 160 else kq
    try:
        fb.tune_set("tc_chunk_queries", 384)
        _, nb_q = fb.fmgp_muygps_predict(dev(X), Y, dev(Z), k, kern, fb.PREC_FP64, with_nbr=True)
    finally:
        fb.tune_set("tc_chunk_queries", prev)
    ref_q, _ = oracle.knn(X, Z, k)
    np.testing.assert_array_equal(nb_q.cpu().numpy(), ref_q)


@pytest.mark.parametrize("fused", [1, 0])
def test_distance_pass_that_gives_up_falls_back_to_the_exact_scan(cuda, fused):
    """With the main-loop wait limit of the tcgen05 distance kernel cut to 1 ns
    its waits run out: the kernel stops, drains its own copies and matrix
    operations (those waits keep their 2 s limit), frees its tensor memory and
    reports the abort, so no query is certified and every one is answered by
    the exhaustive exact scan.  The table is still the oracle's, and a later
    call with the normal limit runs normally."""
    X = _data("u32", 6000, 64, 12)
    ref, ref_d = fb.fmgp_build_knn(dev(X), 20, with_dist=True)
    torch.cuda.synchronize()
    prev = fb.tune_get("tc_wait_ns")
    try:
        fb.tune_set("tc_wait_ns", 1)
        with _Fused(fused):
            nbr, dist = fb.fmgp_build_knn(dev(X), 20, with_dist=True)
            torch.cuda.synchronize()
            redone = fb.diag_counter(2)
    finally:
        fb.tune_set("tc_wait_ns", prev)
    assert redone == 6000, redone  # the aborted pass certified nothing
    assert torch.equal(nbr, ref) and torch.equal(dist, ref_d)
    rows = np.arange(0, 6000, 61)
    ref_i, _ = oracle.knn(X.astype(np.float64), X.astype(np.float64)[rows], 20, rows)
    np.testing.assert_array_equal(nbr.cpu().numpy()[rows], ref_i)
    again, _ = fb.fmgp_build_knn(dev(X), 20)
    torch.cuda.synchronize()
    assert fb.diag_counter(2) < 600 and torch.equal(again, ref)
