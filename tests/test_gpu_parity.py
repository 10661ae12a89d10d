"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  kNN indices and keys bit-exact; FP64 means within
rel-RMS 1e-10; mixed means within rel-RMS 1e-5."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import FP64_TOL, MIXED_TOL, coeffs_to_f64, dev, kern_pair, rel_rms

pytestmark = pytest.mark.gpu


def _gpu_pipeline(W, k, kq, precision, gk):
    X = dev(W.X)
    Y = dev(W.Y)
    Z = dev(W.Z)
    nbr, dist = fb.fmgp_build_knn(X, kq, with_dist=True)
    C, st = fb.fmgp_precompute(X, Y, nbr, k, gk, precision)
    yh, near = fb.fmgp_predict(X, nbr, C, k, gk, Z, precision)
    torch.cuda.synchronize()
    return nbr, dist, C, st, yh, near


# ------------------------------------------------------------------ kNN --
@pytest.mark.parametrize("d", [1, 2, 3])
def test_knn_integer_grid_ties_bitexact(cuda, d):
    rng = np.random.default_rng(100 + d)
    n = 3000
    X = rng.integers(0, 12 if d > 1 else 400, size=(n, d)).astype(np.float64)
    for kq in [1, 9, 33, 70]:
        nbr, dist = fb.fmgp_build_knn(dev(X), kq, with_dist=True)
        ref_i, ref_k = oracle.self_knn(X, kq)
        np.testing.assert_array_equal(nbr.cpu().numpy(), ref_i)
        np.testing.assert_array_equal(dist.cpu().numpy(), ref_k)


def test_knn_tiny_bitexact(cuda):
    W = wl.tiny()
    nbr, dist = fb.fmgp_build_knn(dev(W.X), 30, with_dist=True)
    ref_i, ref_k = oracle.self_knn(W.X, 30)
    np.testing.assert_array_equal(nbr.cpu().numpy(), ref_i)
    np.testing.assert_array_equal(dist.cpu().numpy(), ref_k)


@pytest.mark.parametrize("kq", [1, 49, 127, 150, 160])
def test_knn_spatial_sample_bitexact(cuda, kq):
    W = wl.spatial(n=40_000, m=10)
    nbr, dist = fb.fmgp_build_knn(dev(W.X), kq, with_dist=True)
    rows = np.random.default_rng(0).choice(W.n, 300, replace=False)
    ref_i, ref_k = oracle.knn(W.X, W.X[rows], kq, rows)
    np.testing.assert_array_equal(nbr.cpu().numpy()[rows], ref_i)
    np.testing.assert_array_equal(dist.cpu().numpy()[rows], ref_k)


@pytest.mark.parametrize("d,dtype", [(4, np.float64), (16, np.float32), (64, np.float64),
                                     (784, np.float32)])
def test_knn_bruteforce_bitexact(cuda, d, dtype):
    rng = np.random.default_rng(200 + d)
    n = 700
    X = rng.random((n, d)).astype(dtype)
    X[rng.random((n, d)) < 0.8] = 0
    X[10] = X[20]  # exact duplicate
    for kq in [1, 29, 150]:
        nbr, dist = fb.fmgp_build_knn(dev(X), kq, with_dist=True)
        ref_i, ref_k = oracle.self_knn(X.astype(np.float64), kq)
        np.testing.assert_array_equal(nbr.cpu().numpy(), ref_i)
        np.testing.assert_array_equal(dist.cpu().numpy(), ref_k)


@pytest.mark.parametrize("d,dtype", [(4, np.float64), (8, np.float64), (8, np.float32),
                                     (15, np.float64)])
def test_nearest_scan_bitexact(cuda, d, dtype):
    """The thread-per-query nearest-point scan (4 <= d <= 15): integer grid
    coordinates make many exact ties, which must go to the lowest index
    across the scan's slices; half the rows get a small jitter."""
    rng = np.random.default_rng(300 + d)
    n, m = 9000, 700
    X = rng.integers(0, 4, (n, d)).astype(dtype)
    X[: n // 2] += (rng.random((n // 2, d)) * 0.01).astype(dtype)
    Z = rng.integers(0, 4, (m, d)).astype(dtype)
    Z[::3] += (rng.random((len(Z[::3]), d)) * 0.02).astype(dtype)
    Y = rng.normal(size=(n, 1))
    gk = fb.make_kernel("matern", 1.5, 1.0, 1.0, 1e-2)
    nbr, _ = fb.fmgp_build_knn(dev(X), 4)
    C, _ = fb.fmgp_precompute(dev(X), dev(Y), nbr, 5, gk, fb.PREC_FP64)
    _, near = fb.fmgp_predict(dev(X), nbr, C, 5, gk, dev(Z), fb.PREC_FP64)
    ref, _ = oracle.knn(X.astype(np.float64), Z.astype(np.float64), 1)
    np.testing.assert_array_equal(near.cpu().numpy(), ref[:, 0])


def test_nearest_scan_fp64_near_ties_bitexact(cuda):
    """FP64 points that differ by ~1e-10 collapse onto the same FP32 values:
    the scan's FP32 threshold must let all of them through to the exact key."""
    rng = np.random.default_rng(321)
    n, m, d = 6000, 500, 8
    centres = rng.integers(0, 3, (n // 6, d)).astype(np.float64)
    X = np.repeat(centres, 6, axis=0) + rng.random((n, d)) * 1e-10
    Z = centres[rng.integers(0, len(centres), m)] + rng.random((m, d)) * 1e-10
    Y = rng.normal(size=(n, 1))
    gk = fb.make_kernel("matern", 1.5, 1.0, 1.0, 1e-2)
    nbr, _ = fb.fmgp_build_knn(dev(X), 4)
    C, _ = fb.fmgp_precompute(dev(X), dev(Y), nbr, 5, gk, fb.PREC_FP64)
    _, near = fb.fmgp_predict(dev(X), nbr, C, 5, gk, dev(Z), fb.PREC_FP64)
    ref, _ = oracle.knn(X, Z, 1)
    np.testing.assert_array_equal(near.cpu().numpy(), ref[:, 0])


def test_nearest_test_point_bitexact(cuda):
    W = wl.spatial(n=30_000, m=5_000)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, 4)
    C = torch.zeros((W.n, 5, 1), dtype=torch.float64, device="cuda")
    _, gk = kern_pair(W.kernel)
    # test points outside the training box and exactly on training points too
    Z = np.concatenate([W.Z, W.X[:50], W.Z[:20] * 1.5 - 0.25])
    _, near = fb.fmgp_predict(X, nbr, C, 5, gk, dev(Z))
    ref, _ = oracle.knn(W.X, Z, 1)
    np.testing.assert_array_equal(near.cpu().numpy(), ref[:, 0])


# ------------------------------------------------------- precompute/predict --
def test_fp64_pipeline_tiny(cuda):
    W = wl.tiny()
    ok, gk = kern_pair(W.kernel)
    nbr, dist, C, st, yh, near = _gpu_pipeline(W, 30, 29, fb.PREC_FP64, gk)
    ref_nbr, _ = oracle.self_knn(W.X, 29)
    np.testing.assert_array_equal(nbr.cpu().numpy(), ref_nbr)
    Cr, str_ = oracle.precompute(W.X, W.Y, ref_nbr, 30, ok)
    assert not st.cpu().numpy().any() and not str_.any()
    assert rel_rms(C.cpu().numpy(), Cr) < FP64_TOL
    yr, nr = oracle.predict(W.X, ref_nbr, Cr, ok, W.Z)
    np.testing.assert_array_equal(near.cpu().numpy(), nr)
    assert rel_rms(yh.cpu().numpy(), yr) < FP64_TOL


@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_fp64_pipeline_spatial_shrunk(cuda, nu):
    W = wl.spatial(n=20_000, m=3_000, nu=nu)
    ok, gk = kern_pair(W.kernel)
    nbr, dist, C, st, yh, near = _gpu_pipeline(W, 50, 49, fb.PREC_FP64, gk)
    nb, _ = oracle.self_knn(W.X, 49)  # the oracle's own table
    np.testing.assert_array_equal(nbr.cpu().numpy(), nb)
    rows = np.random.default_rng(1).choice(W.n, 400, replace=False)
    Cr, _ = oracle.precompute(W.X, W.Y, nb, 50, ok, rows=rows)
    assert rel_rms(C.cpu().numpy()[rows], Cr) < FP64_TOL
    Cfull, _ = oracle.precompute(W.X, W.Y, nb, 50, ok)
    yr, nr = oracle.predict(W.X, nb, Cfull, ok, W.Z)
    np.testing.assert_array_equal(near.cpu().numpy(), nr)
    assert rel_rms(yh.cpu().numpy(), yr) < FP64_TOL


def test_fp64_multi_response_highdim_small(cuda):
    W = wl.highdim(n=1500, m=300, d=784, r=10, k=30)
    ok, gk = kern_pair(W.kernel)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, 29)
    nb, _ = oracle.self_knn(W.X.astype(np.float64), 29)  # the oracle's own table
    np.testing.assert_array_equal(nbr.cpu().numpy(), nb)
    C, st = fb.fmgp_precompute(X, dev(W.Y), nbr, 30, gk, fb.PREC_FP64)
    Cr, _ = oracle.precompute(W.X, W.Y, nb, 30, ok)
    assert rel_rms(C.cpu().numpy(), Cr) < FP64_TOL
    yh, near = fb.fmgp_predict(X, nbr, C, 30, gk, dev(W.Z), fb.PREC_FP64)
    yr, nr = oracle.predict(W.X, nb, Cr, ok, W.Z)
    np.testing.assert_array_equal(near.cpu().numpy(), nr)
    assert rel_rms(yh.cpu().numpy(), yr) < FP64_TOL


@pytest.mark.parametrize("k", [1, 2, 33, 64, 128, 129, 150])
def test_fp64_precompute_k_range(cuda, k):
    W = wl.spatial(n=3_000, m=200, nu=1.5)
    ok, gk = kern_pair(W.kernel)
    kq = max(k - 1, 1)
    nbr, _ = fb.fmgp_build_knn(dev(W.X), kq)
    nb, _ = oracle.self_knn(W.X, kq)  # the oracle's own table
    np.testing.assert_array_equal(nbr.cpu().numpy(), nb)
    C, st = fb.fmgp_precompute(dev(W.X), dev(W.Y), nbr, k, gk, fb.PREC_FP64)
    Cr, _ = oracle.precompute(W.X, W.Y, nb, k, ok)
    assert rel_rms(C.cpu().numpy(), Cr) < FP64_TOL
    yh, _ = fb.fmgp_predict(dev(W.X), nbr, C, k, gk, dev(W.Z), fb.PREC_FP64)
    yr, _ = oracle.predict(W.X, nb, Cr, ok, W.Z)
    assert rel_rms(yh.cpu().numpy(), yr) < FP64_TOL


@pytest.mark.parametrize("precision", [fb.PREC_FP64, fb.PREC_MIXED])
def test_k_beyond_shared_memory_is_refused(cuda, precision):
    """k = 160 needs more than 200 KB of shared memory per warp for the FP64
    factor (the mixed form keeps it for its fallback): the call fails with
    FMGP_EUNSUPPORTED instead of launching."""
    W = wl.spatial(n=2_000, m=10, nu=1.5)
    _, gk = kern_pair(W.kernel)
    nbr, _ = fb.fmgp_build_knn(dev(W.X), 159)
    with pytest.raises(fb.FmgpError) as ei:
        fb.fmgp_precompute(dev(W.X), dev(W.Y), nbr, 160, gk, precision)
    assert ei.value.code == fb.FMGP_EUNSUPPORTED


def test_k_equals_n_small(cuda):
    rng = np.random.default_rng(7)
    X = rng.random((40, 2))
    Y = rng.normal(size=(40, 2))
    Z = rng.random((13, 2))
    ok, gk = oracle.kernel("matern", 2.5, 0.3, 1.0, 1e-3), fb.make_kernel("matern", 2.5, 0.3, 1.0, 1e-3)
    nbr, _ = fb.fmgp_build_knn(dev(X), 39)
    C, _ = fb.fmgp_precompute(dev(X), dev(Y), nbr, 40, gk, fb.PREC_FP64)
    yh, _ = fb.fmgp_predict(dev(X), nbr, C, 40, gk, dev(Z), fb.PREC_FP64)
    nb, _ = oracle.self_knn(X, 39)
    Cr, _ = oracle.precompute(X, Y, nb, 40, ok)
    yr, _ = oracle.predict(X, nb, Cr, ok, Z)
    assert rel_rms(yh.cpu().numpy(), yr) < FP64_TOL


def test_predict_m_zero_is_noop(cuda):
    W = wl.tiny(n=200, m=1)
    _, gk = kern_pair(W.kernel)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, 9)
    C, _ = fb.fmgp_precompute(X, dev(W.Y), nbr, 10, gk)
    yh, near = fb.fmgp_predict(X, nbr, C, 10, gk, torch.zeros((0, 2), dtype=torch.float64,
                                                              device="cuda"))
    assert yh.shape == (0, 1)


def test_not_spd_status_and_bad_index(cuda):
    X = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 1.0], [2.0, 0.5], [3.0, 3.0]])
    Y = np.ones((5, 1))
    gk = fb.make_kernel("matern", 1.5, 1.0, 1.0, 0.0)
    nbr, _ = fb.fmgp_build_knn(dev(X), 2)
    C, st = fb.fmgp_precompute(dev(X), dev(Y), nbr, 3, gk)
    s = st.cpu().numpy()
    assert s[0] == fb.BLOCK_NOT_SPD and s[1] == fb.BLOCK_NOT_SPD
    assert np.all(C.cpu().numpy()[0] == 0)
    with pytest.raises(fb.FmgpError) as e:
        fb.fmgp_precompute(dev(X), dev(Y), nbr, 3, gk, with_status=False)
    assert e.value.code == fb.FMGP_ENOTSPD
    bad = nbr.clone()
    bad[3, 0] = 99
    _, st2 = fb.fmgp_precompute(dev(X), dev(Y), bad, 3, fb.make_kernel("matern", 1.5, 1.0, 1.0, 1e-3))
    assert st2.cpu().numpy()[3] == fb.BLOCK_BAD_INDEX


# --------------------------------------------------------------- LOOCV --
@pytest.mark.parametrize("precision", [fb.PREC_FP64])
def test_loocv_tiny(cuda, precision):
    W = wl.tiny()
    ok, gk = kern_pair(W.kernel)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, 30)
    Q, res = fb.fmgp_loocv_objective(X, dev(W.Y), nbr, 30, dev(W.batch), gk, precision)
    nb, _ = oracle.self_knn(W.X, 30)
    Qr, resr = oracle.loocv(W.X, W.Y, nb, 30, W.batch, ok)
    tol = FP64_TOL if precision == fb.PREC_FP64 else MIXED_TOL
    assert abs(Q - Qr) / abs(Qr) < tol
    assert rel_rms(res.cpu().numpy(), resr) < tol


@pytest.mark.parametrize("precision", [fb.PREC_FP64, fb.PREC_MIXED])
def test_loocv_large_k(cuda, precision):
    """k = 140: the FP64 blocks take one CTA each (and so does the mixed
    path's FP64 fallback)."""
    W = wl.spatial(n=4000, m=10, nu=1.5, b=300)
    ok, gk = kern_pair(W.kernel)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, 140)
    Q, res = fb.fmgp_loocv_objective(X, dev(W.Y), nbr, 140, dev(W.batch), gk, precision)
    nb, _ = oracle.self_knn(W.X, 140)
    Qr, resr = oracle.loocv(W.X, W.Y, nb, 140, W.batch, ok)
    tol = FP64_TOL if precision == fb.PREC_FP64 else MIXED_TOL
    assert abs(Q - Qr) / abs(Qr) < tol
    assert rel_rms(res.cpu().numpy(), resr) < tol


# ------------------------------------------------------------ mixed path --
def _mixed_check(W, k, kq, n_rows=None, tol=MIXED_TOL):
    ok, gk = kern_pair(W.kernel)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, kq)
    C, st = fb.fmgp_precompute(X, dev(W.Y), nbr, k, gk, fb.PREC_MIXED)
    yh, near = fb.fmgp_predict(X, nbr, C, k, gk, dev(W.Z), fb.PREC_MIXED)
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert np.all((s == fb.BLOCK_OK) | (s == fb.BLOCK_FP64_RETRY))
    # the oracle's own nearest points and neighbour rows (for the rows needed)
    onear, _ = oracle.knn(W.X, W.Z, 1)
    onear = onear[:, 0]
    np.testing.assert_array_equal(near.cpu().numpy(), onear)
    rows = np.unique(onear).astype(np.int64)
    nb_rows, _ = oracle.knn(W.X, W.X[rows], kq, rows)
    np.testing.assert_array_equal(nbr.cpu().numpy()[rows], nb_rows)
    nb = np.zeros((W.n, kq), np.int32)
    nb[rows] = nb_rows
    Cr, _ = oracle.precompute(W.X, W.Y, nb, k, ok, rows=rows)
    Cfull = np.zeros((W.n, k, W.r))
    Cfull[rows] = Cr
    yr = oracle.predict_given(W.X, nb, Cfull, ok, W.Z, onear)
    err = rel_rms(yh.cpu().numpy(), yr)
    assert err < tol, err
    cerr = rel_rms(coeffs_to_f64(C, fb.PREC_MIXED)[rows], Cr)
    return err, cerr, s


def test_mixed_pipeline_tiny(cuda):
    W = wl.tiny()
    err, cerr, s = _mixed_check(W, 30, 29)
    assert cerr < 1e-6


@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_mixed_spatial(cuda, nu):
    W = wl.spatial(n=60_000, m=4_000, nu=nu)
    err, cerr, s = _mixed_check(W, 50, 50)
    assert (s == fb.BLOCK_FP64_RETRY).mean() < 0.01


def test_mixed_ill_conditioned_large_like(cuda):
    """Matern 5/2 with tau^2 = 1e-5 on dense 3-D points: refinement takes
    several steps and some blocks may go to the FP64 fallback."""
    W = wl.large(n=1_000_000, m=3_000)
    _mixed_check(W, 64, 63)


@pytest.mark.parametrize("k", [129, 150])
def test_mixed_k_beyond_128(cuda, k):
    W = wl.spatial(n=6_000, m=500, nu=1.5)
    _mixed_check(W, k, k - 1)


def test_mixed_highdim_multiresponse(cuda):
    W = wl.highdim(n=2_000, m=300)
    _mixed_check(W, 30, 29)


def test_mixed_fp64_fallback_on_fp32_failure(cuda):
    """Near-duplicate clusters with a tiny nugget: the FP32 factorisation
    breaks down, the block is re-solved in FP64 and flagged FP64_RETRY."""
    rng = np.random.default_rng(11)
    centres = rng.random((300, 2))
    X = (np.repeat(centres, 6, axis=0) + rng.normal(0, 1e-6, (1800, 2)))
    Y = np.sin(7 * X[:, :1]) + np.cos(5 * X[:, 1:])
    Z = rng.random((200, 2))
    spec = wl.KernelSpec("matern", 2.5, 0.2, 1.0, 1e-9)
    ok, gk = kern_pair(spec)
    Xd = dev(X)
    nbr, _ = fb.fmgp_build_knn(Xd, 11)
    C, st = fb.fmgp_precompute(Xd, dev(Y), nbr, 12, gk, fb.PREC_MIXED)
    s = st.cpu().numpy()
    assert (s == fb.BLOCK_FP64_RETRY).sum() > 0
    nb, _ = oracle.self_knn(X, 11)  # the oracle's own table
    np.testing.assert_array_equal(nbr.cpu().numpy(), nb)
    Cr, str_ = oracle.precompute(X, Y, nb, 12, ok)
    Cg = coeffs_to_f64(C, fb.PREC_MIXED)
    retry = (s == fb.BLOCK_FP64_RETRY) & (str_ == 0)
    assert retry.sum() > 0
    # cond(K) ~ 1e10 here: FP64 against FP64 agrees to ~cond * eps
    assert rel_rms(Cg[retry], Cr[retry]) < 1e-4


@pytest.mark.parametrize("precision", [fb.PREC_MIXED])
def test_loocv_mixed(cuda, precision):
    test_loocv_tiny(cuda, precision)
    W = wl.spatial(n=30_000, m=10, nu=1.5, b=3000)
    ok, gk = kern_pair(W.kernel)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, 50)
    Q, res = fb.fmgp_loocv_objective(X, dev(W.Y), nbr, 50, dev(W.batch), gk, precision)
    nb_rows, _ = oracle.knn(W.X, W.X[W.batch], 50, W.batch)  # the oracle's own rows
    nb = np.zeros((W.n, 50), np.int32)
    nb[W.batch] = nb_rows
    Qr, resr = oracle.loocv(W.X, W.Y, nb, 50, W.batch, ok)
    assert abs(Q - Qr) / abs(Qr) < MIXED_TOL
    assert rel_rms(res.cpu().numpy(), resr) < MIXED_TOL


def test_grid_knn_visit_counters(cuda):
    """The optional counters of the grid kNN: every query examines at least kq
    candidates and keys at least kq of them; counting changes no result."""
    W = wl.tiny(n=3000, m=10)
    X = dev(W.X)
    ref, _ = fb.fmgp_build_knn(X, 29)
    fb.tune_set("count_visits", 1)
    try:
        nbr, _ = fb.fmgp_build_knn(X, 29)
        torch.cuda.synchronize()
        exam, keys, nq = fb.diag_counter(3), fb.diag_counter(4), fb.diag_counter(5)
    finally:
        fb.tune_set("count_visits", 0)
    assert torch.equal(nbr, ref)
    assert nq == W.n
    assert 29 * nq <= keys <= exam <= W.n * (W.n - 1)


@pytest.mark.parametrize("d,dtype", [(2, np.float64), (64, np.float32)])
def test_mixed_cta_kernel_all_modes(cuda, d, dtype):
    """Neighbourhoods of k = 100 (too large for one warp's share of an SM): the
    mixed form runs one CTA per neighbourhood.  Precompute, prediction, LOOCV
    and plain MuyGPs prediction, r = 3, against the oracle's own tables."""
    rng = np.random.default_rng(d)
    n, m, k = 4_000, 300, 100
    X = rng.random((n, d)).astype(dtype)
    Z = rng.random((m, d)).astype(dtype)
    Xo, Zo = X.astype(np.float64), Z.astype(np.float64)
    Y = np.stack([np.sin(3 * Xo[:, 0]), np.cos(2 * Xo[:, -1]), Xo[:, 0] * Xo[:, -1]], axis=1)
    spec = wl.KernelSpec("matern", 1.5, 0.35 * np.sqrt(d), 1.0, 1e-3)
    ok, gk = kern_pair(spec)
    Xd, Yd, Zd = dev(X), dev(Y), dev(Z)
    nbr, _ = fb.fmgp_build_knn(Xd, k)
    nb, _ = oracle.self_knn(Xo, k)
    np.testing.assert_array_equal(nbr.cpu().numpy(), nb)
    C, st = fb.fmgp_precompute(Xd, Yd, nbr, k, gk, fb.PREC_MIXED)
    Cr, _ = oracle.precompute(Xo, Y, nb, k, ok)
    assert rel_rms(coeffs_to_f64(C, fb.PREC_MIXED), Cr) < 1e-6
    yh, _ = fb.fmgp_predict(Xd, nbr, C, k, gk, Zd, fb.PREC_MIXED)
    yr, _ = oracle.predict(Xo, nb, Cr, ok, Zo)
    assert rel_rms(yh.cpu().numpy(), yr) < MIXED_TOL
    batch = np.arange(0, n, 7).astype(np.int64)
    Q, res = fb.fmgp_loocv_objective(Xd, Yd, nbr, k, dev(batch), gk, fb.PREC_MIXED)
    Qr, resr = oracle.loocv(Xo, Y, nb, k, batch, ok)
    assert abs(Q - Qr) / abs(Qr) < MIXED_TOL
    assert rel_rms(res.cpu().numpy(), resr) < MIXED_TOL
    ym, _ = fb.fmgp_muygps_predict(Xd, Yd, Zd, k, gk, fb.PREC_MIXED)
    ymr, _ = oracle.muygps_predict(Xo, Y, Zo, k, ok)
    assert rel_rms(ym.cpu().numpy(), ymr) < MIXED_TOL
