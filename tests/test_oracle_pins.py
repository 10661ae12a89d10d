"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics, independent of the oracle's own code (CPU only).

Each pin is chosen so that a plausible slip in the oracle fails it:
 - Matern closed forms vs the Bessel expression of Eq. 3 (scipy.special.kv):
   a wrong sqrt(2 nu) scaling, polynomial term or rho use.
 - RBF as the nu -> infinity limit of Eq. 3: a wrong RBF length-scale reading.
 - kNN vs an all-pairs lexsort with tie-heavy integer grids: selection, order,
   tie rule, self exclusion.
 - Blocks symmetric, nugget only on the diagonal, SPD with lambda_min >= sigma^2 tau^2.
 - k = n reduces Eq. 7 to the dense GP mean of Eq. 2 (scipy cho_solve), for
   several responses: the solve, the cross-covariance, the C layout.
 - Interpolation identity at z = x_i: S_i[0] = i, the row lookup, no nugget in
   the cross-covariance.
 - Leave-one-out block identity: ties the LOOCV objective (Eq. 5) to the
   precomputed C (Eq. 6).
 - sigma^2 invariance of the mean and 1/sigma^2 scaling of C.
 - Long-double re-evaluation bounds the FP64 rounding error.
 - k = 1 and k = 2 neighbourhoods: C and the prediction in closed form (a
   scalar division, the textbook 2 x 2 inverse) with the Bessel-form kernel;
   the LOOCV objective with one neighbour in closed form.
 - Subsampled precompute (Sec. 5): with every training point as a centre it is
   the full method; at a test point whose nearest training point is a centre
   it agrees with the full method; at a centre it interpolates (as Eq. 7 does).
 - Metropolis calibration (Sec. 4.2): with a linear response the posterior of
   the calibrated input is a (truncated) Gaussian in closed form, which the
   chains must reproduce (sign, factor 1/2, prior rejection); with Exp(1)
   draws fixed at 0 the chain only takes strictly better moves; with them at
   +inf every in-range proposal is taken and the others rejected.
"""
import numpy as np
import pytest
import scipy.linalg as sl
from scipy.special import gamma, kv

import oracle
from paper_2205_10879_gb300 import workloads as wl


def matern_bessel(u, nu):
    """Eq. 3 without sigma^2/nugget: 2^(1-nu)/Gamma(nu) (sqrt(2nu) u)^nu K_nu(sqrt(2nu) u)."""
    u = np.asarray(u, np.float64)
    out = np.ones_like(u)
    nz = u > 0
    a = np.sqrt(2 * nu) * u[nz]
    out[nz] = 2 ** (1 - nu) / gamma(nu) * a ** nu * kv(nu, a)
    return out


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_closed_forms_match_bessel(nu):
    rho = 0.37
    u = np.concatenate([[0.0], np.geomspace(1e-6, 30, 400)])
    D = (u * rho) ** 2
    got = oracle.phi(oracle.kernel("matern", nu, rho), D)
    ref = matern_bessel(u, nu)
    assert got[0] == 1.0
    np.testing.assert_allclose(got, ref, rtol=2e-12, atol=1e-300)


def test_rbf_is_the_matern_limit():
    rho = 0.8
    u = np.linspace(0.05, 3.0, 60)
    D = (u * rho) ** 2
    rbf = oracle.phi(oracle.kernel("rbf", 0.0, rho), D)
    errs = []
    for nu in [5.0, 20.0, 80.0]:
        errs.append(np.max(np.abs(matern_bessel(u, nu) - rbf)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3
    # the alternative reading exp(-d^2/rho^2) is far from the limit
    assert np.max(np.abs(np.exp(-u ** 2) - matern_bessel(u, 80.0))) > 0.1


def _canon_keys(X, Q):
    # canonical key: left-to-right FP64 sum of squared differences
    t = Q[:, None, 0] - X[None, :, 0]
    s = t * t
    for j in range(1, X.shape[1]):
        t = Q[:, None, j] - X[None, :, j]
        s = s + t * t
    return s


def _allpairs_knn(X, kq, self_exclude=True, Q=None):
    Qm = X if Q is None else Q
    K = _canon_keys(X, Qm)
    idx = np.arange(X.shape[0])
    out = np.zeros((Qm.shape[0], kq), np.int64)
    for q in range(Qm.shape[0]):
        keys = K[q].copy()
        cand = idx
        if self_exclude:
            cand = idx[idx != q]
            keys = keys[idx != q]
        order = np.lexsort((cand, keys))
        out[q] = cand[order[:kq]]
    return out


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_knn_matches_allpairs_sort_on_tie_heavy_grid(d):
    rng = np.random.default_rng(10 + d)
    X = rng.integers(0, 4, size=(150, d)).astype(np.float64)  # many exact duplicates and ties
    for kq in [1, 7, 40]:
        idx, keys = oracle.self_knn(X, kq)
        np.testing.assert_array_equal(idx, _allpairs_knn(X, kq))
        assert np.all(np.diff(keys, axis=1) >= 0)
        # tie rule: equal keys appear in increasing index order
        eq = np.diff(keys, axis=1) == 0
        assert np.all(np.diff(idx, axis=1)[eq] > 0)
        assert not np.any(idx == np.arange(150)[:, None])


def test_knn_random_points_and_test_queries():
    rng = np.random.default_rng(3)
    X = rng.random((300, 2))
    Z = rng.random((50, 2))
    idx, _ = oracle.self_knn(X, 12)
    np.testing.assert_array_equal(idx, _allpairs_knn(X, 12))
    j, _ = oracle.knn(X, Z, 1)
    np.testing.assert_array_equal(j[:, 0], _allpairs_knn(X, 1, False, Z)[:, 0])


@pytest.mark.parametrize("kind,nu", [("matern", 0.5), ("matern", 1.5), ("matern", 2.5), ("rbf", 0)])
def test_blocks_symmetric_spd_nugget_on_diagonal(kind, nu):
    rng = np.random.default_rng(4)
    X = rng.random((80, 2))
    X[5] = X[9]  # a duplicate pair inside the block
    kern = oracle.kernel(kind, nu, 0.2, 1.7, 1e-3)
    S = np.array([5, 9, 3, 40, 41, 77, 12, 0], np.int32)
    K = oracle.assemble(X, S, kern)
    np.testing.assert_array_equal(K, K.T)
    np.testing.assert_allclose(np.diag(K), 1.7 * (1 + 1e-3), rtol=0, atol=0)
    assert K[0, 1] == pytest.approx(1.7)            # duplicate: no nugget off the diagonal
    assert np.linalg.eigvalsh(K).min() >= 1.7 * 1e-3 * (1 - 1e-8)


def _dense_kernel(A, B, nu, rho, var, kind="matern"):
    d = np.sqrt(((A[:, None, :] - B[None, :, :]) ** 2).sum(-1))
    if kind == "rbf":
        return var * np.exp(-d ** 2 / (2 * rho ** 2))
    return var * matern_bessel(d / rho, nu)


@pytest.mark.parametrize("kind,nu", [("matern", 1.5), ("matern", 0.5), ("rbf", 0.0)])
def test_k_equals_n_is_the_dense_gp_mean(kind, nu):
    rng = np.random.default_rng(5)
    n, r = 60, 3
    X = rng.random((n, 2))
    Y = rng.normal(size=(n, r))
    Z = rng.random((25, 2))
    rho, var, tau2 = 0.3, 2.0, 1e-3
    kern = oracle.kernel(kind, nu, rho, var, tau2)
    nbr, _ = oracle.self_knn(X, n - 1)
    C, st = oracle.precompute(X, Y, nbr, n, kern)
    assert not st.any()
    yh, _ = oracle.predict(X, nbr, C, kern, Z)
    Kxx = _dense_kernel(X, X, nu, rho, var, kind) + var * tau2 * np.eye(n)
    Kzx = _dense_kernel(Z, X, nu, rho, var, kind)
    ref = Kzx @ sl.cho_solve(sl.cho_factor(Kxx, lower=True), Y)
    np.testing.assert_allclose(yh, ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())


def test_interpolation_identity():
    W = wl.tiny(n=400, m=10)
    kern = oracle.kernel("matern", 1.5, 0.1, 1.3, 1e-4)
    nbr, _ = oracle.self_knn(W.X, 29)
    C, _ = oracle.precompute(W.X, W.Y, nbr, 30, kern)
    rows = np.array([0, 17, 123, 399])
    yh, near = oracle.predict(W.X, nbr, C, kern, W.X[rows])
    np.testing.assert_array_equal(near, rows)
    # K(x_i, X_Si) is row 0 of K_Si minus the nugget, so yhat = y_i - sigma^2 tau^2 C_i[0]
    ref = W.Y[rows, 0] - 1.3 * 1e-4 * C[rows, 0, 0]
    np.testing.assert_allclose(yh[:, 0], ref, rtol=1e-9, atol=1e-12)


def test_loo_identity_links_loocv_to_precompute():
    W = wl.tiny(n=500, m=10)
    kern = oracle.kernel("matern", 2.5, 0.15, 1.0, 1e-3)
    kl = 20
    nbr, _ = oracle.self_knn(W.X, kl)
    batch = np.array([3, 50, 77, 200, 499], np.int64)
    Q, res = oracle.loocv(W.X, W.Y, nbr, kl, batch, kern)
    C, _ = oracle.precompute(W.X, W.Y, nbr, kl + 1, kern)
    for q, i in enumerate(batch):
        S = np.concatenate([[i], nbr[i, :kl]]).astype(np.int32)
        Kinv00 = np.linalg.inv(oracle.assemble(W.X, S, kern))[0, 0]
        loo = C[i, 0, 0] / Kinv00
        assert res[q] == pytest.approx(loo ** 2, rel=1e-7)
    assert Q == pytest.approx(res.mean(), rel=1e-14)


def test_sigma2_invariance():
    W = wl.tiny(n=300, m=40)
    nbr, _ = oracle.self_knn(W.X, 19)
    k1 = oracle.kernel("matern", 1.5, 0.1, 1.0, 1e-3)
    k7 = oracle.kernel("matern", 1.5, 0.1, 7.0, 1e-3)
    C1, _ = oracle.precompute(W.X, W.Y, nbr, 20, k1)
    C7, _ = oracle.precompute(W.X, W.Y, nbr, 20, k7)
    np.testing.assert_allclose(C7 * 7.0, C1, rtol=1e-9)
    y1, _ = oracle.predict(W.X, nbr, C1, k1, W.Z)
    y7, _ = oracle.predict(W.X, nbr, C7, k7, W.Z)
    np.testing.assert_allclose(y7, y1, rtol=1e-10, atol=1e-13)


def test_not_spd_block_is_flagged():
    X = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 1.0], [2.0, 0.5]])
    Y = np.ones((4, 1))
    nbr, _ = oracle.self_knn(X, 2)
    kern = oracle.kernel("matern", 1.5, 1.0, 1.0, 0.0)  # no nugget: duplicates make K singular
    C, st = oracle.precompute(X, Y, nbr, 3, kern)
    assert st[0] == 1 and st[1] == 1
    assert np.all(C[0] == 0)


def test_long_double_bounds_fp64_rounding():
    W = wl.tiny()
    kern = oracle.kernel("matern", 1.5, 0.1, 1.0, 1e-4)
    nbr, _ = oracle.self_knn(W.X, 29)
    C, _ = oracle.precompute(W.X, W.Y, nbr, 30, kern)
    yh, near = oracle.predict(W.X, nbr, C, kern, W.Z)
    yl = oracle.fit_predict_ld(W.X, W.Y, nbr, 30, kern, W.Z, near)
    rel = np.linalg.norm(yh - yl) / np.linalg.norm(yl)
    assert rel < 1e-12, rel


def test_accuracy_is_plausible_on_tiny():
    """The method predicts the smooth tiny response well (sanity, not a pin)."""
    W = wl.tiny()
    kern = oracle.kernel("matern", 1.5, 0.1, 1.0, 1e-4)
    nbr, _ = oracle.self_knn(W.X, 29)
    C, _ = oracle.precompute(W.X, W.Y, nbr, 30, kern)
    yh, _ = oracle.predict(W.X, nbr, C, kern, W.Z)
    rmse = np.sqrt(np.mean((yh - W.Ztrue) ** 2))
    assert rmse < 0.05


def test_muygps_with_k_equal_n_is_the_dense_gp_mean():
    """Eq. 8 with every training point as neighbour reduces to Eq. 2."""
    rng = np.random.default_rng(9)
    n, r = 50, 2
    X = rng.random((n, 2))
    Y = rng.normal(size=(n, r))
    Z = rng.random((20, 2))
    rho, var, tau2 = 0.3, 1.5, 1e-3
    kern = oracle.kernel("matern", 2.5, rho, var, tau2)
    yh, _ = oracle.muygps_predict(X, Y, Z, n, kern)
    Kxx = _dense_kernel(X, X, 2.5, rho, var) + var * tau2 * np.eye(n)
    ref = _dense_kernel(Z, X, 2.5, rho, var) @ sl.cho_solve(sl.cho_factor(Kxx, lower=True), Y)
    np.testing.assert_allclose(yh, ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())


def test_muygps_equals_fastmuygps_at_training_points():
    """At z = x_j the test point's own k nearest neighbours are j and its k-1
    nearest others, i.e. S_j, so Eq. 8 and Eq. 7 are the same formula."""
    W = wl.tiny(n=600, m=10)
    kern = oracle.kernel("matern", 1.5, 0.1, 1.0, 1e-4)
    nbr, _ = oracle.self_knn(W.X, 29)
    C, _ = oracle.precompute(W.X, W.Y, nbr, 30, kern)
    rows = np.array([3, 44, 101, 599])
    yf, _ = oracle.predict(W.X, nbr, C, kern, W.X[rows])
    ym, N = oracle.muygps_predict(W.X, W.Y, W.X[rows], 30, kern)
    np.testing.assert_array_equal(N[:, 0], rows)
    np.testing.assert_array_equal(N[:, 1:], nbr[rows])
    np.testing.assert_allclose(ym, yf, rtol=1e-9, atol=1e-12)


# ------------------------------------------------------------------ MCMC --
def _linear_emulator(slope=3.0):
    """A 1-D emulator of y = slope * x on [0, 1]: dense training grid, so the
    posterior mean reproduces the line to ~1e-6."""
    X = np.linspace(0.0, 1.0, 201)[:, None]
    Y = slope * X
    kern = oracle.kernel("rbf", 0.0, 0.05, 1.0, 1e-10)
    nbr, _ = oracle.self_knn(X, 11)
    C, st = oracle.precompute(X, Y, nbr, 12, kern)
    assert not st.any()
    yh, _ = oracle.predict(X, nbr, C, kern, np.array([[0.25], [0.5], [0.75]]))
    np.testing.assert_allclose(yh[:, 0], slope * np.array([0.25, 0.5, 0.75]), atol=1e-5)
    return X, nbr, C, kern


def _draws(seed, steps, chains):
    g = np.random.default_rng(seed)
    return g.standard_normal((steps, chains)), g.exponential(1.0, (steps, chains))


@pytest.mark.parametrize("f_obs", [1.5, 0.15])
def test_mcmc_reproduces_the_closed_form_posterior(f_obs):
    """Likelihood N(f_obs; 3x, 0.3^2) and a uniform prior on [0, 1]: the
    posterior of x is N(f_obs/3, 0.1^2) truncated to [0, 1].  f_obs = 1.5
    puts the mode mid-range; 0.15 puts it half a standard deviation from the
    lower bound, where the truncation moves the mean to about 0.1009."""
    from scipy.stats import truncnorm
    X, nbr, C, kern = _linear_emulator()
    slope, sig = 3.0, 0.3
    mu, sd = f_obs / slope, sig / slope
    ref = truncnorm((0.0 - mu) / sd, (1.0 - mu) / sd, loc=mu, scale=sd)
    steps, chains, burn = 25_000, 16, 500
    noise, expo = _draws(77, steps, chains)
    x0 = np.linspace(0.2, 0.8, chains)
    S, acc, _ = oracle.mcmc(X, nbr, C, kern, [0.0], 0, 0.0, 1.0, f_obs, sig, 0.25, x0, noise,
                            expo)
    post = S[burn:].ravel()
    assert post.min() >= 0.0 and post.max() <= 1.0
    assert abs(post.mean() - ref.mean()) < 4e-3
    assert abs(post.std() / ref.std() - 1.0) < 0.04
    rate = acc.sum() / (steps * chains)
    assert 0.2 < rate < 0.8


def test_mcmc_takes_only_strictly_better_moves_when_expo_is_zero():
    X, nbr, C, kern = _linear_emulator()
    steps, chains = 300, 4
    noise, _ = _draws(78, steps, chains)
    expo = np.zeros_like(noise)
    x0 = np.array([0.05, 0.3, 0.7, 0.95])
    S, acc, margin = oracle.mcmc(X, nbr, C, kern, [0.0], 0, 0.0, 1.0, 1.2, 0.3, 0.1, x0, noise,
                                 expo)
    path = np.vstack([x0[None, :], S])
    yh, _ = oracle.predict(X, nbr, C, kern, path.reshape(-1, 1))
    err = np.abs(1.2 - yh[:, 0]).reshape(path.shape)
    moved = path[1:] != path[:-1]
    assert np.all(err[1:][moved] < err[:-1][moved])
    assert np.all(err[1:][~moved] == err[:-1][~moved])
    assert np.all(margin[moved] > 0) and np.all(margin[~moved] <= 0)
    assert np.array_equal(acc, moved.sum(axis=0))
    assert np.all(np.abs(path[-1] - 0.4) < 0.02)


def test_mcmc_with_infinite_expo_takes_every_in_range_proposal():
    X, nbr, C, kern = _linear_emulator()
    steps, chains = 200, 3
    noise, _ = _draws(79, steps, chains)
    expo = np.full_like(noise, np.inf)
    x0 = np.array([0.1, 0.5, 0.9])
    S, acc, margin = oracle.mcmc(X, nbr, C, kern, [0.0], 0, 0.0, 1.0, 1.5, 0.3, 0.2, x0, noise,
                                 expo)
    x = x0.copy()
    for t in range(steps):
        prop = x + 0.2 * noise[t]
        ok = (prop >= 0.0) & (prop <= 1.0)
        x = np.where(ok, prop, x)
        np.testing.assert_array_equal(S[t], x)
        assert np.all(np.isneginf(margin[t][~ok]))
    assert np.array_equal(acc, (S != np.vstack([x0[None, :], S[:-1]])).sum(axis=0))


# --------------------------------------------------- subsampled precompute --
def _subsample_setup():
    W = wl.tiny(n=1500, m=400)
    kern = oracle.kernel("matern", 1.5, 0.1, 1.0, 1e-4)
    nbr, _ = oracle.self_knn(W.X, 29)
    C, _ = oracle.precompute(W.X, W.Y, nbr, 30, kern)
    return W, kern, nbr, C


def test_subsample_with_every_row_is_the_full_method():
    W, kern, nbr, C = _subsample_setup()
    rows = np.arange(W.n)
    Cs, _ = oracle.precompute(W.X, W.Y, nbr, 30, kern, rows=rows)
    yr, cr = oracle.predict_rows(W.X, nbr, rows, Cs, kern, W.Z)
    yf, nf = oracle.predict(W.X, nbr, C, kern, W.Z)
    np.testing.assert_array_equal(cr, nf)
    np.testing.assert_array_equal(yr, yf)


def test_subsample_agrees_where_the_nearest_point_is_a_centre():
    """Half the training points as centres: test points whose global nearest
    training point is a centre use the same S and C row as the full method;
    the others use another centre and differ."""
    W, kern, nbr, C = _subsample_setup()
    rows = np.sort(np.random.default_rng(5).choice(W.n, W.n // 2, replace=False))
    Cs, _ = oracle.precompute(W.X, W.Y, nbr, 30, kern, rows=rows)
    yr, cr = oracle.predict_rows(W.X, nbr, rows, Cs, kern, W.Z)
    yf, nf = oracle.predict(W.X, nbr, C, kern, W.Z)
    same = np.isin(nf, rows)
    assert 0 < same.sum() < W.m
    np.testing.assert_array_equal(cr[same], nf[same])
    np.testing.assert_array_equal(yr[same], yf[same])
    assert np.all(np.isin(cr, rows))
    assert np.all(cr[~same] != nf[~same])


def test_subsample_interpolates_at_centres():
    """At z = x_c (c a centre) the prediction is y_c - sigma^2 tau^2 C_c[0]."""
    W, kern, nbr, _ = _subsample_setup()
    rows = np.arange(0, W.n, 3)
    Cs, _ = oracle.precompute(W.X, W.Y, nbr, 30, kern, rows=rows)
    yr, cr = oracle.predict_rows(W.X, nbr, rows, Cs, kern, W.X[rows])
    np.testing.assert_array_equal(cr, rows)
    np.testing.assert_allclose(yr, W.Y[rows] - 1e-4 * Cs[:, 0, :], rtol=0, atol=1e-9)


def _nearest_other(X, i):
    d2 = ((X - X[i]) ** 2).sum(1)
    d2[i] = np.inf
    return int(np.argmin(d2))


def test_small_neighbourhoods_match_closed_forms():
    """k = 1 and k = 2 reduce Eqs. 6-7 to a scalar division and the textbook
    2 x 2 inverse, with the kernel from the Bessel form of Eq. 3: pins the
    assembly (variance, nugget on the diagonal only), the solve and the
    prediction's use of S_{j*} = [j*, its neighbour]."""
    W = wl.tiny(n=300, m=25)
    s2, tau2, rho, nu = 1.7, 3e-3, 0.1, 1.5
    kern = oracle.kernel("matern", nu, rho, s2, tau2)
    X, y, Z = W.X, W.Y[:, 0], W.Z
    nn = np.array([_nearest_other(X, i) for i in range(W.n)])
    # k = 1: C_i = y_i / (s2 (1 + tau2)); yhat(z) = s2 phi(|z - x_j*|) C_j*
    C1, _ = oracle.precompute(X, W.Y, nn[:, None].astype(np.int32), 1, kern)
    np.testing.assert_allclose(C1[:, 0, 0], y / (s2 * (1 + tau2)), rtol=1e-13)
    yh1, near = oracle.predict(X, nn[:, None].astype(np.int32), C1, kern, Z)
    dz = np.sqrt(((Z - X[near]) ** 2).sum(1))
    np.testing.assert_allclose(yh1[:, 0], matern_bessel(dz / rho, nu) * y[near] / (1 + tau2),
                               rtol=1e-11)
    # k = 2: S_i = [i, nn(i)], K = s2 [[1+tau2, p], [p, 1+tau2]]
    C2, _ = oracle.precompute(X, W.Y, nn[:, None].astype(np.int32), 2, kern)
    p = matern_bessel(np.sqrt(((X - X[nn]) ** 2).sum(1)) / rho, nu)
    a = 1 + tau2
    det = s2 * (a * a - p * p)
    c0 = (a * y - p * y[nn]) / det
    c1 = (-p * y + a * y[nn]) / det
    np.testing.assert_allclose(C2[:, 0, 0], c0, rtol=1e-9)
    np.testing.assert_allclose(C2[:, 1, 0], c1, rtol=1e-9)
    yh2, near2 = oracle.predict(X, nn[:, None].astype(np.int32), C2, kern, Z)
    j = near2
    pz0 = matern_bessel(np.sqrt(((Z - X[j]) ** 2).sum(1)) / rho, nu)
    pz1 = matern_bessel(np.sqrt(((Z - X[nn[j]]) ** 2).sum(1)) / rho, nu)
    np.testing.assert_allclose(yh2[:, 0], s2 * (pz0 * c0[j] + pz1 * c1[j]), rtol=1e-9,
                               atol=1e-12)


def test_loocv_with_one_neighbour_is_a_scaled_copy():
    """k = 1 in Eqs. 4-5: each batch point is predicted from its nearest other
    point alone, yhat_i = phi(d_ij) y_j / (1 + tau2), so Q is the mean squared
    difference."""
    W = wl.tiny(n=250, m=5)
    tau2, rho = 1e-2, 0.2
    kern = oracle.kernel("matern", 0.5, rho, 2.0, tau2)
    X, y = W.X, W.Y[:, 0]
    nn = np.array([_nearest_other(X, i) for i in range(W.n)], np.int32)
    batch = np.array([0, 9, 41, 100, 249], np.int64)
    Q, res = oracle.loocv(X, W.Y, nn[:, None], 1, batch, kern)
    d = np.sqrt(((X[batch] - X[nn[batch]]) ** 2).sum(1))
    yh = matern_bessel(d / rho, 0.5) * y[nn[batch]] / (1 + tau2)
    np.testing.assert_allclose(res, (y[batch] - yh) ** 2, rtol=1e-10, atol=1e-15)
    assert Q == pytest.approx(np.mean((y[batch] - yh) ** 2), rel=1e-10)
