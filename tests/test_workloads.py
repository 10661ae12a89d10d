"""The seeded input recipes (shared by the GPU tests and the oracle) have the
shapes, ranges, structure and determinism their documentation states (CPU)."""
import numpy as np
import pytest

from paper_2205_10879_gb300 import workloads as wl


def _check_batch(W, b):
    assert W.batch.dtype == np.int64 and W.batch.shape == (min(b, W.n),)
    assert np.all(np.diff(W.batch) > 0)  # sorted, without replacement
    assert W.batch[0] >= 0 and W.batch[-1] < W.n


@pytest.mark.parametrize("make", [lambda: wl.tiny(n=800, m=200, b=100),
                                  lambda: wl.spatial(n=3000, m=700, b=300),
                                  lambda: wl.highdim(n=500, m=120, b=50),
                                  lambda: wl.large(n=3000, m=500, b=200),
                                  lambda: wl.borehole(n=2000, m=400, b=100)])
def test_recipes_are_deterministic(make):
    a, b = make(), make()
    for f in ("X", "Y", "Z", "Ztrue", "batch"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_tiny_recipe():
    W = wl.tiny()
    assert (W.n, W.m, W.d, W.r, W.k) == (2000, 500, 2, 1, 30)
    assert W.kernel == wl.KernelSpec("matern", 1.5, 0.1, 1.0, 1e-4)
    assert W.X.min() >= 0 and W.X.max() < 1 and W.Z.min() >= 0 and W.Z.max() < 1
    f = np.sin(2 * np.pi * W.X[:, 0]) * np.cos(2 * np.pi * W.X[:, 1])
    assert 0.009 < np.std(W.Y[:, 0] - f) < 0.011  # N(0, 0.01^2) noise
    _check_batch(W, 500)


def test_spatial_and_large_recipes():
    S = wl.spatial(n=20_000, m=4_000, b=1_000)
    assert (S.d, S.r, S.k) == (2, 1, 50) and S.kernel == wl.KernelSpec("matern", 1.5, 0.1, 1.0, 1e-3)
    assert wl.spatial(n=100, m=10, nu=0.5).kernel.nu == 0.5
    # 20 random Fourier features scaled by sqrt(2/20): unit variance, plus small noise
    assert 0.7 < np.std(S.Y) < 1.3
    L = wl.large(n=5_000, m=1_000, b=500)
    assert (L.d, L.k) == (3, 64) and L.kernel == wl.KernelSpec("matern", 2.5, 0.1, 1.0, 1e-5)
    assert L.X.min() >= 0 and L.X.max() < 1
    _check_batch(S, 1_000)
    _check_batch(L, 500)


def test_highdim_recipe():
    W = wl.highdim(n=2_000, m=300, b=200)
    assert W.X.dtype == np.float32 and W.X.shape == (2_000, 784) and W.r == 10 and W.k == 30
    assert W.kernel == wl.KernelSpec("rbf", 0.0, 7.0, 1.0, 1e-2)
    zero = np.mean(W.X == 0)
    assert abs(zero - 0.8) < 0.003  # 80 % exact zeros
    nz = W.X[W.X != 0]
    assert nz.min() > 0 and nz.max() <= 1  # U(0, 1]
    # centred one-hot responses: each row is e_c - mu, so rows sum to 0 and
    # the training column means vanish
    np.testing.assert_allclose(W.Y.sum(axis=1), 0.0, atol=1e-12)
    np.testing.assert_allclose(W.Y.mean(axis=0), 0.0, atol=1e-12)
    mu = W.extra["col_mean"]
    hot = np.argmax(W.Y, axis=1)
    np.testing.assert_allclose(W.Y[np.arange(W.n), hot], 1.0 - mu[hot], atol=1e-12)


def test_borehole_recipe_is_a_latin_hypercube():
    n, m = 3_000, 600
    W = wl.borehole(n=n, m=m, b=100)
    assert W.d == 8 and W.k == 150 and W.kernel.kind == "rbf" and W.kernel.length_scale == 43.27
    U = np.vstack([W.X, W.Z]) * wl.BOREHOLE_SCALE  # back to unit-cube coordinates
    N = n + m
    for j in range(8):
        if j in wl.BOREHOLE_VARYING:
            strata = np.floor(U[:, j] * N + 1e-9).astype(int)
            assert sorted(strata) == list(range(N))  # one point per stratum
        else:
            np.testing.assert_allclose(U[:, j], 0.5)
    # responses are the flow function, centred by the training mean
    assert abs(W.Y.mean()) < 1e-9
    assert 0.0 < W.extra["u_true"] < 1.0
