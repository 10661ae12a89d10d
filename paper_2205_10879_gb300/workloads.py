"""Seeded synthetic inputs for the FastMuyGPs posterior-mean path.

This module holds none of the method's arithmetic: it only draws features,
responses and batches with numpy's PCG64 generator.  It imports nothing from
the rest of the package, so both the CUDA-path tests and the oracle can be fed
from it.

Workloads (the paper's datasets are not available, so these stand in for them
with the paper's shapes):
  tiny     n=2,000  m=500     d=2   y = sin(2 pi x1) cos(2 pi x2) + N(0, 0.01^2)
           Matern nu=1.5, rho=0.1, sigma^2=1, tau^2=1e-4, k=30
  spatial  n=150,000 m=50,000 d=2   y = 20 random Fourier features + N(0, 0.05^2)
           Matern nu in {0.5, 1.5}, rho=0.1, tau^2=1e-3, k=50
           (stands in for the 2-D MODIS surface-temperature problem of Sec. 4.1:
           105,569 train / 42,740 test on a spatial grid)
  highdim  n=60,000 m=10,000  d=784 float32, 80% exact zeros else U(0,1],
           r=10 one-hot responses of argmax(x W), centred by the training column
           mean; RBF rho=7, tau^2=1e-2, k=30
           (stands in for the 400-D star-galaxy images of Sec. 4.3)
  large    n=10,000,000 m=1,000,000 d=3, 50 random Fourier features + N(0, 0.02^2),
           Matern nu=2.5, rho=0.1, tau^2=1e-5, k=64
  borehole n=100,000 m=20,000 d=8 (4 varying), the borehole flow function of
           Sec. 4.2 on a Latin hypercube, inputs pre-scaled per coordinate, RBF,
           k=150; also the MCMC calibration target of Sec. 4.2 (r_w = 0.09)
Seeds: workload number c (tiny=1, spatial=2, highdim=3, large=4, serving=5,
borehole=6)
uses 1000c for X, +1 noise, +2 Z, +3 Fourier features / linear map, +4 the
LOOCV batch, +5 held-out test noise.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

WORKLOAD_IDS = {"tiny": 1, "spatial": 2, "highdim": 3, "large": 4, "serving": 5, "borehole": 6}


@dataclass
class KernelSpec:
    kind: str = "matern"      # "matern" or "rbf"
    nu: float = 1.5
    length_scale: float = 0.1
    variance: float = 1.0
    nugget: float = 1e-4


@dataclass
class Workload:
    name: str
    X: np.ndarray             # n x d (float64, or float32 for highdim)
    Y: np.ndarray             # n x r float64
    Z: np.ndarray             # m x d
    Ztrue: np.ndarray         # m x r noisy held-out responses at Z
    k: int
    kernel: KernelSpec
    batch: np.ndarray         # LOOCV batch (int64, sampled without replacement)
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def m(self):
        return self.Z.shape[0]

    @property
    def d(self):
        return self.X.shape[1]

    @property
    def r(self):
        return self.Y.shape[1]


def _rng(c, off):
    return np.random.default_rng(1000 * c + off)


def rff_response(P, omega, phase):
    """Sum of Q random Fourier features sqrt(2/Q) cos(omega_q . x + b_q)."""
    Q = omega.shape[0]
    out = np.zeros(P.shape[0], np.float64)
    step = 1 << 18
    for s in range(0, P.shape[0], step):
        out[s:s + step] = np.cos(P[s:s + step] @ omega.T + phase).sum(axis=1)
    return out * np.sqrt(2.0 / Q)


def _batch(c, n, b):
    b = min(b, n)
    return np.sort(_rng(c, 4).choice(n, size=b, replace=False)).astype(np.int64)


def tiny(n=2000, m=500, k=30, b=500):
    c = 1
    X = _rng(c, 0).random((n, 2))
    Z = _rng(c, 2).random((m, 2))

    def f(P):
        return np.sin(2 * np.pi * P[:, 0]) * np.cos(2 * np.pi * P[:, 1])
    Y = (f(X) + _rng(c, 1).normal(0, 0.01, n))[:, None]
    Zt = (f(Z) + _rng(c, 5).normal(0, 0.01, m))[:, None]
    return Workload("tiny", X, Y, Z, Zt, k, KernelSpec("matern", 1.5, 0.1, 1.0, 1e-4),
                    _batch(c, n, b))


def _spatial_like(name, c, n, m, d, nfeat, noise, k, kern, b, sigma_w=8 * np.pi):
    X = _rng(c, 0).random((n, d))
    Z = _rng(c, 2).random((m, d))
    g = _rng(c, 3)
    omega = g.normal(0.0, sigma_w, (nfeat, d))
    phase = g.uniform(0.0, 2 * np.pi, nfeat)
    Y = (rff_response(X, omega, phase) + _rng(c, 1).normal(0, noise, n))[:, None]
    Zt = (rff_response(Z, omega, phase) + _rng(c, 5).normal(0, noise, m))[:, None]
    return Workload(name, X, Y, Z, Zt, k, kern, _batch(c, n, b))


def spatial(n=150_000, m=50_000, k=50, nu=1.5, b=10_000):
    return _spatial_like("spatial", 2, n, m, 2, 20, 0.05, k,
                         KernelSpec("matern", nu, 0.1, 1.0, 1e-3), b)


def large(n=10_000_000, m=1_000_000, k=64, b=10_000):
    return _spatial_like("large", 4, n, m, 3, 50, 0.02, k,
                         KernelSpec("matern", 2.5, 0.1, 1.0, 1e-5), b)


def highdim(n=60_000, m=10_000, d=784, r=10, k=30, b=5_000):
    c = 3

    def feats(g, rows):
        P = g.random((rows, d), dtype=np.float32)
        P = np.float32(1.0) - P                       # U(0,1]
        P[g.random((rows, d)) < 0.8] = 0.0
        return P
    X = feats(_rng(c, 0), n)
    Z = feats(_rng(c, 2), m)
    W = _rng(c, 3).normal(0.0, 1.0, (d, r))
    lab_x = np.argmax(X.astype(np.float64) @ W, axis=1)
    lab_z = np.argmax(Z.astype(np.float64) @ W, axis=1)
    Y = np.eye(r)[lab_x]
    mu = Y.mean(axis=0)
    Y = Y - mu
    Zt = np.eye(r)[lab_z] - mu
    return Workload("highdim", X, Y, Z, Zt, k, KernelSpec("rbf", 0.0, 7.0, 1.0, 1e-2),
                    _batch(c, n, b), extra={"labels_test": lab_z, "col_mean": mu})


def serving_models(count=8, seed_scale=1.0, n_max: Optional[int] = None):
    """Eight resident models: n log-uniform in [1e4, 2e6], d in {2,3,16,64},
    k in {16,32,64,128}, Matern or RBF, rho = 0.1 sqrt(d), responses from random
    Fourier features with omega ~ N(0, (8 pi)^2 / d)."""
    c = 5
    g = _rng(c, 3)
    ds = [2, 3, 16, 64]
    ks = [16, 32, 64, 128]
    specs = []
    for j in range(count):
        n = int(np.exp(g.uniform(np.log(1e4), np.log(2e6))) * seed_scale)
        if n_max is not None:
            n = min(n, n_max)
        d = ds[j % 4]
        k = ks[(j // 2) % 4] if j < 8 else ks[j % 4]
        kind = "matern" if j % 2 == 0 else "rbf"
        nu = [0.5, 1.5, 2.5][j % 3]
        specs.append(dict(n=max(n, 4 * k), d=d, k=k,
                          kernel=KernelSpec(kind, nu if kind == "matern" else 0.0,
                                            0.1 * np.sqrt(d), 1.0, 1e-3)))
    models = []
    for j, s in enumerate(specs):
        gj = np.random.default_rng(1000 * c + 100 + j)
        X = gj.random((s["n"], s["d"]))
        omega = gj.normal(0.0, 8 * np.pi / np.sqrt(s["d"]), (20, s["d"]))
        phase = gj.uniform(0.0, 2 * np.pi, 20)
        Y = (rff_response(X, omega, phase) + gj.normal(0, 0.05, s["n"]))[:, None]
        models.append(dict(X=X, Y=Y, k=s["k"], kernel=s["kernel"], omega=omega, phase=phase))
    return models


def serving_requests(models, count, seed=5005, max_points=65_536):
    """Request stream: (model id, test points) with log-uniform sizes 1..65,536,
    test points drawn like the model's training inputs."""
    g = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        j = int(g.integers(len(models)))
        size = int(np.exp(g.uniform(0.0, np.log(max_points))))
        d = models[j]["X"].shape[1]
        out.append((j, g.random((max(size, 1), d))))
    return out


# Borehole flow (Sec. 4.2).  Physical inputs in the order r_w, r, T_u, H_u,
# T_l, H_l, L, K_w with the ranges the paper lists; flow in m^3/yr.
BOREHOLE_LO = np.array([0.05, 100.0, 63070.0, 990.0, 63.1, 700.0, 1120.0, 9855.0])
BOREHOLE_HI = np.array([0.15, 50000.0, 115600.0, 1110.0, 116.0, 820.0, 1680.0, 12045.0])
# per-coordinate divisors that make the model anisotropic (Sec. 4.2)
BOREHOLE_SCALE = np.array([0.0625, 0.25, 1.0, 0.25, 0.5, 0.25, 0.125, 0.5])
BOREHOLE_VARYING = (0, 1, 2, 4)        # r_w, r, T_u, T_l; the rest sit at mid-range


def borehole_flow(P):
    """The borehole function on physical inputs P (N x 8)."""
    rw, r, tu, hu, tl, hl, ln, kw = (P[:, j] for j in range(8))
    lg = np.log(r / rw)
    return 2.0 * np.pi * tu * (hu - hl) / (lg * (1.0 + 2.0 * ln * tu / (lg * rw * rw * kw) + tu / tl))


def borehole_unit_to_model(U):
    """Unit-cube coordinates (N x 8) -> model inputs (each column divided by its scale)."""
    return U / BOREHOLE_SCALE


def borehole_unit_to_physical(U):
    return BOREHOLE_LO + U * (BOREHOLE_HI - BOREHOLE_LO)


def borehole(n=100_000, m=20_000, k=150, b=10_000, length_scale=43.27, nugget=1e-8):
    """One Latin hypercube of n + m points over the four varying inputs (the
    fixed four at mid-range), split at random into n training and m test
    points; responses centred by the training mean.  extra holds the MCMC
    calibration target: r_w = 0.09 (unit coordinate 0.4) with the other
    inputs at mid-range, its centred flow, and the base model input z0."""
    c = 6
    N = n + m
    g = _rng(c, 0)
    U = np.full((N, 8), 0.5)
    for j in BOREHOLE_VARYING:
        U[:, j] = (g.permutation(N) + g.random(N)) / N
    perm = _rng(c, 2).permutation(N)
    tr, te = np.sort(perm[:n]), np.sort(perm[n:])
    f = borehole_flow(borehole_unit_to_physical(U))
    mean = float(f[tr].mean())
    X = borehole_unit_to_model(U[tr])
    Z = borehole_unit_to_model(U[te])
    u_true = np.full((1, 8), 0.5)
    u_true[0, 0] = (0.09 - BOREHOLE_LO[0]) / (BOREHOLE_HI[0] - BOREHOLE_LO[0])
    f_obs = float(borehole_flow(borehole_unit_to_physical(u_true))[0]) - mean
    extra = {"y_mean": mean, "u_true": float(u_true[0, 0]), "f_obs": f_obs,
             "z0": borehole_unit_to_model(u_true)[0], "dim": 0,
             "lo": 0.0, "hi": 1.0 / BOREHOLE_SCALE[0], "scale": float(BOREHOLE_SCALE[0])}
    return Workload("borehole", X, (f[tr] - mean)[:, None], Z, (f[te] - mean)[:, None], k,
                    KernelSpec("rbf", 0.0, length_scale, 1.0, nugget), _batch(c, n, b), extra)


def by_name(name, **kw):
    return {"tiny": tiny, "spatial": spatial, "highdim": highdim, "large": large,
            "borehole": borehole}[name](**kw)
