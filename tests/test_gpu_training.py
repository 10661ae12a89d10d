"""MuyGPs hyperparameter training (Algorithm 1) over the GPU LOOCV objective:
the optimiser lowers Q, its optimum agrees with a grid search of the
oracle's Q, and the GPU objective at the optimum matches the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import training
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import MIXED_TOL, dev

pytestmark = pytest.mark.gpu


def test_length_scale_optimum_matches_oracle_grid(cuda):
    pytest.importorskip("scipy")
    W = wl.tiny(n=2000, m=10, b=400)
    X, Y, B = dev(W.X), dev(W.Y), dev(W.batch)
    start = fb.make_kernel("matern", 1.5, 0.5, 1.0, 1e-4)
    out = training.optimize_hyperparameters(X, Y, B, 30, start, params=("length_scale",),
                                            bounds={"length_scale": (1e-3, 10.0)})
    assert out["q_best"] < out["q_start"]
    rho = out["theta"]["length_scale"]
    # oracle Q on a log grid around the optimum: the optimum is not beaten
    nb, _ = oracle.self_knn(W.X, 30)
    grid = np.geomspace(rho / 4, rho * 4, 25)
    qs = [oracle.loocv(W.X, W.Y, nb, 30, W.batch, oracle.kernel("matern", 1.5, g, 1.0, 1e-4))[0]
          for g in grid]
    q_at = oracle.loocv(W.X, W.Y, nb, 30, W.batch, oracle.kernel("matern", 1.5, rho, 1.0, 1e-4))[0]
    assert q_at <= min(qs) * (1 + 1e-3)
    assert abs(out["q_best"] - q_at) / q_at < MIXED_TOL
