"""Plain MuyGPs prediction (Eq. 8), the comparator FastMuyGPs accelerates:
neighbour tables of the test points bit-exact, predictions within the
path's tolerance of the oracle, and equal to FastMuyGPs at training points."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import FP64_TOL, MIXED_TOL, dev, kern_pair, rel_rms

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [fb.PREC_FP64, fb.PREC_MIXED])
@pytest.mark.parametrize("name", ["tiny", "spatial", "large", "d16", "borehole"])
def test_muygps_matches_oracle(cuda, prec, name):
    if name == "tiny":
        W = wl.tiny(m=400)
    elif name == "spatial":
        W = wl.spatial(n=20_000, m=1_500, nu=0.5)
    elif name == "large":
        W = wl.large(n=200_000, m=800)
    elif name == "borehole":
        W = wl.borehole(n=5_000, m=200, k=150, nugget=1e-5)
    else:
        rng = np.random.default_rng(4)
        X = rng.random((6000, 16))
        Z = rng.random((300, 16))
        W = wl.Workload("d16", X, np.sin(3 * X.sum(1, keepdims=True)), Z, Z[:, :1], 20,
                        wl.KernelSpec("rbf", 0.0, 0.5, 1.0, 1e-3), np.arange(5))
    ok, gk = kern_pair(W.kernel)
    yh, nb = fb.fmgp_muygps_predict(dev(W.X), dev(W.Y), dev(W.Z), W.k, gk, prec, with_nbr=True)
    yr, nr = oracle.muygps_predict(W.X, W.Y, W.Z, W.k, ok)
    np.testing.assert_array_equal(nb.cpu().numpy(), nr)
    tol = FP64_TOL if prec == fb.PREC_FP64 else MIXED_TOL
    assert rel_rms(yh.cpu().numpy(), yr) < tol


def test_muygps_equals_fastmuygps_at_training_points(cuda):
    W = wl.spatial(n=10_000, m=10, nu=1.5)
    _, gk = kern_pair(W.kernel)
    X, Y = dev(W.X), dev(W.Y)
    nbr, _ = fb.fmgp_build_knn(X, 49)
    C, _ = fb.fmgp_precompute(X, Y, nbr, 50, gk, fb.PREC_FP64)
    rows = torch.tensor([0, 17, 4242, 9999], device="cuda")
    Zt = X[rows].contiguous()
    yf, _ = fb.fmgp_predict(X, nbr, C, 50, gk, Zt, fb.PREC_FP64)
    ym, nm = fb.fmgp_muygps_predict(X, Y, Zt, 50, gk, fb.PREC_FP64, with_nbr=True)
    assert torch.equal(nm[:, 0], rows.to(torch.int32))
    assert torch.equal(nm[:, 1:], nbr[rows])
    assert rel_rms(ym.cpu().numpy(), yf.cpu().numpy()) < 1e-12
