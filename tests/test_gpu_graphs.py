"""Batching form: the asynchronous entry points (kNN table, precompute with a
status array, prediction) can be captured into one CUDA graph after a
warm-up call and replayed; replays reproduce the eager results bit for bit.
Also checks that the autotuner's choices leave results unchanged."""
import numpy as np
import pytest
import torch

from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import dev, kern_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [fb.PREC_FP64, fb.PREC_MIXED])
def test_pipeline_replays_from_a_cuda_graph(cuda, prec):
    W = wl.spatial(n=20_000, m=3_000, nu=1.5)
    _, gk = kern_pair(W.kernel)
    X, Y, Z = dev(W.X), dev(W.Y), dev(W.Z)
    k = 50
    nbr = torch.empty((W.n, k - 1), dtype=torch.int32, device="cuda")
    C = torch.empty(fb.coeff_shape(W.n, k, 1, prec),
                    dtype=torch.float64 if prec == fb.PREC_FP64 else torch.float32, device="cuda")
    st = torch.empty(W.n, dtype=torch.int8, device="cuda")
    yh = torch.empty((W.m, 1), dtype=torch.float64, device="cuda")
    near = torch.empty(W.m, dtype=torch.int32, device="cuda")

    def step():
        fb.fmgp_build_knn(X, k - 1, nbr_out=nbr)
        fb.fmgp_precompute(X, Y, nbr, k, gk, prec, C_out=C, status_out=st)
        fb.fmgp_predict(X, nbr, C, k, gk, Z, prec, Yhat_out=yh, nearest_out=near)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ref_y, ref_n, ref_c = yh.clone(), near.clone(), C.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(2):
        yh.zero_()
        C.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(yh, ref_y) and torch.equal(near, ref_n) and torch.equal(C, ref_c)


def test_autotuner_choices_keep_results(cuda):
    W = wl.spatial(n=30_000, m=2_000, nu=0.5)
    _, gk = kern_pair(W.kernel)
    X, Y, Z = dev(W.X), dev(W.Y), dev(W.Z)
    fb.autotune_reset()
    nbr0, d0 = fb.fmgp_build_knn(X, 50, with_dist=True)
    C0, _ = fb.fmgp_precompute(X, Y, nbr0, 50, gk, fb.PREC_MIXED)
    t = fb.fmgp_autotune_knn(X, 50)
    w = fb.fmgp_autotune_precompute(X, Y, nbr0, 50, gk, fb.PREC_MIXED, sample_rows=5000)
    assert t > 0 and w >= 1
    nbr1, d1 = fb.fmgp_build_knn(X, 50, with_dist=True)
    C1, _ = fb.fmgp_precompute(X, Y, nbr1, 50, gk, fb.PREC_MIXED)
    assert torch.equal(nbr0, nbr1) and torch.equal(d0, d1)
    assert torch.equal(C0, C1)
    fb.autotune_reset()
