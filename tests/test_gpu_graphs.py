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


@pytest.mark.parametrize("prec", [fb.PREC_FP64, fb.PREC_MIXED])
def test_whole_step_with_loocv_replays_from_a_cuda_graph(cuda, prec):
    """kNN table, precompute, prediction and the LOOCV objective (written to
    device memory by fmgp_loocv_objective_device) in one graph: replays give
    the eager results bit for bit, and Q equals fmgp_loocv_objective's."""
    W = wl.spatial(n=20_000, m=3_000, nu=0.5, b=2_000)
    _, gk = kern_pair(W.kernel)
    X, Y, Z, B = dev(W.X), dev(W.Y), dev(W.Z), dev(W.batch)
    k = 50
    nbr = torch.empty((W.n, k), dtype=torch.int32, device="cuda")
    C = torch.empty(fb.coeff_shape(W.n, k, 1, prec),
                    dtype=torch.float64 if prec == fb.PREC_FP64 else torch.float32, device="cuda")
    st = torch.empty(W.n, dtype=torch.int8, device="cuda")
    yh = torch.empty((W.m, 1), dtype=torch.float64, device="cuda")
    near = torch.empty(W.m, dtype=torch.int32, device="cuda")
    Q = torch.empty(1, dtype=torch.float64, device="cuda")
    fails = torch.empty(1, dtype=torch.int32, device="cuda")
    res = torch.empty(len(W.batch), dtype=torch.float64, device="cuda")

    def step():
        fb.fmgp_build_knn(X, k, nbr_out=nbr)
        fb.fmgp_precompute(X, Y, nbr, k, gk, prec, C_out=C, status_out=st)
        fb.fmgp_predict(X, nbr, C, k, gk, Z, prec, Yhat_out=yh, nearest_out=near)
        fb.fmgp_loocv_objective_device(X, Y, nbr, k, B, gk, prec, Q_out=Q, fails_out=fails,
                                       resid_out=res)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ref = [t.clone() for t in (nbr, C, yh, near, Q, res)]
    assert int(fails.item()) == 0
    Qh, _ = fb.fmgp_loocv_objective(X, Y, nbr, k, B, gk, prec)
    assert Qh == float(Q.item())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(2):
        for t in (C, yh, Q, res):
            t.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(ref, (nbr, C, yh, near, Q, res)))


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
    cw, panel, pers = fb.autotune_choice(50, 2, 1, fb.PREC_MIXED)
    assert cw == w and panel in (4, 8) and pers in (0, 1)
    nbr1, d1 = fb.fmgp_build_knn(X, 50, with_dist=True)
    C1, _ = fb.fmgp_precompute(X, Y, nbr1, 50, gk, fb.PREC_MIXED)
    assert torch.equal(nbr0, nbr1) and torch.equal(d0, d1)
    assert torch.equal(C0, C1)
    fb.autotune_reset()


@pytest.mark.parametrize("panel", [4, 8])
def test_every_panel_width_gives_the_same_predictions(cuda, panel):
    """Both instantiated Cholesky panel widths of the mixed kernel give
    predictions that agree with the FP64 path (the FP32 dot products are
    summed in a different order, so the factor differs in rounding; the
    refinement removes it), and each width reproduces itself bit for bit."""
    W = wl.spatial(n=20_000, m=2_000, nu=1.5)
    _, gk = kern_pair(W.kernel)
    X, Y, Z = dev(W.X), dev(W.Y), dev(W.Z)
    for k in (24, 50):
        nbr, _ = fb.fmgp_build_knn(X, k - 1)
        C64, _ = fb.fmgp_precompute(X, Y, nbr, k, gk, fb.PREC_FP64)
        y64, _ = fb.fmgp_predict(X, nbr, C64, k, gk, Z, fb.PREC_FP64)
        fb.tune_set("block_panel", panel)
        try:
            C, _ = fb.fmgp_precompute(X, Y, nbr, k, gk, fb.PREC_MIXED)
            C2, _ = fb.fmgp_precompute(X, Y, nbr, k, gk, fb.PREC_MIXED)
        finally:
            fb.tune_set("block_panel", 0)
        assert torch.equal(C, C2)
        y, _ = fb.fmgp_predict(X, nbr, C, k, gk, Z, fb.PREC_MIXED)
        rel = float(torch.linalg.norm(y - y64) / torch.linalg.norm(y64))
        assert rel < 1e-7, rel


@pytest.mark.parametrize("prec", [fb.PREC_MIXED, fb.PREC_FP64])
@pytest.mark.parametrize("k", [50, 120])
def test_persistent_and_multiwave_launches_agree(cuda, prec, k):
    """The neighbourhood kernels give bit-identical coefficients, LOOCV
    residuals and MuyGPs predictions whether they run persistent (one wave of
    CTAs claiming neighbourhoods from a device counter) or as eight waves of
    grid-stride CTAs: a neighbourhood's arithmetic does not depend on the warp
    or CTA that runs it.  k = 50 runs the one-warp kernels, k = 120 the
    CTA-per-neighbourhood ones."""
    W = wl.spatial(n=12_000, m=700, nu=1.5, b=900)
    _, gk = kern_pair(W.kernel)
    X, Y, Z, B = dev(W.X), dev(W.Y), dev(W.Z), dev(W.batch)
    nbr, _ = fb.fmgp_build_knn(X, k - 1)
    nbr_l, _ = fb.fmgp_build_knn(X, k)
    out = {}
    for p in (1, 0):
        fb.tune_set("block_persistent", p)
        try:
            assert fb.tune_get("block_persistent") == p
            C, st = fb.fmgp_precompute(X, Y, nbr, k, gk, prec)
            Q, res = fb.fmgp_loocv_objective(X, Y, nbr_l, k, B, gk, prec)
            yh, _ = fb.fmgp_muygps_predict(X, Y, Z, k, gk, prec)
        finally:
            fb.tune_set("block_persistent", -1)
        torch.cuda.synchronize()
        assert int((st != 0).sum()) == 0
        out[p] = (C, Q, res, yh)
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][2], out[1][2])
    assert torch.equal(out[0][3], out[1][3])
