"""Serving form: resident models and the continuous-batching server.

The key property: a request's predictions do not depend on what else is in
flight, so results are bit-identical when each request runs alone and when
all requests arrive at once and get batched and overlapped."""
import threading

import numpy as np
import pytest
import torch

from paper_2205_10879_gb300 import _binding as fb
from paper_2205_10879_gb300 import workloads as wl
from gpu_helpers import dev, kern_pair

pytestmark = pytest.mark.gpu


def _fit(W, k, prec):
    _, gk = kern_pair(W.kernel)
    X = dev(W.X)
    nbr, _ = fb.fmgp_build_knn(X, max(k - 1, 1))
    C, _ = fb.fmgp_precompute(X, dev(W.Y), nbr, k, gk, prec)
    return fb.FmgpModel(X, nbr, C, k, gk, prec)


def _wide(n, d, dtype, seed):
    rng = np.random.default_rng(seed)
    X = rng.random((n, d)).astype(dtype)
    Z = rng.random((700, d)).astype(dtype)
    return wl.Workload(f"d{d}", X, np.sin(X.sum(1, keepdims=True)).astype(np.float64), Z,
                       Z[:, :1].astype(np.float64), 20, wl.KernelSpec("rbf", 0.0, 0.7, 1.0, 1e-3),
                       np.arange(5))


@pytest.mark.parametrize("prec", [fb.PREC_FP64, fb.PREC_MIXED])
@pytest.mark.parametrize("shape", ["grid", "scan", "tensor64", "tensor32"])
def test_model_predict_matches_fmgp_predict(cuda, prec, shape):
    """A resident model (search grid, FP32 scan copy, or packed tensor-core
    training side, each built once) predicts exactly what fmgp_predict does."""
    if shape == "grid":
        W, k = wl.tiny(), 30
    elif shape == "scan":
        W, k = _wide(5000, 8, np.float64, 1), 20
    elif shape == "tensor64":
        W, k = _wide(6000, 24, np.float64, 2), 20
    else:
        W, k = _wide(6000, 40, np.float32, 3), 20
    md = _fit(W, k, prec)
    Z = dev(W.Z)
    c0 = fb.diag_counter(1)
    y1, n1 = md.predict(Z)
    torch.cuda.synchronize()
    if shape.startswith("tensor"):
        assert fb.diag_counter(1) == c0 + 1, "tensor-core path not taken"
    y2, n2 = fb.fmgp_predict(md.X, md.nbr, md.C, k, md.kernel, Z, prec)
    assert torch.equal(n1, n2)
    assert torch.equal(y1, y2)
    assert md.device_bytes() > 0
    md.close()


def _models():
    a = _fit(wl.tiny(n=4000, m=10), 30, fb.PREC_FP64)
    b = _fit(wl.large(n=60_000, m=10), 64, fb.PREC_MIXED)
    rng = np.random.default_rng(3)
    Xh = rng.random((5000, 16))  # enough rows for the tensor-core lookup
    W16 = wl.Workload("d16", Xh, np.sin(Xh.sum(1, keepdims=True)), Xh[:5], Xh[:5, :1], 16,
                      wl.KernelSpec("rbf", 0.0, 0.4, 1.0, 1e-3), np.arange(5))
    c = _fit(W16, 16, fb.PREC_FP64)
    return [a, b, c]


def _requests(models, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        j = int(rng.integers(len(models)))
        size = int(np.exp(rng.uniform(0, np.log(3000))))
        out.append((j, rng.random((size, models[j].d))))
    return out


def test_server_results_same_alone_and_in_the_mix(cuda):
    models = _models()
    reqs = _requests(models, 36, 5)
    # alone: one stream, each request waited for before the next is submitted
    srv = fb.FmgpServer(models, streams=1)
    alone = []
    for j, Z in reqs:
        rid = srv.submit(j, Z, with_nearest=True)
        assert srv.wait(rid, 60_000)
        Y, N = srv.result(rid)
        alone.append((Y.copy(), N.copy()))
    srv.close()
    # mix: four streams, everything submitted at once from two threads
    srv = fb.FmgpServer(models, streams=4)
    ids = [None] * len(reqs)

    def submit(lo, hi):
        for q in range(lo, hi):
            ids[q] = srv.submit(reqs[q][0], reqs[q][1], with_nearest=True)
    ts = [threading.Thread(target=submit, args=(0, 18)), threading.Thread(target=submit, args=(18, 36))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for q, rid in enumerate(ids):
        assert srv.wait(rid, 60_000)
        Y, N = srv.result(rid)
        assert np.array_equal(Y, alone[q][0]), q
        assert np.array_equal(N, alone[q][1]), q
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["mean_batch_requests"] > 1.0  # requests were batched together
    srv.close()
    # and both equal a direct prediction through the model
    for q, (j, Z) in enumerate(reqs[:6]):
        y, n = models[j].predict(dev(Z))
        assert np.array_equal(y.cpu().numpy(), alone[q][0])


def test_server_admission_by_memory(cuda):
    md = _fit(wl.tiny(n=4000, m=10), 30, fb.PREC_FP64)
    per_req = 1000 * (2 * 8 + 8 + 4) + 3 * 256
    srv = fb.FmgpServer([md], device_budget_bytes=2 * per_req + 100, host_staging_bytes=1 << 22,
                        streams=4)
    rng = np.random.default_rng(1)
    ids = [srv.submit(0, rng.random((1000, 2))) for _ in range(20)]
    qs = []
    for rid in ids:
        assert srv.wait(rid, 60_000)
        qs.append(srv.times(rid)[0])
    assert max(qs) > 0.0
    with pytest.raises(fb.FmgpError) as e:
        srv.submit(0, rng.random((10_000, 2)))
    assert e.value.code == fb.FMGP_ENOMEM
    assert srv.stats()["rejected"] == 1
    srv.close()
    md.close()


def test_split_requests_same_as_whole(cuda):
    """With pieces of 700 points, requests of up to 3,000 points are split
    and their pieces batched and overlapped with other requests on four
    streams; every result equals the unsplit one-stream result bit for bit."""
    models = _models()
    reqs = _requests(models, 30, 8)
    whole = fb.FmgpServer(models, streams=1)
    ref = []
    for j, Z in reqs:
        rid = whole.submit(j, Z, with_nearest=True)
        assert whole.wait(rid, 60_000)
        Y, N = whole.result(rid)
        ref.append((Y.copy(), N.copy()))
    whole.close()
    srv = fb.FmgpServer(models, streams=4, max_batch_points=700)
    ids = [srv.submit(j, Z, with_nearest=True) for j, Z in reqs]
    for q, rid in enumerate(ids):
        assert srv.wait(rid, 60_000)
        Y, N = srv.result(rid)
        assert np.array_equal(Y, ref[q][0]) and np.array_equal(N, ref[q][1]), q
    st = srv.stats()
    pieces = st["batches"] * st["mean_batch_requests"]
    assert round(pieces) == sum(-(-Z.shape[0] // 700) for _, Z in reqs) > len(reqs)
    srv.close()


def test_served_mixed_model_matches_the_oracle(cuda):
    """A mixed-precision model served through the batching server, checked
    directly against the FP64 oracle (its own neighbour rows, coefficients and
    nearest points) within the mixed path's tolerance."""
    import oracle
    from gpu_helpers import MIXED_TOL, rel_rms
    W = wl.tiny(n=3000, m=600, k=30)
    ok, _ = kern_pair(W.kernel)
    md = _fit(W, 30, fb.PREC_MIXED)
    srv = fb.FmgpServer([md], streams=3, max_batch_points=128)
    parts = np.array_split(np.arange(W.m), 7)
    ids = [srv.submit(0, W.Z[p], with_nearest=True) for p in parts]
    got_y, got_n = np.zeros((W.m, 1)), np.zeros(W.m, np.int32)
    for p, rid in zip(parts, ids):
        assert srv.wait(rid, 60_000)
        Y, N = srv.result(rid)
        got_y[p], got_n[p] = Y, N
    srv.close()
    ref_nb, _ = oracle.self_knn(W.X, 29)
    Cr, _ = oracle.precompute(W.X, W.Y, ref_nb, 30, ok)
    yr, nr = oracle.predict(W.X, ref_nb, Cr, ok, W.Z)
    np.testing.assert_array_equal(got_n, nr)
    assert rel_rms(got_y, yr) < MIXED_TOL
    md.close()
