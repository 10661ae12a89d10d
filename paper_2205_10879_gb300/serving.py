"""Serving harness: fit resident models through the C ABI and drive the
continuous-batching server with a Poisson request stream, reporting
predictions/s and per-request latency percentiles."""
import threading
import time

import numpy as np
import torch

from . import _binding as fb


def fit_model(X, Y, k, kernel_spec, precision, device="cuda", timings=None):
    """kNN table + precompute + resident model for one training set.  With a
    dict `timings`, the kNN table, precompute and model creation times (ms,
    CUDA events on the current stream) are stored in it."""
    s = kernel_spec
    gk = fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(device)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).to(device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    nbr, _ = fb.fmgp_build_knn(Xd, max(k - 1, 1))
    ev[1].record()
    C, _ = fb.fmgp_precompute(Xd, Yd, nbr, k, gk, precision, with_status=False)
    ev[2].record()
    model = fb.FmgpModel(Xd, nbr, C, k, gk, precision)
    ev[3].record()
    if timings is not None:
        torch.cuda.synchronize()
        timings.update(knn_ms=ev[0].elapsed_time(ev[1]), precompute_ms=ev[1].elapsed_time(ev[2]),
                       model_ms=ev[2].elapsed_time(ev[3]))
    return model


def run_poisson(server, models, rate_hz, count, seed, max_points=65_536):
    """Submit `count` requests with exponential inter-arrival times at
    `rate_hz`; sizes log-uniform in [1, max_points], points uniform in the
    unit cube of the model's dimension.  Returns per-request latencies (ms),
    total points, the wall time from first submission to last completion and
    the per-request sizes."""
    rng = np.random.default_rng(seed)
    plan = []
    for _ in range(count):
        j = int(rng.integers(len(models)))
        size = max(1, int(np.exp(rng.uniform(0.0, np.log(max_points)))))
        plan.append((j, rng.random((size, models[j].d))))
    gaps = rng.exponential(1.0 / rate_hz, size=count) if rate_hz > 0 else np.zeros(count)
    ids = []
    t0 = time.perf_counter()
    nxt = t0
    for (j, Z), g in zip(plan, gaps):
        nxt += g
        while True:
            now = time.perf_counter()
            if now >= nxt:
                break
            time.sleep(min(nxt - now, 0.0005))
        ids.append(server.submit(j, Z))
    lat = []
    for rid in ids:
        server.wait(rid, -1)
        lat.append(server.times(rid)[1])
    wall = time.perf_counter() - t0
    for rid in ids:
        server.release(rid)
    pts = sum(Z.shape[0] for _, Z in plan)
    return np.array(lat), pts, wall, np.array([Z.shape[0] for _, Z in plan])


SIZE_BUCKETS = ((1, 255), (256, 4095), (4096, 65536))


def latency_summary(lat, pts, wall, sizes=None):
    """p50 / p99 / mean latency and throughput; with the request sizes, the
    same percentiles per size bucket (1-255, 256-4095, 4096-65536 points)."""
    out = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "requests": int(len(lat)),
           "predictions_per_s": pts / wall, "points": int(pts), "wall_s": wall}
    if sizes is not None:
        by = {}
        for lo, hi in SIZE_BUCKETS:
            sel = (sizes >= lo) & (sizes <= hi)
            if sel.any():
                by[f"{lo}-{hi}"] = {"p50_ms": float(np.percentile(lat[sel], 50)),
                                    "p99_ms": float(np.percentile(lat[sel], 99)),
                                    "requests": int(sel.sum())}
        out["by_size"] = by
    return out
