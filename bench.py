"""FastMuyGPs posterior-mean benchmark on GB300.

One step = the whole hot path over one batch of the spatial 2-D workload
(n = 150,000 training + m = 50,000 test points uniform in [0,1]^2, 20 random
Fourier features + N(0, 0.05^2), Matern nu = 1.5, rho = 0.1, tau^2 = 1e-3,
k = 50): self-kNN table (A1), kernel assembly + Cholesky + solve for every
training point (A2-A3), nearest-training-point lookup (A4), gather-dot
prediction (A5) and the LOOCV objective over a batch of b = 10,000 (A6).

value = (n + m) / step time [points/s]; per-phase rates (precompute pts/s,
predictions/s, kNN queries/s, LOOCV pts/s) and the plain FP64 path's numbers
are reported beside it.  Inputs are resident in HBM before timing; L2 (129 MB)
is flushed between timed steps by writing a 512 MB buffer.  e2e repeats the
step from pinned host buffers with the copies inside the timed region.

--workload selects another configuration: tiny (n = 2,000, m = 500, k = 30,
Matern 3/2, the oracle's sanity case), large (n = 10^7, m = 10^6, d = 3, k = 64,
Matern 5/2, nugget 1e-5), highdim (the 784-D ten-response leg alone),
highdim-knn (its kNN table alone) or nearest-d64 (tensor-core nearest-point
lookup).

--impl reference times the FP64 CPU oracle (OpenMP, all host cores): one
whole pass over the workload per step (for the 10^7-point workload a bounded
sample of rows, extrapolated per point).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "predictions/s + precompute pts/s vs FP64 plain at equal RMSE; p50/p99 latency"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="auto", choices=["auto", "mixed", "fp64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--serving-requests", type=int, default=300)
    p.add_argument("--serving-piece", type=int, default=8192,
                   help="test points per piece of a request / per launched batch")
    p.add_argument("--n", type=int, default=150_000)
    p.add_argument("--m", type=int, default=50_000)
    p.add_argument("--k", type=int, default=50)
    p.add_argument("--b", type=int, default=10_000)
    p.add_argument("--nu", type=float, default=1.5)
    p.add_argument("--workload", default="spatial", choices=["spatial", "tiny", "large", "highdim", "highdim-knn", "nearest-d64"])
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-muygps", action="store_true")
    p.add_argument("--no-highdim", action="store_true")
    p.add_argument("--no-borehole", action="store_true")
    p.add_argument("--no-subsample", action="store_true")
    p.add_argument("--no-graph", action="store_true")
    p.add_argument("--no-training", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--tune", action="append", default=[], metavar="KEY=VALUE",
                   help="library tuning key set before the run (fmgp_tune_set), repeatable")
    p.add_argument("--mcmc-chains", type=int, default=8192)
    p.add_argument("--mcmc-steps", type=int, default=1221)
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device=None):
    """Max of a per-rank float over all ranks (identity without a process
    group).  NCCL needs a CUDA tensor, gloo a CPU one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(a):
    if a.workload == "tiny":
        return {"workload": "tiny-2d", "n_train": 2_000, "m_test": 500, "d": 2, "k": 30, "r": 1,
                "kernel": "matern nu=1.5 rho=0.1 tau2=1e-4", "loocv_batch": 500,
                "l2": "flushed between steps (512 MB write)"}
    if a.workload == "large":
        return {"workload": "large-3d", "n_train": 10_000_000, "m_test": 1_000_000, "d": 3,
                "k": 64, "r": 1, "kernel": "matern nu=2.5 rho=0.1 tau2=1e-5", "loocv_batch": 10_000,
                "l2": "inputs larger than L2 (129 MB)"}
    return {"workload": "spatial-2d", "n_train": a.n, "m_test": a.m, "d": 2, "k": a.k,
            "r": 1, "kernel": f"matern nu={a.nu} rho=0.1 tau2=1e-3", "loocv_batch": a.b,
            "l2": "flushed between steps (512 MB write)"}


def make_workload(a):
    from paper_2205_10879_gb300 import workloads as wl
    if a.workload == "large":
        return wl.large()
    if a.workload == "tiny":
        return wl.tiny(n=2_000, m=500, k=30, b=500)
    return wl.spatial(n=a.n, m=a.m, k=a.k, nu=a.nu, b=a.b)


# ------------------------------------------------------- ncu evidence ----
# Per-launch DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) and
# pipe utilisation from one ncu capture of the kernel (summary and command in
# the named profile).  They are reported only while the kernel's sources still
# hash to the values captured; any change turns them into null.
NCU_EVIDENCE = {
    "block_mixed_kernel": {
        "traffic": 33702912 + 8795392,
        "issue_active_pct": 69.2, "fma_pipe_pct": 35.6, "alu_pipe_pct": 41.5,
        "profile": "profiles/block_mixed_kernel_spatial.md",
        "sources": {"paper_2205_10879_gb300/csrc/mixed.cu": "7d26d3abee645b68",
                    "paper_2205_10879_gb300/csrc/df.cuh": "859745e469e825d6",
                    "paper_2205_10879_gb300/csrc/block.cuh": "698a2212b42899b6"},
    },
}


def ncu_evidence(kernel):
    import hashlib
    ev = NCU_EVIDENCE.get(kernel)
    if not ev:
        return None
    for path, h in ev["sources"].items():
        try:
            with open(os.path.join(ROOT, path), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest()[:16] != h:
                    return None
        except OSError:
            return None
    return ev


# ----------------------------------------------------------------- peaks --
def measured_peaks():
    """The machine's measured HBM copy bandwidth and cuBLAS BF16 rates
    (MEASURED_PEAKS.json beside this file), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def bf16_peak():
    """Dense BF16 tensor peak in TFLOP/s for a kernel timed alone: the measured
    burst figure, else 1900 (an earlier GB300 measurement)."""
    p = measured_peaks()
    return float(p["bf16_tflops"]) if p and p.get("bf16_tflops") else 1900.0


def bf16_peak_source():
    p = measured_peaks()
    return "measured (bf16_tflops, burst)" if p and p.get("bf16_tflops") else "fallback"


def alu_peak(fb, dev, pipe, sm_mhz=None):
    """FMA-pipe peak in TFLOP/s measured in this run by the library's probe
    kernel (fmgp_peak_probe), with the unit-count figure at the sampled clock
    beside it."""
    import torch
    v = fb.peak_probe(pipe) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    per_clk = 256 if pipe == "fp32" else 4  # flops per SM per clock: 128 FFMA / 2 DFMA
    mhz = sm_mhz or 2070.0
    return v, {"peak_source": f"measured in this run: fmgp_peak_probe ({pipe} FMA, best of 3 "
                              f"launches of ~30 ms)",
               "peak_unit_count": sms * per_clk * mhz * 1e6 / 1e12,
               "peak_unit_count_note": f"{sms} SMs x {per_clk // 2} FMA/clk x 2 x {mhz:.0f} MHz"}


# ----------------------------------------------------------------- flops --
def precompute_flops_per_point(k, d, r):
    """Algorithmic FP operations of one neighbourhood (A2 + A3): k(k-1)/2 kernel
    entries at 3d (distance) + 6 (scale, sqrt, exp, polynomial; transcendentals
    counted once), Cholesky k^3/3, two triangular solves 2 k^2 r."""
    return k * (k - 1) / 2 * (3 * d + 6) + k ** 3 / 3 + 2 * k * k * r


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during timing."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ our arm ----
def run_ours(a):
    import torch
    from paper_2205_10879_gb300 import _binding as fb
    from paper_2205_10879_gb300 import workloads as wl

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    fb.load()
    for kv in a.tune:
        key, val = kv.split("=", 1)
        fb.tune_set(key, float(val))
    W = make_workload(a)
    s = W.kernel
    gk = fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)
    k, kq = W.k, W.k  # one table serves precompute (k-1 columns) and LOOCV (k columns)
    X = torch.from_numpy(W.X).to(dev)
    Y = torch.from_numpy(W.Y).to(dev)
    Z = torch.from_numpy(W.Z).to(dev)
    batch = torch.from_numpy(W.batch).to(dev)
    n, m, b = W.n, W.m, W.b if hasattr(W, "b") else len(W.batch)
    b = len(W.batch)

    def pick_precision():
        if a.precision == "fp64":
            return fb.PREC_FP64
        if a.precision == "mixed":
            return fb.PREC_MIXED
        try:  # auto: the mixed form when this build has it
            nb, _ = fb.fmgp_build_knn(X[:1000].contiguous(), 8)
            fb.fmgp_precompute(X[:1000].contiguous(), Y[:1000].contiguous(), nb, 9, gk,
                               fb.PREC_MIXED)
            return fb.PREC_MIXED
        except fb.FmgpError:
            return fb.PREC_FP64

    prec = pick_precision()
    nbr = torch.empty((n, kq), dtype=torch.int32, device=dev)
    # launch shapes picked by the library's autotuner on this workload before
    # timing (results do not depend on them)
    tuned = None
    if not a.no_autotune:
        fb.fmgp_build_knn(X, kq, nbr_out=nbr)
        gt = fb.fmgp_autotune_knn(X, kq)
        fb.fmgp_autotune_precompute(X, Y, nbr, k, gk, prec, sample_rows=min(n, 200_000))
        w, pw, pers = fb.autotune_choice(k, W.d, 1, prec, X.dtype)
        tuned = {"grid_target": gt if gt > 0 else None, "block_warps": w,
                 "cholesky_panel": pw or None, "persistent": pers,
                 "sample_rows": min(n, 200_000)}
    C = torch.empty(fb.coeff_shape(n, k, 1, prec),
                    dtype=torch.float64 if prec == fb.PREC_FP64 else torch.float32, device=dev)
    st = torch.empty(n, dtype=torch.int8, device=dev)
    yh = torch.empty((m, 1), dtype=torch.float64, device=dev)
    near = torch.empty(m, dtype=torch.int32, device=dev)
    resid = torch.empty(b, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    Qd = torch.empty(1, dtype=torch.float64, device=dev)
    fails_d = torch.zeros(1, dtype=torch.int32, device=dev)

    def step(p, C_, ev=None):
        if ev: ev[0].record(stream)
        fb.fmgp_build_knn(X, kq, nbr_out=nbr)
        if ev: ev[1].record(stream)
        fb.fmgp_precompute(X, Y, nbr, k, gk, p, C_out=C_, status_out=st)
        if ev: ev[2].record(stream)
        fb.fmgp_predict(X, nbr, C_, k, gk, Z, p, Yhat_out=yh, nearest_out=near)
        if ev: ev[3].record(stream)
        # Eq. 5 objective left in device memory: no host round trip inside the
        # device-timed step (the e2e leg reads its results back every step);
        # checked against the host-returning entry point after timing
        fb.fmgp_loocv_objective_device(X, Y, nbr, k, batch, gk, p, Q_out=Qd, fails_out=fails_d,
                                       resid_out=resid)
        if ev: ev[4].record(stream)

    def timed(p, C_, steps, warmup):
        for _ in range(warmup):
            step(p, C_)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = fb.kernel_launches()
        for i in range(steps):
            flush.zero_()
            step(p, C_, evs[i])
        torch.cuda.synchronize()
        launches = (fb.kernel_launches() - l0) / steps
        ph = np.array([[evs[i][j].elapsed_time(evs[i][j + 1]) for j in range(4)]
                       for i in range(steps)])
        return ph, launches

    clk = ClockSampler(local)
    clk.start()
    ph, launches = timed(prec, C, a.steps, a.warmup)
    clocks = clk.stop()
    step_ms = ph.sum(axis=1)
    ms = float(step_ms.mean())
    ms = max_over_ranks(ms, dev)
    phase_ms = ph.mean(axis=0)
    yh_main = yh.cpu().numpy().copy()
    st_main = st.cpu().numpy().copy()
    # the device-side objective of the timed steps against the host-returning call
    q_dev, q_fails = float(Qd.item()), int(fails_d.item())
    q_host, _ = fb.fmgp_loocv_objective(X, Y, nbr, k, batch, gk, prec, resid_out=resid)
    loocv_check = {"Q": q_host, "device_Q_equal": q_dev == q_host, "failed_blocks": q_fails}
    rmse = float(np.sqrt(np.mean((yh_main - W.Ztrue) ** 2)))
    out = {}
    # the plain FP64 path on the same workload, for the "vs FP64 plain" comparison
    fp64 = None
    if prec != fb.PREC_FP64 and not a.no_fp64:
        C64 = torch.empty((n, k, 1), dtype=torch.float64, device=dev)
        ph64, _ = timed(fb.PREC_FP64, C64, max(2, a.steps // 2), 1)
        y64 = yh.cpu().numpy().copy()
        p64 = ph64.mean(axis=0)
        fp64 = {"ms_per_step": float(ph64.sum(axis=1).mean()),
                "precompute_pts_per_s": n / (p64[1] * 1e-3),
                "predictions_per_s": m / (p64[2] * 1e-3),
                "rmse": float(np.sqrt(np.mean((y64 - W.Ztrue) ** 2))),
                "rel_rms_vs_fp64": float(np.linalg.norm(yh_main - y64) / np.linalg.norm(y64))}
        r64 = fp64["rmse"]
        fp64["rmse_rel_diff"] = abs(rmse - r64) / r64
        fp64["equal_rmse"] = bool(abs(rmse - r64) <= 1e-3 * r64)
        del C64
    # the paper's comparator on the same test points: plain MuyGPs prediction
    # (each test point's own k neighbours and one Cholesky per test point)
    muy = None
    if not a.no_muygps:
        ymu = torch.empty((m, 1), dtype=torch.float64, device=dev)
        fb.fmgp_muygps_predict(X, Y, Z, k, gk, prec, Yhat_out=ymu)
        torch.cuda.synchronize()
        tm = []
        for _ in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fb.fmgp_muygps_predict(X, Y, Z, k, gk, prec, Yhat_out=ymu)
            e1.record()
            torch.cuda.synchronize()
            tm.append(e0.elapsed_time(e1))
        mu_ms = float(np.mean(tm))
        yv = ymu.cpu().numpy()
        muy = {"ms": mu_ms, "predictions_per_s": m / (mu_ms * 1e-3),
               "rmse": float(np.sqrt(np.mean((yv - W.Ztrue) ** 2))),
               "fastmuygps_speedup_predict": mu_ms / phase_ms[2]}
    # roofline of the dominant kernel (the precompute block kernel: one launch per step)
    fl = precompute_flops_per_point(k, W.d, 1) * n
    pre_s = phase_ms[1] * 1e-3
    if prec == fb.PREC_FP64:
        roof = {"bound": "alu", "pipe": "fp64", "kernel": "block_f64_kernel"}
    else:
        roof = {"bound": "alu", "pipe": "fp32", "kernel": "block_mixed_kernel"}
    peak, psrc = alu_peak(fb, dev, roof["pipe"], clocks["sm_mhz"] if clocks else None)
    other = "fp64" if roof["pipe"] == "fp32" else "fp32"
    alu_peaks = {roof["pipe"] + "_tflops": peak,
                 other + "_tflops": alu_peak(fb, dev, other)[0],
                 "source": "fmgp_peak_probe in this run (FMA chains on every SM, best of 3)"}
    achieved = fl / pre_s / 1e12
    ev = ncu_evidence(roof["kernel"]) if a.workload == "spatial" else None
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": ev["traffic"] if ev else None, "flops_per_launch": fl,
                 "ncu": ({k: ev[k] for k in ("issue_active_pct", "fma_pipe_pct", "alu_pipe_pct",
                                              "profile")} if ev else None)})
    roof.update(psrc)
    # e2e: same step from pinned host buffers, copies inside the timed region
    e2e = None
    if not a.no_e2e:
        hX = torch.from_numpy(W.X).pin_memory()
        hY = torch.from_numpy(W.Y).pin_memory()
        hZ = torch.from_numpy(W.Z).pin_memory()
        hB = torch.from_numpy(W.batch).pin_memory()
        hOut = torch.empty((m, 1), dtype=torch.float64).pin_memory()
        dX, dY, dZ, dB = (torch.empty_like(t, device=dev) for t in (hX, hY, hZ, hB))

        def e2e_step():
            dX.copy_(hX, non_blocking=True)
            dY.copy_(hY, non_blocking=True)
            dZ.copy_(hZ, non_blocking=True)
            dB.copy_(hB, non_blocking=True)
            fb.fmgp_build_knn(dX, kq, nbr_out=nbr)
            fb.fmgp_precompute(dX, dY, nbr, k, gk, prec, C_out=C, status_out=st)
            fb.fmgp_predict(dX, nbr, C, k, gk, dZ, prec, Yhat_out=yh, nearest_out=near)
            Q, _ = fb.fmgp_loocv_objective(dX, dY, nbr, k, dB, gk, prec, resid_out=resid)
            hOut.copy_(yh, non_blocking=True)
            return Q
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        t_e = []
        for _ in range(a.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e2e_step()
            e1.record(stream)
            torch.cuda.synchronize()
            t_e.append(e0.elapsed_time(e1))
        e_ms = float(np.mean(t_e))
        e2e = {"value": (n + m) / (e_ms * 1e-3) * ws, "unit": "points/s",
               "ms_per_step": e_ms,
               "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in (hX, hY, hZ, hB))),
               "d2h_bytes_per_step": int(hOut.numel() * hOut.element_size() + 8)}
    # kNN work per query (untimed call with the grid search's counters on)
    knn_visits = None
    if W.X.shape[1] <= 3:
        fb.tune_set("count_visits", 1)
        try:
            fb.fmgp_build_knn(X, kq, nbr_out=nbr)
            torch.cuda.synchronize()
            nq = fb.diag_counter(5)
            if nq > 0:
                knn_visits = {"candidates_examined_per_query": fb.diag_counter(3) / nq,
                              "fp64_keys_per_query": fb.diag_counter(4) / nq, "kq": kq}
        finally:
            fb.tune_set("count_visits", 0)
    line = {
        "metric": METRIC, "value": (n + m) / (ms * 1e-3) * ws, "unit": "points/s",
        "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == fb.PREC_FP64 else "f32+df64",
        "precision": "fp64" if prec == fb.PREC_FP64 else "mixed",
        "data": "synthetic", "config": workload_config(a),
        "phases_ms": {"knn": phase_ms[0], "precompute": phase_ms[1], "predict": phase_ms[2],
                      "loocv": phase_ms[3]},
        "loocv_objective": loocv_check,
        "precompute_pts_per_s": n / (phase_ms[1] * 1e-3),
        "precompute_with_knn_pts_per_s": n / ((phase_ms[0] + phase_ms[1]) * 1e-3),
        "predictions_per_s": m / (phase_ms[2] * 1e-3),
        "knn_queries_per_s": n / (phase_ms[0] * 1e-3), "knn_work": knn_visits,
        "loocv_pts_per_s": b / (phase_ms[3] * 1e-3),
        "rmse": rmse, "fp64_path": fp64, "muygps_predict": muy, "roofline": roof, "e2e": e2e,
        "block_status": {str(v): int(c) for v, c in zip(*np.unique(st_main, return_counts=True))},
        "gpu_launches": launches, "clocks": clocks, "autotuned": tuned, "alu_peaks": alu_peaks,
    }
    if not a.no_highdim:
        line["highdim"] = highdim_bench(a, dev)
    if not a.no_training and a.workload == "spatial":
        line["training"] = training_bench(X, Y, batch, k, nbr, gk, prec)
    if not a.no_graph and a.workload == "spatial":
        line["cuda_graph"] = graph_bench(X, Y, Z, batch, k, kq, gk, prec, nbr, C, st, yh, near)
    if not a.no_subsample and a.workload == "spatial":
        line["subsampled"] = subsample_bench(W, X, Y, Z, nbr, k, gk, prec, rmse, dev)
    if not a.no_borehole:
        line["borehole"] = borehole_bench(a, dev)
    if not a.no_serving:
        line["serving"] = serving_bench(a, dev)
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(W, a)
        yo = line["cpu_baseline"].pop("_predictions", None)
        if yo is not None:  # the oracle predicted every test point: end-to-end parity
            line["rel_rms_vs_oracle"] = float(np.linalg.norm(yh_main - yo) / np.linalg.norm(yo))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------- high-d kNN (A1) ----
def highdim_knn_bench(a, dev, steps, warmup):
    """A1 on the 784-D workload: self kNN table (kq = 29) of n = 60,000 FP32
    points (80% exact zeros), through the tensor-core candidate search with
    certified exact re-rank.  Tensor roofline: 2 * n_pad * n_pad * d_pad BF16
    flops of the distance GEMM over the whole call's time (an upper bound on
    the GEMM kernel's own time)."""
    import torch
    from paper_2205_10879_gb300 import _binding as fb
    from paper_2205_10879_gb300 import workloads as wl
    W = wl.highdim()
    X = torch.from_numpy(W.X).to(dev)
    nbr = torch.empty((W.n, 29), dtype=torch.int32, device=dev)
    for _ in range(warmup):
        fb.fmgp_build_knn(X, 29, nbr_out=nbr)
    torch.cuda.synchronize()
    ts = []
    c0 = fb.diag_counter(1)
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fb.fmgp_build_knn(X, 29, nbr_out=nbr)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    n_pad = (W.n + 255) // 256 * 256
    d_pad = (W.d + 63) // 64 * 64
    flops = 2.0 * n_pad * n_pad * d_pad
    peak = bf16_peak()
    ach = flops / (ms * 1e-3) / 1e12
    return {"workload": "highdim-784 self kNN", "n": W.n, "d": W.d, "kq": 29, "ms": ms,
            "knn_queries_per_s": W.n / (ms * 1e-3), "tensor_core_calls": fb.diag_counter(1) - c0,
            "uncertified_queries": fb.diag_counter(2),
            "roofline_call": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                              "frac": ach / peak, "note": "whole call incl. pack/select/re-rank"}}


def highdim_bench(a, dev, steps=2):
    """The high-dimensional multi-response configuration end to end (the
    stand-in for the 400-D star-galaxy images of Sec. 4.3): n = 60,000
    training and m = 10,000 test points, d = 784 FP32 features with 80% exact
    zeros, r = 10 centred one-hot responses, RBF rho = 7, tau^2 = 1e-2,
    k = 30, LOOCV batch of 5,000.  Per precision: kNN table (tensor cores,
    kq = 30), precompute, prediction (nearest point + gather-dot) and LOOCV,
    each timed with CUDA events; RMSE against the held-out centred one-hot
    responses, classification accuracy (argmax of the predicted responses
    plus the column means, as Table 2 reports), and the mixed form's
    difference from the FP64 form."""
    import torch
    from paper_2205_10879_gb300 import _binding as fb
    from paper_2205_10879_gb300 import workloads as wl
    W = wl.highdim()
    s = W.kernel
    gk = fb.make_kernel(s.kind, s.nu, s.length_scale, s.variance, s.nugget)
    X, Y, Z = (torch.from_numpy(v).to(dev) for v in (W.X, W.Y, W.Z))
    batch = torch.from_numpy(W.batch).to(dev)
    k = kq = W.k
    mu = W.extra["col_mean"]
    labels = W.extra["labels_test"]
    nbr = torch.empty((W.n, kq), dtype=torch.int32, device=dev)
    yh = torch.empty((W.m, W.r), dtype=torch.float64, device=dev)
    near = torch.empty(W.m, dtype=torch.int32, device=dev)
    resid = torch.empty(len(W.batch), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    out = {"workload": "highdim-784: n=60000 m=10000 d=784 (80% zeros, FP32) r=10 rbf rho=7 "
                       "tau2=1e-2 k=30", "n": W.n, "m": W.m, "d": W.d, "r": W.r, "k": k,
           "loocv_batch": len(W.batch)}
    preds = {}
    for name, prec in (("mixed", fb.PREC_MIXED), ("fp64", fb.PREC_FP64)):
        C = torch.empty(fb.coeff_shape(W.n, k, W.r, prec),
                        dtype=torch.float64 if prec == fb.PREC_FP64 else torch.float32, device=dev)
        st = torch.empty(W.n, dtype=torch.int8, device=dev)

        def step(ev=None):
            if ev: ev[0].record(stream)
            fb.fmgp_build_knn(X, kq, nbr_out=nbr)
            if ev: ev[1].record(stream)
            fb.fmgp_precompute(X, Y, nbr, k, gk, prec, C_out=C, status_out=st)
            if ev: ev[2].record(stream)
            fb.fmgp_predict(X, nbr, C, k, gk, Z, prec, Yhat_out=yh, nearest_out=near)
            if ev: ev[3].record(stream)
            Q, _ = fb.fmgp_loocv_objective(X, Y, nbr, k, batch, gk, prec, resid_out=resid)
            if ev: ev[4].record(stream)
            return Q
        step()
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        for i in range(steps):
            Q = step(evs[i])
        torch.cuda.synchronize()
        ph = np.array([[evs[i][j].elapsed_time(evs[i][j + 1]) for j in range(4)]
                       for i in range(steps)]).mean(axis=0)
        y = yh.cpu().numpy().copy()
        preds[name] = y
        stv = st.cpu().numpy()
        out[name] = {"phases_ms": {"knn": ph[0], "precompute": ph[1], "predict": ph[2],
                                   "loocv": ph[3]},
                     "ms_per_step": float(ph.sum()),
                     "knn_queries_per_s": W.n / (ph[0] * 1e-3),
                     "precompute_pts_per_s": W.n / (ph[1] * 1e-3),
                     "predictions_per_s": W.m / (ph[2] * 1e-3),
                     "loocv_pts_per_s": len(W.batch) / (ph[3] * 1e-3),
                     "rmse": float(np.sqrt(np.mean((y - W.Ztrue) ** 2))),
                     "accuracy": float(np.mean(np.argmax(y + mu, axis=1) == labels)),
                     "loocv_q": Q,
                     "block_status": {str(v): int(c) for v, c in zip(*np.unique(stv, return_counts=True))}}
        del C, st
    r64 = out["fp64"]["rmse"]
    out["mixed_rel_rms_vs_fp64"] = float(np.linalg.norm(preds["mixed"] - preds["fp64"]) /
                                         np.linalg.norm(preds["fp64"]))
    out["equal_rmse"] = bool(abs(out["mixed"]["rmse"] - r64) <= 1e-3 * r64)
    out["knn"] = highdim_knn_bench(a, dev, steps=max(2, steps), warmup=1)
    return out


def nearest_bench(a, dev, steps, warmup):
    """A4 at d >= 16: the nearest training point of m = 65,536 queries among
    n = 200,000 FP64 points uniform in [0,1]^64 (the largest request and d >= 16
    model size of the serving mix), through fmgp_predict (FP64, k = 32, RBF).
    Tensor roofline: 2 * m_pad * n_pad * d_pad BF16 flops of the distance GEMM
    over the whole call's time."""
    import torch
    from paper_2205_10879_gb300 import _binding as fb
    rng = np.random.default_rng(64)
    n, m, d = 200_000, 65_536, 64
    X = torch.from_numpy(rng.random((n, d))).to(dev)
    Y = torch.from_numpy(np.sin(3.0 * rng.random((n, 1)))).to(dev)
    Z = torch.from_numpy(rng.random((m, d))).to(dev)
    kern = fb.make_kernel("rbf", 0.0, 1.0, 1.0, 1e-2)
    k = 32
    nbr, _ = fb.fmgp_build_knn(X, k - 1)
    C, _ = fb.fmgp_precompute(X, Y, nbr, k, kern, fb.PREC_FP64, with_status=False)
    yhat = torch.empty((m, 1), dtype=torch.float64, device=dev)
    near = torch.empty(m, dtype=torch.int32, device=dev)
    for _ in range(warmup):
        fb.fmgp_predict(X, nbr, C, k, kern, Z, Yhat_out=yhat, nearest_out=near)
    torch.cuda.synchronize()
    ts = []
    c0 = fb.diag_counter(1)
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fb.fmgp_predict(X, nbr, C, k, kern, Z, Yhat_out=yhat, nearest_out=near)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    flops = 2.0 * ((m + 127) // 128 * 128) * ((n + 255) // 256 * 256) * 64
    peak = bf16_peak()
    ach = flops / (ms * 1e-3) / 1e12
    return {"workload": "nearest-d64: nearest of 65,536 queries among 200,000 points, d = 64",
            "n": n, "m": m, "d": d, "k": k, "ms": ms, "predictions_per_s": m / (ms * 1e-3),
            "tensor_core_calls": fb.diag_counter(1) - c0,
            "uncertified_queries": fb.diag_counter(2),
            "roofline_call": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                              "frac": ach / peak,
                              "note": "whole call incl. pack/select/re-rank/gather-dot"}}


# -------------------------------------------------------------- training ----
def training_bench(X, Y, batch, k, nbr, gk, prec):
    """Hyperparameter training (Algorithm 1): L-BFGS-B on log rho over the
    LOOCV objective of the step's batch (each evaluation on the GPU), started
    from half the workload's length scale."""
    import torch
    from paper_2205_10879_gb300 import _binding as fb
    from paper_2205_10879_gb300 import training
    start = fb.Kernel(gk.kind, gk.nu, gk.length_scale * 0.5, gk.variance, gk.nugget)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = training.optimize_hyperparameters(X, Y, batch, k, start, params=("length_scale",),
                                            precision=prec, nbr=nbr)
    wall = time.perf_counter() - t0
    return {"params": "length_scale", "start": start.length_scale,
            "found": res["theta"]["length_scale"], "workload_value": gk.length_scale,
            "q_start": res["q_start"], "q_best": res["q_best"], "evaluations": res["evaluations"],
            "seconds": wall, "evaluations_per_s": res["evaluations"] / wall,
            "batch": int(batch.numel()), "k": k}


# ------------------------------------------------------------ CUDA graph ----
def graph_bench(X, Y, Z, batch, k, kq, gk, prec, nbr, C, st, yh, near, reps=5):
    """The whole step (kNN table, precompute, prediction and the LOOCV
    objective written to device memory) captured once in a CUDA graph and
    replayed, against the same four calls launched eagerly."""
    import torch
    from paper_2205_10879_gb300 import _binding as fb
    Q = torch.empty(1, dtype=torch.float64, device=X.device)
    res = torch.empty(batch.numel(), dtype=torch.float64, device=X.device)

    def three():
        fb.fmgp_build_knn(X, kq, nbr_out=nbr)
        fb.fmgp_precompute(X, Y, nbr, k, gk, prec, C_out=C, status_out=st)
        fb.fmgp_predict(X, nbr, C, k, gk, Z, prec, Yhat_out=yh, nearest_out=near)
        fb.fmgp_loocv_objective_device(X, Y, nbr, k, batch, gk, prec, Q_out=Q, resid_out=res)

    def timed(f):
        f()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    eager_ms = timed(three)
    ref = yh.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        three()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    l0 = fb.kernel_launches()
    with torch.cuda.graph(g):
        three()
    launches = fb.kernel_launches() - l0
    graph_ms = timed(g.replay)
    same = bool(torch.equal(yh, ref))
    del g
    return {"phases": "knn + precompute + predict + loocv", "eager_ms": eager_ms, "graph_replay_ms": graph_ms,
            "kernels_in_graph": int(launches), "replay_equals_eager": same}


# ------------------------------------------------ subsampled precompute ----
def subsample_bench(W, X, Y, Z, nbr, k, gk, prec, rmse_full, dev):
    """The subsampling of precomputed coefficients proposed in Sec. 5, on the
    step's workload and precision: C for a random fraction of the training
    points (the centres), prediction from the nearest centre.  Coefficient
    memory, precompute and prediction time, RMSE against the full method's."""
    import torch
    from paper_2205_10879_gb300 import _binding as fb
    out = {"rmse_full": rmse_full, "centres": []}
    for frac in (0.5, 0.25):
        s = int(W.n * frac)
        rows = torch.from_numpy(np.sort(np.random.default_rng(9).choice(W.n, s, replace=False))
                                .astype(np.int32)).to(dev)
        fb.fmgp_precompute_rows(X, Y, nbr, k, gk, rows, prec)
        (C, _), ms_pre = _timed(lambda: fb.fmgp_precompute_rows(X, Y, nbr, k, gk, rows, prec), dev)
        fb.fmgp_predict_rows(X, nbr, rows, C, k, gk, Z, prec)
        (yh, _), ms_pred = _timed(lambda: fb.fmgp_predict_rows(X, nbr, rows, C, k, gk, Z, prec), dev)
        rmse = float(np.sqrt(np.mean((yh.cpu().numpy() - W.Ztrue) ** 2)))
        out["centres"].append({"fraction": frac, "s": s, "coeff_bytes": int(C.numel() * C.element_size()),
                               "precompute_ms": ms_pre, "predict_ms": ms_pred, "rmse": rmse,
                               "rmse_vs_full": rmse / rmse_full})
    return out


# ------------------------------------------------- borehole + MCMC (4.2) ----
def _timed(fn, dev):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def borehole_bench(a, dev):
    """The borehole emulator of Sec. 4.2 (Table 1): n = 100,000 training and
    m = 20,000 test points, 8 inputs (4 varying), RBF rho = 43.27, k = 150,
    FP64 path (the near-flat kernel puts the blocks far beyond FP32's reach).
    Times kNN, precompute, the test-set prediction (the paper's 0.109 s on a
    P100) and plain MuyGPs prediction (its 1.32 s), RMSE against the exact
    flow; then the MCMC calibration of r_w from the flow at r_w = 0.09:
    chains x steps Metropolis samples (10^7 by default) on the device."""
    import torch
    from paper_2205_10879_gb300 import _binding as fb
    from paper_2205_10879_gb300 import workloads as wl
    W = wl.borehole()
    kern = W.kernel
    gk = fb.make_kernel(kern.kind, kern.nu, kern.length_scale, kern.variance, kern.nugget)
    X, Y, Z = (torch.from_numpy(v).to(dev) for v in (W.X, W.Y, W.Z))
    k = W.k
    fb.fmgp_build_knn(X, k - 1)  # warm-up (module load, pools)
    (nbr, _), ms_knn = _timed(lambda: fb.fmgp_build_knn(X, k - 1), dev)
    (C, st), ms_pre = _timed(lambda: fb.fmgp_precompute(X, Y, nbr, k, gk, fb.PREC_FP64), dev)
    fb.fmgp_predict(X, nbr, C, k, gk, Z, fb.PREC_FP64)
    (yh, _), ms_pred = _timed(lambda: fb.fmgp_predict(X, nbr, C, k, gk, Z, fb.PREC_FP64), dev)
    rmse = float(np.sqrt(np.mean((yh.cpu().numpy() - W.Ztrue) ** 2)))
    (ym, _), ms_muy = _timed(lambda: fb.fmgp_muygps_predict(X, Y, Z, k, gk, fb.PREC_FP64), dev)
    rmse_muy = float(np.sqrt(np.mean((ym.cpu().numpy() - W.Ztrue) ** 2)))
    (_, stm), ms_pre_mixed = _timed(lambda: fb.fmgp_precompute(X, Y, nbr, k, gk, fb.PREC_MIXED), dev)
    out = {"workload": "borehole n=100000 m=20000 d=8 k=150 rbf rho=43.27 tau2=1e-8",
           "knn_ms": ms_knn, "precompute_ms": ms_pre, "predict_ms": ms_pred,
           "predictions_per_s": W.m / (ms_pred * 1e-3), "rmse": rmse,
           "paper_predict_s": 0.109, "paper_rmse": 1.12e-2,
           "muygps_predict_ms": ms_muy, "muygps_rmse": rmse_muy, "paper_muygps_predict_s": 1.32,
           "not_spd_blocks": int((st.cpu().numpy() == 1).sum()),
           "mixed_precompute_ms": ms_pre_mixed,
           "mixed_block_status": {str(v): int(c) for v, c in
                                  zip(*np.unique(stm.cpu().numpy(), return_counts=True))}}
    # MCMC calibration of r_w (coordinate 0): prior uniform over its range
    e = W.extra
    model = fb.FmgpModel(X, nbr, C, k, gk, fb.PREC_FP64)
    chains, steps = a.mcmc_chains, a.mcmc_steps
    g = torch.Generator(device=dev)
    g.manual_seed(6006)
    noise = torch.randn((steps, chains), generator=g, dtype=torch.float64, device=dev)
    expo = torch.empty((steps, chains), dtype=torch.float64, device=dev).exponential_(1.0, generator=g)
    x0 = np.random.default_rng(6007).uniform(e["lo"], e["hi"], chains)
    sigma, step = 1.0, 0.3
    w = max(1, min(steps, 8))
    model.mcmc(e["z0"], e["dim"], e["lo"], e["hi"], e["f_obs"], sigma, step, x0, noise[:w].contiguous(),
               expo[:w].contiguous())
    (S, acc, _), ms_mcmc = _timed(lambda: model.mcmc(e["z0"], e["dim"], e["lo"], e["hi"], e["f_obs"],
                                                     sigma, step, x0, noise, expo), dev)
    burn = min(200, steps // 2)
    post = S[burn:] * e["scale"]  # unit-cube coordinate of r_w
    mean_u = float(post.mean())
    out["mcmc"] = {"chains": chains, "steps": steps, "samples": chains * steps, "ms": ms_mcmc,
                   "samples_per_s": chains * steps / (ms_mcmc * 1e-3),
                   "accept_rate": float(acc.sum().item()) / (chains * steps),
                   "posterior_mean_unit": mean_u, "posterior_sd_unit": float(post.std()),
                   "truth_unit": e["u_true"], "rel_error": abs(mean_u - e["u_true"]) / e["u_true"],
                   "paper_posterior_mean_unit": 0.3998, "burn_in_steps": burn,
                   "sigma_obs": sigma, "proposal_sd": step}
    model.close()
    return out


# ------------------------------------------------------------- serving ----
def serving_bench(a, dev):
    """Eight resident models at their full sizes (n log-uniform in [1e4, 2e6],
    d in {2,3,16,64}, k in {16,32,64,128}, Matern/RBF, mixed precision; the
    d >= 16 tables from the tensor-core search), one continuous-batching
    server (4 streams), Poisson request streams of log-uniform 1..65,536
    points at 25%, 50%, 75% and 90% of the measured saturation rate: p50/p99
    latency (submission to results in host memory) and predictions/s.  Each
    model's fit (kNN table, precompute, resident model) is timed."""
    from paper_2205_10879_gb300 import _binding as fb
    from paper_2205_10879_gb300 import serving, workloads as wl
    specs = wl.serving_models()
    models, fits = [], []
    t0 = time.perf_counter()
    for s in specs:
        tm = {}
        c0 = fb.diag_counter(1)
        models.append(serving.fit_model(s["X"], s["Y"], s["k"], s["kernel"], fb.PREC_MIXED,
                                        timings=tm))
        tm.update(n=int(s["X"].shape[0]), d=int(s["X"].shape[1]), k=int(s["k"]),
                  tensor_core_knn=bool(fb.diag_counter(1) > c0))
        if tm["tensor_core_knn"]:
            tm["uncertified_queries"] = fb.diag_counter(2)
        fits.append(tm)
    fit_s = time.perf_counter() - t0
    srv = fb.FmgpServer(models, device_budget_bytes=4 << 30, host_staging_bytes=2 << 30,
                        streams=4, max_batch_points=a.serving_piece)
    # saturation: a burst of requests all at once
    lat, pts, wall, sz = serving.run_poisson(srv, models, 0.0, max(40, a.serving_requests // 4), 11)
    sat = serving.latency_summary(lat, pts, wall, sz)
    req_rate = sat["requests"] / sat["wall_s"]
    out = {"models": fits, "fit_seconds": fit_s, "streams": 4, "piece_points": a.serving_piece,
           "saturation": sat}
    for frac in (0.25, 0.5, 0.75, 0.9):
        lat, pts, wall, sz = serving.run_poisson(srv, models, frac * req_rate, a.serving_requests,
                                                 12 + int(frac * 100))
        out[f"load_{int(frac * 100)}"] = serving.latency_summary(lat, pts, wall, sz)
    st = srv.stats()
    # batches hold pieces of one model up to piece_points points; a piece of a
    # large request fills one alone, small requests share one
    st["mean_batch_points"] = st["points"] / st["batches"] if st["batches"] else 0.0
    out["server"] = st
    srv.close()
    for m in models:
        m.close()
    return out


# ------------------------------------------------------------- oracle ----
def oracle_full(W, min_seconds=10.0, max_repeats=4):
    """Time the FP64 oracle on the whole workload: self kNN table and
    precompute of every training point, 1-NN + prediction of every test
    point, LOOCV over the batch (nothing extrapolated).  The step is repeated
    until about min_seconds of CPU work have been timed."""
    import oracle
    ok = oracle.kernel(W.kernel.kind, W.kernel.nu, W.kernel.length_scale, W.kernel.variance,
                       W.kernel.nugget)
    ph = np.zeros(4)
    reps = 0
    while reps < max_repeats and (reps == 0 or ph.sum() < min_seconds):
        t0 = time.perf_counter()
        nbr, _ = oracle.self_knn(W.X, W.k)
        t1 = time.perf_counter()
        C, _ = oracle.precompute(W.X, W.Y, nbr, W.k, ok)
        t2 = time.perf_counter()
        yo, _ = oracle.predict(W.X, nbr, C, ok, W.Z)
        t3 = time.perf_counter()
        oracle.loocv(W.X, W.Y, nbr, W.k, W.batch, ok)
        t4 = time.perf_counter()
        ph += np.array([t1 - t0, t2 - t1, t3 - t2, t4 - t3])
        reps += 1
    ph /= reps
    return {"value": (W.n + W.m) / ph.sum(), "unit": "points/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"the whole workload, {reps} times: {W.n} training rows (kNN + precompute), "
                      f"{W.m} test points (1-NN + predict), {len(W.batch)} LOOCV points; "
                      f"nothing extrapolated",
            "sample_seconds": float(ph.sum() * reps),
            "precompute_pts_per_s": W.n / ph[1], "predictions_per_s": W.m / ph[2],
            "knn_queries_per_s": W.n / ph[0], "_predictions": yo}


def oracle_sample(W, a, samples):
    """Time the FP64 oracle on a bounded sample: kNN + precompute for s1
    training rows, 1-NN + prediction for s2 test points, LOOCV for s3 batch
    points; extrapolate each phase to the full workload."""
    import oracle
    s1, s2, s3 = min(samples[0], W.n), min(samples[1], W.m), min(samples[2], samples[0], W.n)
    rng = np.random.default_rng(7)
    ok = oracle.kernel(W.kernel.kind, W.kernel.nu, W.kernel.length_scale, W.kernel.variance,
                       W.kernel.nugget)
    rows = np.sort(rng.choice(W.n, s1, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    nb_rows, _ = oracle.knn(W.X, W.X[rows], W.k, rows)
    t1 = time.perf_counter()
    nbr = np.zeros((W.n, W.k), np.int32)
    nbr[rows] = nb_rows
    oracle.precompute(W.X, W.Y, nbr, W.k, ok, rows=rows)
    t2 = time.perf_counter()
    # prediction: 1-NN scan + gather-dot (coefficients of arbitrary value: cost is the same)
    tz = rng.choice(W.m, s2, replace=False)
    near, _ = oracle.knn(W.X, W.Z[tz], 1)
    C = np.zeros((W.n, W.k, 1))
    # j* is taken from the sampled rows (whose neighbour table exists); the work is identical
    oracle.predict_given(W.X, nbr, C, ok, W.Z[tz], rows[np.arange(s2) % s1].astype(np.int32))
    t3 = time.perf_counter()
    lb = rows[:s3]
    oracle.loocv(W.X, W.Y, nbr, W.k, lb, ok)
    t4 = time.perf_counter()
    per_knn = (t1 - t0) / s1
    per_pre = (t2 - t1) / s1
    per_pred = (t3 - t2) / s2
    per_loo = (t4 - t3) / s3
    b = len(W.batch)
    step_s = W.n * (per_knn + per_pre) + W.m * per_pred + b * per_loo
    return {"value": (W.n + W.m) / step_s, "unit": "points/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"{s1} training rows (kNN + precompute), {s2} test points (1-NN + predict), "
                      f"{s3} LOOCV points of the same workload; extrapolated per point",
            "sample_seconds": t4 - t0,
            "precompute_pts_per_s": 1.0 / per_pre, "predictions_per_s": 1.0 / per_pred,
            "knn_queries_per_s": 1.0 / per_knn}


def oracle_baseline(W, a):
    """The spatial workload is timed whole (a few seconds on 16 cores); the
    10^7-point workload on a sample of about the same cost, extrapolated.
    A one-thread run of a small sample is reported beside it."""
    import oracle
    if a.workload == "large":
        r = oracle_sample(W, a, samples=(6000, 6000, 2000))
    else:
        r = oracle_full(W)
    cores = oracle.max_threads()
    oracle.set_threads(1)
    try:
        one = oracle_sample(W, a, samples=(300, 300, 100) if a.workload == "large"
                            else (2000, 2000, 500))
    finally:
        oracle.set_threads(cores)
    r["single_thread"] = {"value": one["value"], "unit": "points/s", "cores": 1,
                          "sample": one["sample"], "sample_seconds": one["sample_seconds"]}
    return r


def run_reference(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2205_10879_gb300 import workloads as wl
    W = make_workload(a)
    res = []
    for i in range(a.warmup + a.steps):
        # one step = one pass of the oracle over the workload (the large
        # workload: one extrapolated sample)
        r = oracle_sample(W, a, samples=(6000, 6000, 2000)) if a.workload == "large" \
            else oracle_full(W, min_seconds=0.0, max_repeats=1)
        r.pop("_predictions", None)
        if i >= a.warmup:
            res.append(r)
    v = float(np.mean([r["value"] for r in res]))
    cpu = dict(res[-1])
    cpu["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s",
            "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": (W.n + W.m) / v * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(a), "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _free_port():
    import socket
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    return port


def relaunch_replicas(a):
    """--gpus N > 1 outside torchrun: run this same command as N ranks (one per
    GPU; RANK, LOCAL_RANK, WORLD_SIZE and a rendezvous on 127.0.0.1 in the
    environment, as torchrun sets them) and return the first non-zero exit
    status; inside torchrun check that the world size is the one asked for."""
    ws = os.environ.get("WORLD_SIZE")
    if a.gpus > 1 and ws is None:
        port = str(_free_port())
        procs = []
        for r in range(a.gpus):
            env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(a.gpus),
                       LOCAL_WORLD_SIZE=str(a.gpus), MASTER_ADDR="127.0.0.1", MASTER_PORT=port)
            procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__)] + sys.argv[1:],
                                          env=env))
        rcs = [p.wait() for p in procs]
        return next((rc for rc in rcs if rc != 0), 0)
    if ws is not None and int(ws) != a.gpus and a.gpus != 1:
        sys.stderr.write(f"bench.py: --gpus {a.gpus} but WORLD_SIZE={ws}\n")
        return 2
    return None


def main():
    a = parse()
    rc = relaunch_replicas(a)
    if rc is not None:
        sys.exit(rc)
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "highdim":
        import torch
        from paper_2205_10879_gb300 import _binding as fb
        fb.load()
        print(json.dumps(highdim_bench(a, torch.device("cuda", 0), max(2, a.steps))))
    elif a.workload == "highdim-knn":
        import torch
        from paper_2205_10879_gb300 import _binding as fb
        fb.load()
        print(json.dumps(highdim_knn_bench(a, torch.device("cuda", 0), a.steps, a.warmup)))
    elif a.workload == "nearest-d64":
        import torch
        from paper_2205_10879_gb300 import _binding as fb
        fb.load()
        print(json.dumps(nearest_bench(a, torch.device("cuda", 0), a.steps, a.warmup)))
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
