"""Shared helpers of the GPU parity tests: run the CUDA path through the
C ABI and the oracle on the same seeded inputs, and compare."""
import numpy as np
import torch

import oracle
from paper_2205_10879_gb300 import _binding as fb

FP64_TOL = 1e-10   # rel-RMS of means, FP64 path vs the FP64 oracle
MIXED_TOL = 1e-5   # rel-RMS of means, mixed path vs the FP64 oracle


def rel_rms(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def kern_pair(spec):
    """(oracle kernel, library kernel) for a workloads.KernelSpec."""
    ok = oracle.kernel(spec.kind, spec.nu, spec.length_scale, spec.variance, spec.nugget)
    gk = fb.make_kernel(spec.kind, spec.nu, spec.length_scale, spec.variance, spec.nugget)
    return ok, gk


def coeffs_to_f64(C, precision):
    C = C.cpu()
    if precision == fb.PREC_FP64:
        return C.numpy()
    c = C.numpy().astype(np.float64)
    return c[..., 0] + c[..., 1]
