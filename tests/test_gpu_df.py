"""The double-float primitives of the mixed-precision path (pairs of FP32
numbers, about 48 significant bits), run on the device through the
diagnostic entry point fmgp_df_eval and checked against FP64 numpy over the
argument ranges the kernels use: exp(-a) for a in [0, 88) (a = sqrt(2 nu) d / rho
or d^2 / (2 rho^2)) and sqrt(D) for squared distances D.  The bound asserted
is the one the kernels are written for: relative error below 1e-13 (for
exp(-a) with a < 32; beyond, where exp(-a) < 1.3e-14, FP32 accuracy, i.e. an
absolute error below 5e-19)."""
import numpy as np
import pytest
import torch

from paper_2205_10879_gb300 import _binding as fb
from gpu_helpers import dev

pytestmark = pytest.mark.gpu


def _as_pair(x):
    """The FP64 value of the double-float pair the kernel forms from x."""
    hi = x.astype(np.float32).astype(np.float64)
    lo = (x - hi).astype(np.float32).astype(np.float64)
    return hi + lo


def _exp_args():
    rng = np.random.default_rng(31)
    parts = [rng.uniform(0.0, 88.0, 200_000), rng.uniform(0.0, 1.0, 50_000),
             rng.uniform(0.0, 1e-3, 10_000), np.exp(rng.uniform(-40.0, 0.0, 10_000)),
             np.arange(0, 88 * 256) / 256.0,                  # table points exactly
             np.arange(1, 88 * 256) / 256.0 - 1e-9,           # just below them
             np.array([0.0, 5e-324, 1e-30, 87.999999, 60.0])]
    return np.concatenate(parts)


def test_df_exp_neg_relative_error(cuda):
    x = _exp_args()
    y = fb.df_eval("exp_neg", dev(x)).cpu().numpy()
    xd = _as_pair(x)
    ref = np.exp(-xd)
    err = np.abs(y - ref)
    table = x.astype(np.float32) < 32.0  # the rule is applied to the high half of the pair
    rel = err[table] / ref[table]
    assert rel.max() < 1e-13, (rel.max(), x[table][np.argmax(rel)])
    # beyond 32 (values below 1.3e-14): FP32 accuracy, absolute error tiny
    normal = ~table & (ref > 1e-37)  # FP32 normal range
    assert (err[normal] / ref[normal]).max() < 2e-5
    assert err[~table].max() < 5e-19  # exp(-32) * 2e-5 = 2.5e-19


def test_df_exp_neg_out_of_range_is_zero(cuda):
    x = np.array([88.0, 88.5, 100.0, 1e30, np.inf, np.nan])
    y = fb.df_eval("exp_neg", dev(x)).cpu().numpy()
    assert np.all(y == 0.0)


def test_df_sqrt_relative_error(cuda):
    rng = np.random.default_rng(32)
    x = np.concatenate([np.exp(rng.uniform(np.log(1e-12), np.log(1e6), 200_000)),
                        rng.uniform(0.0, 4.0, 50_000), np.array([1.0, 4.0, 2.0, 1e-30])])
    y = fb.df_eval("sqrt", dev(x)).cpu().numpy()
    ref = np.sqrt(_as_pair(x))
    rel = np.abs(y - ref) / ref
    assert rel.max() < 1e-13, (rel.max(), x[np.argmax(rel)])
    z = fb.df_eval("sqrt", dev(np.array([0.0, -1.0, -1e-30]))).cpu().numpy()
    assert np.all(z == 0.0)
