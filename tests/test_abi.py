"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no GPU needed: nothing is called that computes)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2205_10879_gb300 import build as fbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fmgp_[a-z0-9_]+)\s*\(", text):
            syms.add(m.group(1))
    return syms


def test_header_declares_the_four_path_entry_points():
    syms = declared_symbols()
    for s in ["fmgp_build_knn", "fmgp_precompute", "fmgp_predict", "fmgp_loocv_objective",
              "fmgp_last_error"]:
        assert s in syms


def test_library_exports_every_declared_symbol():
    path = fbuild.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in sorted(declared_symbols()) if not hasattr(lib, s)]
    assert not missing, missing


def test_version_and_error_calls_need_no_gpu():
    lib = ctypes.CDLL(fbuild.build())
    lib.fmgp_version.restype = ctypes.c_char_p
    lib.fmgp_last_error.restype = ctypes.c_char_p
    assert lib.fmgp_version().decode().count(".") == 2
    assert isinstance(lib.fmgp_last_error(), bytes)


def test_argument_errors_are_caught_on_the_host():
    """Bad arguments return FMGP_EINVAL before any CUDA call (so this runs without a GPU)."""
    from paper_2205_10879_gb300 import _binding as b
    lib = b.load()
    P = ctypes.c_void_p
    fake = P(16)  # never dereferenced: validation fails first
    k = b.make_kernel("matern", 1.5, 0.1, 1.0, 1e-4)
    # kq > n - 1
    assert lib.fmgp_build_knn(fake, b.F64, 10, 2, 10, fake, None, 0, None) == b.FMGP_EINVAL
    # n < 2, d < 1, null X
    assert lib.fmgp_build_knn(fake, b.F64, 1, 2, 1, fake, None, 0, None) == b.FMGP_EINVAL
    assert lib.fmgp_build_knn(fake, b.F64, 10, 0, 1, fake, None, 0, None) == b.FMGP_EINVAL
    assert lib.fmgp_build_knn(None, b.F64, 10, 2, 1, fake, None, 0, None) == b.FMGP_EINVAL
    # unsupported nu / negative nugget / bad precision
    bad_nu = b.make_kernel("matern", 1.0, 0.1, 1.0, 1e-4)
    neg_nug = b.make_kernel("matern", 1.5, 0.1, 1.0, -1e-4)
    for kk in (bad_nu, neg_nug):
        rc = lib.fmgp_precompute(fake, b.F64, fake, 100, 2, 1, fake, 29, 30, ctypes.byref(kk),
                                 b.PREC_FP64, fake, None, None)
        assert rc == b.FMGP_EINVAL
    assert lib.fmgp_precompute(fake, b.F64, fake, 100, 2, 1, fake, 29, 30, ctypes.byref(k), 7,
                               fake, None, None) == b.FMGP_EINVAL
    # k > n, nbr_ld < k-1
    assert lib.fmgp_precompute(fake, b.F64, fake, 10, 2, 1, fake, 29, 30, ctypes.byref(k),
                               b.PREC_FP64, fake, None, None) == b.FMGP_EINVAL
    assert lib.fmgp_precompute(fake, b.F64, fake, 100, 2, 1, fake, 20, 30, ctypes.byref(k),
                               b.PREC_FP64, fake, None, None) == b.FMGP_EINVAL
    # LOOCV needs nbr_ld >= k and b >= 1
    q = ctypes.c_double(0)
    assert lib.fmgp_loocv_objective(fake, b.F64, fake, 100, 2, 1, fake, 29, 30, fake, 10,
                                    ctypes.byref(k), b.PREC_FP64, ctypes.byref(q), None,
                                    None) == b.FMGP_EINVAL
    assert lib.fmgp_loocv_objective(fake, b.F64, fake, 100, 2, 1, fake, 30, 30, fake, 0,
                                    ctypes.byref(k), b.PREC_FP64, ctypes.byref(q), None,
                                    None) == b.FMGP_EINVAL
    # predict: m < 0
    assert lib.fmgp_predict(fake, b.F64, 100, 2, fake, 29, fake, 30, 1, ctypes.byref(k),
                            b.PREC_FP64, fake, -1, fake, None, None) == b.FMGP_EINVAL
    assert b"m = -1" in lib.fmgp_last_error()
    # model: flags other than borrow (0) / copy (1)
    h = ctypes.c_void_p(16)
    assert lib.fmgp_model_create(fake, b.F64, 100, 2, fake, 29, fake, 30, 1, ctypes.byref(k),
                                 b.PREC_FP64, 2, ctypes.byref(h), None) == b.FMGP_EINVAL
    assert h.value is None and b"flags = 2" in lib.fmgp_last_error()


def test_tuning_keys_are_host_only_and_range_checked():
    """Launch-shape and path controls: defaults, round trip, refusal of
    unknown keys and out-of-range values (host code only)."""
    from paper_2205_10879_gb300 import _binding as b
    lib = b.load()
    lib.fmgp_tune_get.restype = ctypes.c_double
    lib.fmgp_tune_set.argtypes = [ctypes.c_char_p, ctypes.c_double]
    lib.fmgp_tune_get.argtypes = [ctypes.c_char_p]
    defaults = {b"tensor_cores": 1.0, b"tc_fused_select": 1.0, b"tc_oversample": 4.0,
                b"block_warps": 0.0, b"count_visits": 0.0, b"tc_fused_r": 0.0,
                b"block_persistent": -1.0}
    for key, v in defaults.items():
        assert lib.fmgp_tune_get(key) == v, key
    assert lib.fmgp_tune_get(b"no_such_key") == -1.0
    assert lib.fmgp_tune_set(b"no_such_key", 1.0) == b.FMGP_EINVAL
    for key, bad in ((b"tc_oversample", 1.0), (b"tc_oversample", 5.0), (b"block_warps", 9.0),
                     (b"grid_target", 0.5), (b"tc_fused_r", 12.0), (b"block_persistent", 2.0),
                     (b"block_persistent", 0.5)):
        assert lib.fmgp_tune_set(key, bad) == b.FMGP_EINVAL, key
        assert lib.fmgp_tune_get(key) == defaults.get(key, 12.0)
    try:
        assert lib.fmgp_tune_set(b"tc_oversample", 3.0) == 0
        assert lib.fmgp_tune_get(b"tc_oversample") == 3.0
        assert lib.fmgp_tune_set(b"tc_fused_select", 0.0) == 0
        assert lib.fmgp_tune_get(b"tc_fused_select") == 0.0
        assert lib.fmgp_tune_set(b"block_persistent", 0.0) == 0
        assert lib.fmgp_tune_get(b"block_persistent") == 0.0
    finally:
        lib.fmgp_tune_set(b"tc_oversample", 4.0)
        lib.fmgp_tune_set(b"tc_fused_select", 1.0)
        lib.fmgp_tune_set(b"block_persistent", -1.0)
