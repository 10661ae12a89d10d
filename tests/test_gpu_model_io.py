"""Fitted models saved to a file and loaded back (fmgp_model_save /
fmgp_model_load): the loaded model predicts bit-identically to the one that
was saved, for every nearest-point search (grid at d <= 3, scan at
4 <= d <= 15, tensor cores at d >= 16), both precision forms and both input
dtypes; a damaged file is refused."""
import os

import numpy as np
import pytest
import torch

from paper_2205_10879_gb300 import _binding as fb
from gpu_helpers import dev

pytestmark = pytest.mark.gpu


def _fit(n, d, k, prec, dtype, seed):
    rng = np.random.default_rng(seed)
    X = rng.random((n, d)).astype(dtype)
    Y = np.stack([np.sin(4 * X[:, 0]), np.cos(3 * X[:, -1])], axis=1).astype(np.float64)
    kern = fb.make_kernel("matern", 1.5, 0.3 * np.sqrt(d), 1.3, 1e-3)
    Xd, Yd = dev(X), dev(Y)
    if k > 1:
        nbr, _ = fb.fmgp_build_knn(Xd, k - 1)
    else:  # S_i = [i]: the table is not read
        nbr = torch.zeros((n, 1), dtype=torch.int32, device="cuda")
    C, _ = fb.fmgp_precompute(Xd, Yd, nbr, k, kern, prec)
    return fb.FmgpModel(Xd, nbr, C, k, kern, prec), rng


@pytest.mark.parametrize("d,dtype,prec", [(2, np.float64, fb.PREC_MIXED),
                                          (3, np.float32, fb.PREC_FP64),
                                          (8, np.float64, fb.PREC_FP64),
                                          (24, np.float32, fb.PREC_MIXED)])
def test_saved_model_predicts_identically(cuda, tmp_path, d, dtype, prec):
    model, rng = _fit(6000, d, 24, prec, dtype, d)
    Z = dev(rng.random((700, d)).astype(dtype))
    y0, j0 = model.predict(Z)
    path = tmp_path / "model.fmgp"
    model.save(path)
    loaded = fb.FmgpModel.load(path)
    assert (loaded.n, loaded.d, loaded.r, loaded.k) == (6000, d, 2, 24)
    assert loaded.precision == prec and loaded.dtype == model.dtype
    assert abs(loaded.kernel.length_scale - model.kernel.length_scale) == 0
    model.close()  # the loaded model owns its own copies
    y1, j1 = loaded.predict(Z)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1) and torch.equal(j0, j1)
    loaded.close()


def test_single_point_neighbourhood_model_has_no_table(cuda, tmp_path):
    model, rng = _fit(3000, 2, 1, fb.PREC_FP64, np.float64, 5)
    Z = dev(rng.random((100, 2)))
    y0, _ = model.predict(Z)
    model.save(tmp_path / "k1.fmgp")
    size = os.path.getsize(tmp_path / "k1.fmgp")
    assert size == 128 + 3000 * 2 * 8 + 3000 * 1 * 2 * 8  # header, X, C: no neighbour table
    loaded = fb.FmgpModel.load(tmp_path / "k1.fmgp")
    y1, _ = loaded.predict(Z)
    assert torch.equal(y0, y1)
    loaded.close()
    model.close()


def test_damaged_or_truncated_file_is_refused(cuda, tmp_path):
    model, _ = _fit(2000, 2, 10, fb.PREC_FP64, np.float64, 9)
    path = tmp_path / "m.fmgp"
    model.save(path)
    model.close()
    data = bytearray(path.read_bytes())
    bad = bytearray(data)
    bad[128 + 5000] ^= 0x01  # one bit of X
    (tmp_path / "bad.fmgp").write_bytes(bytes(bad))
    with pytest.raises(fb.FmgpError) as e:
        fb.FmgpModel.load(tmp_path / "bad.fmgp")
    assert e.value.code == fb.FMGP_EIO and "checksum" in str(e.value)
    (tmp_path / "short.fmgp").write_bytes(bytes(data[:-8]))
    with pytest.raises(fb.FmgpError) as e:
        fb.FmgpModel.load(tmp_path / "short.fmgp")
    assert e.value.code == fb.FMGP_EIO and "truncated" in str(e.value)
    hdr = bytearray(data)
    hdr[40] ^= 0xFF  # the shape fields no longer match the array sizes
    (tmp_path / "hdr.fmgp").write_bytes(bytes(hdr))
    with pytest.raises(fb.FmgpError) as e:
        fb.FmgpModel.load(tmp_path / "hdr.fmgp")
    assert e.value.code == fb.FMGP_EIO


@pytest.mark.parametrize("d,dtype,prec", [(2, np.float64, fb.PREC_MIXED),
                                          (8, np.float32, fb.PREC_FP64)])
def test_copying_model_outlives_the_callers_arrays(cuda, d, dtype, prec):
    """FMGP_MODEL_COPY: the model keeps X, the neighbour table and C in device
    memory of its own.  It predicts bit-identically to a borrowing model, also
    after the caller has overwritten and freed its arrays, and the copies are
    charged to the context bound when the model was created (released with
    the model)."""
    rng = np.random.default_rng(40 + d)
    n, k = 5000, 20
    X = rng.random((n, d)).astype(dtype)
    Y = np.stack([np.sin(4 * X[:, 0]), np.cos(3 * X[:, -1])], axis=1).astype(np.float64)
    kern = fb.make_kernel("matern", 1.5, 0.3 * np.sqrt(d), 1.3, 1e-3)
    Xd, Yd = dev(X), dev(Y)
    nbr, _ = fb.fmgp_build_knn(Xd, k - 1)
    C, _ = fb.fmgp_precompute(Xd, Yd, nbr, k, kern, prec)
    Z = dev(rng.random((600, d)).astype(dtype))
    borrowed = fb.FmgpModel(Xd, nbr, C, k, kern, prec)
    y0, j0 = borrowed.predict(Z)
    torch.cuda.synchronize()
    borrowed.close()
    own = sum(t.numel() * t.element_size() for t in (Xd, nbr, C))
    ctx = fb.Context(64 << 20)
    try:
        with ctx:
            copied = fb.FmgpModel(Xd, nbr, C, k, kern, prec, copy=True)
        assert ctx.bytes_in_use() >= own
        Xd.fill_(7.0)
        nbr.fill_(0)
        C.fill_(float("nan"))
        del Xd, nbr, C
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        y1, j1 = copied.predict(Z)
        torch.cuda.synchronize()
        assert torch.equal(y0, y1) and torch.equal(j0, j1)
        copied.close()
        assert ctx.bytes_in_use() == 0
    finally:
        ctx.close()
