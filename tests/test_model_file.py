"""Model files that are not model files are refused on the host, before any
device call (so this runs without a GPU)."""
import ctypes
import struct

import pytest

from paper_2205_10879_gb300 import _binding as fb


def _load(path):
    lib = fb.load()
    h = ctypes.c_void_p()
    return lib.fmgp_model_load(str(path).encode(), ctypes.byref(h), None), lib.fmgp_last_error()


def test_missing_file(tmp_path):
    rc, msg = _load(tmp_path / "absent.fmgp")
    assert rc == fb.FMGP_EIO and b"cannot open" in msg


def test_not_a_model_file(tmp_path):
    p = tmp_path / "x.fmgp"
    p.write_bytes(b"GIF89a" + bytes(200))
    rc, msg = _load(p)
    assert rc == fb.FMGP_EIO and b"not a model file" in msg
    p.write_bytes(b"FMGPMODL")  # shorter than a header
    rc, _ = _load(p)
    assert rc == fb.FMGP_EIO


def test_unsupported_version(tmp_path):
    p = tmp_path / "v.fmgp"
    p.write_bytes(b"FMGPMODL" + struct.pack("<II", 2, 128) + bytes(112))
    rc, msg = _load(p)
    assert rc == fb.FMGP_EIO and b"version 2" in msg


def test_inconsistent_sizes(tmp_path):
    # version 1 header whose array sizes do not match its shapes
    hdr = b"FMGPMODL" + struct.pack("<IIiiqiiiiii", 1, 128, 1, 0, 100, 2, 1, 5, 4, 0, 0)
    hdr += struct.pack("<dddd", 1.5, 0.1, 1.0, 1e-4) + struct.pack("<QQQQ", 1, 2, 3, 0) + bytes(8)
    assert len(hdr) == 128
    p = tmp_path / "s.fmgp"
    p.write_bytes(hdr)
    rc, msg = _load(p)
    assert rc == fb.FMGP_EIO and b"inconsistent" in msg


def test_null_arguments():
    lib = fb.load()
    h = ctypes.c_void_p()
    assert lib.fmgp_model_load(None, ctypes.byref(h), None) == fb.FMGP_EINVAL
    assert lib.fmgp_model_save(None, b"x", None) == fb.FMGP_EINVAL
